/*
 * mpwsd_oracle.c -- plain FP64 CPU oracle for two-stage near-ML decoding with
 * multipoint code-weight sphere decoding (MP-WSD), arXiv 2602.08501.
 *
 * TEST INFRASTRUCTURE. This file exists to check the GPU library, not to be
 * used by it. Only tests/, __graft_entry__.smoke() and the cpu_baseline /
 * reference legs of bench.py load it. It shares no code, header, table or
 * helper with the CUDA path; the two meet only through inputs produced by the
 * seeded generator in synth/ (or by this oracle) and through their outputs.
 *
 * Everything here is written for clarity, one frame and one path at a time,
 * in FP64 (bits are stored one per byte). What each part restates:
 *   - code model, CRC precoding, BPSK x(c) = 1 - 2c ........ Sec. II-B
 *   - Hamming shells / code-weight sphere / translation ..... Sec. II-C, Eqs. (1)-(3)
 *   - stage 1: list decoding, CRC on the most reliable
 *     candidate, early termination .......................... Sec. III-A
 *   - stage 1 alternative: ordered-statistics decoding
 *     OSD(order) as the anchor list (the RM experiment) ..... Sec. IV-A
 *   - stage 2: MP-WSD update Eq. (4), Algorithm 1 with the
 *     top-m filter by the correlation gain of Eq. (5) and the
 *     exact-ED search, strict-improvement hop, final argmin ... Sec. III-B/C
 *   - filter size m = max(10, ceil(0.02 |S_r(0)|)) ........... Sec. IV-A
 * Readings where the paper is silent (min-sum SCL, CRC bit order, tie rules)
 * are stated beside the code that takes them. All of them are also listed in
 * the design notes of the repository.
 *
 * Exactness: inputs y on the 2^-19 grid with |y| < 16 make every LLR, path
 * metric and gain below an exact FP64 number; ||y - x||^2 is exact whenever
 * it is below 2^15 (always for n <= 64).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAXN 128

/* ------------------------------------------------------------------------ */
/* Code algebra (Sec. II-B)                                                  */
/* ------------------------------------------------------------------------ */

/* F^{(x)m}: Kronecker power of the 2x2 kernel [[1,0],[1,1]], built by the
 * definition of the Kronecker product, block by block. Row-major n x n bytes. */
void or_kron_power(int m, uint8_t *F) {
    int n = 1 << m;
    memset(F, 0, (size_t)n * n);
    F[0] = 1;
    int s = 1; /* current size */
    while (s < n) {
        /* new = [[cur, 0], [cur, cur]] written into the top-left 2s x 2s block */
        for (int i = 0; i < s; i++)
            for (int j = 0; j < s; j++) {
                uint8_t v = F[i * n + j];
                F[(i + s) * n + j] = v;
                F[(i + s) * n + (j + s)] = v;
                F[i * n + (j + s)] = 0;
            }
        s *= 2;
    }
}

/* c = u F^{(x)m} over F2, using the top-left h x h block of F (stride n),
 * which is F^{(x)log2 h}. */
static void encode_block(const uint8_t *F, int n, int h, const uint8_t *u, uint8_t *c) {
    for (int j = 0; j < h; j++) c[j] = 0;
    for (int i = 0; i < h; i++)
        if (u[i])
            for (int j = 0; j < h; j++) c[j] ^= F[i * n + j];
}

/* Reed-Muller RM(r, m) in the Arikan form: row i of F^{(x)m} has weight
 * 2^popcount(i); the code keeps the rows of weight >= 2^(m-r). frozen[i] = 1
 * for the rows it drops. Returns the dimension k. */
int or_rm_frozen(int m, int r, uint8_t *frozen) {
    int n = 1 << m, k = 0;
    for (int i = 0; i < n; i++) {
        int w = 0;
        for (int b = 0; b < m; b++) w += (i >> b) & 1;
        frozen[i] = (uint8_t)(w < m - r);
        k += !frozen[i];
    }
    return k;
}

/* CRC remainder by polynomial long division over F2 (Sec. II-B, CRC precoding).
 * Reading: msg[0] is the coefficient of the highest power, the generator is
 * g(x) = x^len + sum_{b<len} bit_b(poly) x^b, the remainder is that of
 * msg(x) x^len mod g(x), initial value 0, no reflection, no final XOR;
 * r[0] is the coefficient of x^(len-1). */
void or_crc(const uint8_t *msg, int k, uint32_t poly, int len, uint8_t *r) {
    uint8_t d[OR_MAXN + 64];
    for (int i = 0; i < k; i++) d[i] = msg[i] & 1;
    for (int i = 0; i < len; i++) d[k + i] = 0;
    for (int i = 0; i < k; i++) {
        if (!d[i]) continue;
        /* subtract g(x) aligned with the leading term at position i */
        d[i] ^= 1;
        for (int b = 0; b < len; b++) {
            int coef = (int)((poly >> (len - 1 - b)) & 1u); /* coefficient of x^(len-1-b) */
            d[i + 1 + b] ^= (uint8_t)coef;
        }
    }
    for (int i = 0; i < len; i++) r[i] = d[k + i];
}

/* ------------------------------------------------------------------------ */
/* Code handle                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    int n, m, k;
    uint8_t frozen[OR_MAXN];
    int info[OR_MAXN]; /* non-frozen indices, ascending */
    uint8_t *F;        /* n x n */
    int k_info, crc_len;
    uint32_t crc_poly;
    int64_t P;          /* number of patterns */
    uint8_t *pat;       /* P x n bytes */
    int *pat_w;         /* Hamming weights */
    int *pat_supp;      /* P x n: support indices of each pattern, ascending */
    int filter_m;       /* Sec. IV-A: m = max(10, ceil(0.02 |S|)) */
} or_code;

static int bit_of(const uint64_t *words, int j) { return (int)((words[j >> 6] >> (j & 63)) & 1u); }

or_code *or_code_create(int n, const uint8_t *frozen, int k_info, uint32_t crc_poly, int crc_len,
                        const uint64_t *patterns, int64_t n_patterns) {
    int m = 0;
    while ((1 << m) < n) m++;
    if ((1 << m) != n || n > OR_MAXN || n < 2) return NULL;
    or_code *c = (or_code *)calloc(1, sizeof(or_code));
    c->n = n;
    c->m = m;
    c->F = (uint8_t *)malloc((size_t)n * n);
    or_kron_power(m, c->F);
    c->k = 0;
    for (int i = 0; i < n; i++) {
        c->frozen[i] = frozen[i] ? 1 : 0;
        if (!c->frozen[i]) c->info[c->k++] = i;
    }
    c->k_info = k_info;
    c->crc_len = crc_len;
    c->crc_poly = crc_poly;
    c->P = n_patterns;
    int W = (n + 63) / 64;
    c->pat = (uint8_t *)malloc((size_t)(n_patterns > 0 ? n_patterns : 1) * n);
    c->pat_w = (int *)malloc(sizeof(int) * (size_t)(n_patterns > 0 ? n_patterns : 1));
    c->pat_supp = (int *)malloc(sizeof(int) * (size_t)(n_patterns > 0 ? n_patterns : 1) * n);
    for (int64_t p = 0; p < n_patterns; p++) {
        int w = 0;
        for (int j = 0; j < n; j++) {
            uint8_t b = (uint8_t)bit_of(patterns + p * W, j);
            c->pat[p * n + j] = b;
            if (b) c->pat_supp[p * n + w++] = j;
        }
        c->pat_w[p] = w;
    }
    int64_t m2 = (int64_t)ceil(0.02 * (double)n_patterns);
    c->filter_m = (int)(m2 > 10 ? m2 : 10);
    return c;
}

void or_code_free(or_code *c) {
    if (!c) return;
    free(c->F);
    free(c->pat);
    free(c->pat_w);
    free(c->pat_supp);
    free(c);
}

int or_code_filter_m(const or_code *c) { return c->filter_m; }

/* u -> codeword c = u F^{(x)m} */
void or_encode(const or_code *c, const uint8_t *u, uint8_t *cw) { encode_block(c->F, c->n, c->n, u, cw); }

/* Does codeword cw pass the CRC? F^{(x)m} is its own inverse over F2, so
 * u = cw F^{(x)m}; the CRC is taken over v = u at the non-frozen indices,
 * v = [message (k_info bits), parity (crc_len bits)]. Returns 1 when the
 * frozen positions are zero and the parity matches. */
static int crc_ok_codeword(const or_code *c, const uint8_t *cw) {
    uint8_t u[OR_MAXN], v[OR_MAXN], r[64];
    encode_block(c->F, c->n, c->n, cw, u);
    for (int i = 0; i < c->n; i++)
        if (c->frozen[i] && u[i]) return 0;
    for (int t = 0; t < c->k; t++) v[t] = u[c->info[t]];
    if (c->crc_len == 0) return 1;
    or_crc(v, c->k_info, c->crc_poly, c->crc_len, r);
    for (int b = 0; b < c->crc_len; b++)
        if (r[b] != v[c->k_info + b]) return 0;
    return 1;
}

int or_crc_ok_codeword(const or_code *c, const uint8_t *cw) { return crc_ok_codeword(c, cw); }

/* ------------------------------------------------------------------------ */
/* Stage 1: min-sum SC-list decoding (Sec. III-A)                            */
/* ------------------------------------------------------------------------ */
/* Reading: the paper names "LLR-based SCL" without formulas. We take the
 * min-sum check-node update f(a,b) = sign(a) sign(b) min(|a|,|b|) with
 * sign(0) = +1, the variable-node update g(a,b,beta) = b + (1 - 2 beta) a,
 * channel LLR lambda_j = y_j (the scale 2/sigma^2 does not change any
 * decision of min-sum SCL), hard decision HD(l) = 0 if l >= 0 else 1, and the
 * path metric PM += |l| when the decided bit differs from HD(l). */

static double f_minsum(double a, double b) {
    double sa = a >= 0 ? 1.0 : -1.0, sb = b >= 0 ? 1.0 : -1.0;
    double ma = fabs(a), mb = fabs(b);
    return sa * sb * (ma < mb ? ma : mb);
}

/* LLR of the leaf with relative index i inside a node of size S whose
 * channel-side LLRs are lam[0..S-1], given the decisions u[0..i-1] of the
 * node's leaves. Computed from scratch by descending the tree: the left half
 * of the node carries a XOR b, the right half carries b (c = [(a^b)F', bF']). */
static double leaf_llr(const uint8_t *F, int n, const double *lam, int S, const uint8_t *u, int i) {
    if (S == 1) return lam[0];
    int h = S / 2;
    double child[OR_MAXN / 2];
    if (i < h) {
        for (int j = 0; j < h; j++) child[j] = f_minsum(lam[j], lam[j + h]);
        return leaf_llr(F, n, child, h, u, i);
    }
    uint8_t beta[OR_MAXN / 2];
    encode_block(F, n, h, u, beta); /* re-encoding of the decided left half */
    for (int j = 0; j < h; j++) child[j] = lam[j + h] + (beta[j] ? -lam[j] : lam[j]);
    return leaf_llr(F, n, child, h, u + h, i - h);
}

/* All n leaf LLRs for a fixed decision vector u (used by tests that evaluate
 * the path metric of every message by brute force). */
void or_leaf_llrs(const or_code *c, const double *y, const uint8_t *u, double *out) {
    for (int i = 0; i < c->n; i++) out[i] = leaf_llr(c->F, c->n, y, c->n, u, i);
}

typedef struct {
    double pm;
    int parent;
    int u;
} scl_cand;

static int cand_cmp(const void *pa, const void *pb) {
    const scl_cand *a = (const scl_cand *)pa, *b = (const scl_cand *)pb;
    if (a->pm < b->pm) return -1;
    if (a->pm > b->pm) return 1;
    if (a->parent != b->parent) return a->parent < b->parent ? -1 : 1;
    return a->u < b->u ? -1 : (a->u > b->u ? 1 : 0);
}

/* SC-list decode of one frame. Reading of the list management: at an info
 * leaf each path spawns u = 0 and u = 1; the 2|list| children are ordered by
 * (PM, parent position in the current list, u) ascending and the first
 * min(2|list|, L) are kept. At the end the list is stably sorted by PM.
 * Outputs u_list (count x n bytes) and pm_list, best first. Returns count. */
int or_scl(const or_code *c, const double *y, int L, uint8_t *u_list, double *pm_list) {
    int n = c->n;
    if (L < 1) return 0;
    uint8_t *u = (uint8_t *)calloc((size_t)L * n, 1), *u2 = (uint8_t *)calloc((size_t)L * n, 1);
    double *pm = (double *)calloc((size_t)L, sizeof(double)), *pm2 = (double *)calloc((size_t)L, sizeof(double));
    double *lam = (double *)calloc((size_t)L, sizeof(double));
    scl_cand *cand = (scl_cand *)malloc(sizeof(scl_cand) * 2 * (size_t)L);
    int count = 1;
    for (int i = 0; i < n; i++) {
        for (int p = 0; p < count; p++) lam[p] = leaf_llr(c->F, n, y, n, u + (size_t)p * n, i);
        if (c->frozen[i]) {
            for (int p = 0; p < count; p++) {
                u[(size_t)p * n + i] = 0;
                if (lam[p] < 0) pm[p] += fabs(lam[p]);
            }
            continue;
        }
        int nc = 0;
        for (int p = 0; p < count; p++)
            for (int b = 0; b < 2; b++) {
                int hd = lam[p] >= 0 ? 0 : 1;
                cand[nc].pm = pm[p] + (b != hd ? fabs(lam[p]) : 0.0);
                cand[nc].parent = p;
                cand[nc].u = b;
                nc++;
            }
        qsort(cand, (size_t)nc, sizeof(scl_cand), cand_cmp);
        int keep = nc < L ? nc : L;
        for (int q = 0; q < keep; q++) {
            memcpy(u2 + (size_t)q * n, u + (size_t)cand[q].parent * n, (size_t)n);
            u2[(size_t)q * n + i] = (uint8_t)cand[q].u;
            pm2[q] = cand[q].pm;
        }
        uint8_t *tu = u; u = u2; u2 = tu;
        double *tp = pm; pm = pm2; pm2 = tp;
        count = keep;
    }
    /* final stable sort by PM (insertion sort keeps equal keys in list order) */
    int *ord = (int *)malloc(sizeof(int) * (size_t)count);
    for (int q = 0; q < count; q++) ord[q] = q;
    for (int q = 1; q < count; q++) {
        int v = ord[q], t = q - 1;
        while (t >= 0 && pm[ord[t]] > pm[v]) { ord[t + 1] = ord[t]; t--; }
        ord[t + 1] = v;
    }
    for (int q = 0; q < count; q++) {
        memcpy(u_list + (size_t)q * n, u + (size_t)ord[q] * n, (size_t)n);
        pm_list[q] = pm[ord[q]];
    }
    free(ord);
    free(u); free(u2); free(pm); free(pm2); free(lam); free(cand);
    return count;
}

/* ------------------------------------------------------------------------ */
/* Code-weight sphere S_r(0) \ {0}: enumeration of codewords (Sec. II-C)     */
/* ------------------------------------------------------------------------ */
/* Partial codewords for message halves: a k-bit message integer a (info bit t
 * at bit k-1-t, i.e. the lowest info index is the most significant bit) is
 * split as a = hi * 2^kl + lo; its codeword is Thi[hi] ^ Tlo[lo]. */
typedef struct {
    int kl, kh;
    uint64_t (*Tlo)[2];
    uint64_t (*Thi)[2];
} half_tables;

static void half_tables_build(const or_code *c, half_tables *t) {
    int n = c->n, k = c->k;
    uint64_t G[64][2];
    for (int r = 0; r < k; r++) {
        G[r][0] = G[r][1] = 0;
        for (int j = 0; j < n; j++)
            if (c->F[c->info[r] * n + j]) G[r][j >> 6] |= 1ull << (j & 63);
    }
    t->kl = k / 2;
    t->kh = k - t->kl;
    t->Tlo = malloc(sizeof(uint64_t[2]) * ((size_t)1 << t->kl));
    t->Thi = malloc(sizeof(uint64_t[2]) * ((size_t)1 << t->kh));
    for (uint64_t x = 0; x < (1ull << t->kl); x++) {
        t->Tlo[x][0] = t->Tlo[x][1] = 0;
        for (int b = 0; b < t->kl; b++)
            if ((x >> b) & 1ull) { t->Tlo[x][0] ^= G[k - 1 - b][0]; t->Tlo[x][1] ^= G[k - 1 - b][1]; }
    }
    for (uint64_t x = 0; x < (1ull << t->kh); x++) {
        t->Thi[x][0] = t->Thi[x][1] = 0;
        for (int b = 0; b < t->kh; b++)
            if ((x >> b) & 1ull) {
                t->Thi[x][0] ^= G[k - 1 - (b + t->kl)][0];
                t->Thi[x][1] ^= G[k - 1 - (b + t->kl)][1];
            }
    }
}

static void half_tables_free(half_tables *t) {
    free(t->Tlo);
    free(t->Thi);
}

/* All codewords of the given weights, in the order (weight ascending, then
 * the message integer), where the message integer of a codeword is its info
 * vector (u at the non-frozen indices, ascending) read with the lowest index
 * as the most significant bit. Written bit-packed (bit j of word j/64 = c_j).
 * If out is NULL only counts. Returns the number of codewords found, or -1
 * if max_out is too small. Brute force over all 2^k messages. */
int64_t or_enumerate(const or_code *c, const int *weights, int n_weights, uint64_t *out, int64_t max_out) {
    int W = (c->n + 63) / 64;
    half_tables t;
    half_tables_build(c, &t);
    int64_t total = 0;
    for (int wi = 0; wi < n_weights; wi++) {
        int wt = weights[wi];
        for (uint64_t hi = 0; hi < (1ull << t.kh); hi++)
            for (uint64_t lo = 0; lo < (1ull << t.kl); lo++) {
                uint64_t c0 = t.Thi[hi][0] ^ t.Tlo[lo][0], c1 = t.Thi[hi][1] ^ t.Tlo[lo][1];
                if (__builtin_popcountll(c0) + __builtin_popcountll(c1) != wt) continue;
                if (out) {
                    if (total >= max_out) { half_tables_free(&t); return -1; }
                    out[total * W] = c0;
                    if (W > 1) out[total * W + 1] = c1;
                }
                total++;
            }
    }
    half_tables_free(&t);
    return total;
}

/* Weight distribution A_w, w = 0..n, by brute force over all 2^k messages. */
void or_weight_distribution(const or_code *c, int64_t *A) {
    for (int w = 0; w <= c->n; w++) A[w] = 0;
    half_tables t;
    half_tables_build(c, &t);
    for (uint64_t hi = 0; hi < (1ull << t.kh); hi++)
        for (uint64_t lo = 0; lo < (1ull << t.kl); lo++)
            A[__builtin_popcountll(t.Thi[hi][0] ^ t.Tlo[lo][0]) + __builtin_popcountll(t.Thi[hi][1] ^ t.Tlo[lo][1])]++;
    half_tables_free(&t);
}

/* ------------------------------------------------------------------------ */
/* Stage 2: MP-WSD, Algorithm 1 (Sec. III-B) with the filter of Eq. (5)      */
/* ------------------------------------------------------------------------ */

static double sq_dist(const double *y, const uint8_t *cw, int n) {
    double s = 0.0;
    for (int j = 0; j < n; j++) {
        double d = y[j] - (1.0 - 2.0 * cw[j]);
        s += d * d;
    }
    return s;
}

typedef struct {
    int iters;           /* iterations of the outer loop that ran */
    double min_gap;      /* smallest ED gap between the chosen and the runner-up, over all decisions */
    int64_t evals;       /* (active trajectory, pattern) pairs scored by the filter */
    /* The same count without retired twins. A trajectory is retired when, right
     * after a hop, it sits on the centre of a live lower-numbered trajectory of
     * the frame. Live means that trajectory hopped there in the same iteration
     * or stopped there, and is not retired itself. From then on the two make
     * the same decisions, or the row would stop next anyway, so the GPU scores
     * only the lower one. This counts work only: nothing of the algorithm
     * above changes. */
    int64_t evals_distinct;
    int final_k;         /* winning path */
} wsd_info;

/* Min-heap of the m best gains seen so far: the root is the weakest kept entry
 * (smallest gain; among equal gains, the largest pattern index). */
typedef struct {
    double g;
    int64_t p;
} gain_ent;

static int weaker(const gain_ent *a, const gain_ent *b) {
    if (a->g != b->g) return a->g < b->g;
    return a->p > b->p;
}

static void heap_sift_down(gain_ent *h, int size, int i) {
    for (;;) {
        int l = 2 * i + 1, r = l + 1, s = i;
        if (l < size && weaker(&h[l], &h[s])) s = l;
        if (r < size && weaker(&h[r], &h[s])) s = r;
        if (s == i) return;
        gain_ent t = h[i]; h[i] = h[s]; h[s] = t;
        i = s;
    }
}

static void heap_sift_up(gain_ent *h, int i) {
    while (i > 0) {
        int parent = (i - 1) / 2;
        if (!weaker(&h[i], &h[parent])) return;
        gain_ent t = h[i]; h[i] = h[parent]; h[parent] = t;
        i = parent;
    }
}

/* One frame of Algorithm 1. anchors: count x n bytes (list order), out: n bytes. */
static void mpwsd_frame(const or_code *c, const double *y, const uint8_t *anchors, int count, int J,
                        uint8_t *out, wsd_info *info) {
    int n = c->n;
    int64_t P = c->P;
    int m = c->filter_m;
    if (m > P) m = (int)P;
    uint8_t *ck = (uint8_t *)malloc((size_t)count * n + 1); /* current centres */
    uint8_t *active = (uint8_t *)malloc((size_t)count + 1);
    uint8_t *retired = (uint8_t *)malloc((size_t)count + 1); /* not counted in evals_distinct */
    gain_ent *heap = (gain_ent *)malloc(sizeof(gain_ent) * (size_t)(m + 1));
    double xhat[OR_MAXN];
    memcpy(ck, anchors, (size_t)count * n);
    for (int k = 0; k < count; k++) {
        active[k] = 1;
        retired[k] = 0;
    }
    info->iters = 0;
    info->min_gap = INFINITY;
    info->evals = 0;
    info->evals_distinct = 0;
    for (int it = 1; it <= J; it++) {
        int updated = 0;
        info->iters = it;
        for (int k = 0; k < count; k++) {
            if (!active[k]) continue;
            uint8_t *cur = ck + (size_t)k * n;
            for (int j = 0; j < n; j++) xhat[j] = 1.0 - 2.0 * cur[j];
            /* Filter: the set M_k of the m patterns with the largest gain
             * G_k(c) = sum_{j in supp c} -2 y_j xhat_{k,j}  (Eq. 5);
             * among equal gains the lower pattern index is preferred. */
            int hs = 0;
            for (int64_t p = 0; p < P; p++) {
                const int *sp = c->pat_supp + (size_t)p * n;
                double g = 0.0;
                for (int t = 0; t < c->pat_w[p]; t++) g += -2.0 * y[sp[t]] * xhat[sp[t]];
                gain_ent e = {g, p};
                if (hs < m) {
                    heap[hs] = e;
                    heap_sift_up(heap, hs);
                    hs++;
                } else if (m > 0 && weaker(&heap[0], &e)) {
                    heap[0] = e;
                    heap_sift_down(heap, hs, 0);
                }
            }
            info->evals += P;
            if (!retired[k]) info->evals_distinct += P;
            /* Search: exact squared Euclidean distance of every candidate in
             * M_k; ties keep the lowest pattern index. */
            double ed_cur = sq_dist(y, cur, n);
            double best = INFINITY, second = INFINITY;
            int64_t bestp = -1;
            uint8_t cand[OR_MAXN];
            for (int q = 0; q < hs; q++) {
                const uint8_t *pp = c->pat + (size_t)heap[q].p * n;
                for (int j = 0; j < n; j++) cand[j] = cur[j] ^ pp[j];
                double ed = sq_dist(y, cand, n);
                if (ed < best || (ed == best && heap[q].p < bestp)) {
                    if (bestp >= 0 && best < second) second = best;
                    best = ed;
                    bestp = heap[q].p;
                } else if (ed < second) {
                    second = ed;
                }
            }
            /* Update rule: hop only on strict improvement (Algorithm 1). */
            double gap;
            if (bestp >= 0 && best < ed_cur) {
                const uint8_t *pp = c->pat + (size_t)bestp * n;
                for (int j = 0; j < n; j++) cur[j] ^= pp[j];
                updated = 1;
                gap = (second < ed_cur ? second : ed_cur) - best;
            } else {
                active[k] = 0;
                gap = (bestp >= 0 ? best : INFINITY) - ed_cur;
            }
            if (gap < info->min_gap) info->min_gap = gap;
        }
        for (int k = 0; k < count; k++) {
            if (!active[k] || retired[k]) continue;  /* only rows that hopped in this iteration */
            for (int k2 = 0; k2 < k && !retired[k]; k2++)
                if (!retired[k2] && memcmp(ck + (size_t)k2 * n, ck + (size_t)k * n, (size_t)n) == 0) retired[k] = 1;
        }
        if (!updated) break;
    }
    /* Final decision: the path with the smallest ED; ties keep the lowest k. */
    double best = INFINITY;
    int bk = 0;
    for (int k = 0; k < count; k++) {
        double ed = sq_dist(y, ck + (size_t)k * n, n);
        if (ed < best) { best = ed; bk = k; }
    }
    for (int k = 0; k < count; k++) {
        if (memcmp(ck + (size_t)k * n, ck + (size_t)bk * n, (size_t)n) == 0) continue;
        double gap = sq_dist(y, ck + (size_t)k * n, n) - best;
        if (gap < info->min_gap) info->min_gap = gap;
    }
    memcpy(out, ck + (size_t)bk * n, (size_t)n);
    info->final_k = bk;
    free(ck);
    free(active);
    free(retired);
    free(heap);
}

/* ------------------------------------------------------------------------ */
/* Two-stage decoder over a batch (Sec. III-A + III-B), threaded by frames   */
/* ------------------------------------------------------------------------ */

enum { OR_RULE_TOP1 = 0, OR_RULE_ANY = 1 };

typedef struct {
    const or_code *c;
    const double *y;
    int64_t B;
    int L, J, rule, aom;
    int osd_order;      /* < 0: SC-list stage 1; >= 0: OSD(osd_order) stage 1 */
    uint64_t *cw_out;   /* B x W */
    uint16_t *flags;    /* B */
    double *min_gap;    /* B, may be NULL */
    uint8_t *anchors_out; /* B x L x n, may be NULL: stage-1 list (u -> codewords) */
    int64_t *evals;     /* B, may be NULL */
    int64_t *evals_distinct; /* B, may be NULL */
    int64_t next;       /* shared frame counter */
    pthread_mutex_t lock;
} batch_job;

/* ------------------------------------------------------------------------ */
/* Stage 1 alternative: OSD(order) list (Sec. IV-A uses OSD anchors)            */
/* ------------------------------------------------------------------------ */
/* The paper names OSD without details; this is the standard construction:
 *  1. hard decisions hd_j = [y_j < 0] and reliabilities |y_j|;
 *  2. positions in decreasing reliability, ties to the lower index;
 *  3. the most reliable basis (MRB): walking the positions in that order, a
 *     position joins when its generator column is independent of the ones
 *     already chosen, until k are chosen. Gauss-Jordan on the generator makes
 *     row t of G_sys the codeword that is 1 at the t-th chosen position and 0
 *     at the other chosen ones (unique: the chosen columns are invertible);
 *  4. c0 = XOR of the rows t with hd = 1 at the t-th chosen position (the
 *     codeword that agrees with hd on the MRB);
 *  5. candidates c0 XOR (rows of F) for every F with |F| <= order, enumerated
 *     by |F|, then lexicographically;
 *  6. discrepancy D(c) = sum_j |y_j| [c_j != hd_j]; ED(c) = ||y||^2 + n -
 *     2 sum_j |y_j| + 4 D(c), so D orders candidates as ED does;
 *  7. the list: the min(L, #candidates) smallest D, ties in enumeration order.
 * Returns the list size; cw_list (L x n bytes) and d_list (L) hold it. */
typedef struct {
    double d;
    int64_t idx;
} osd_cand;

static int osd_cmp(const void *pa, const void *pb) {
    const osd_cand *a = (const osd_cand *)pa, *b = (const osd_cand *)pb;
    if (a->d != b->d) return a->d < b->d ? -1 : 1;
    return a->idx < b->idx ? -1 : (a->idx > b->idx ? 1 : 0);
}

typedef struct {
    double r;
    int j;
} rel_pos;

static int rel_cmp(const void *pa, const void *pb) {
    const rel_pos *a = (const rel_pos *)pa, *b = (const rel_pos *)pb;
    if (a->r != b->r) return a->r > b->r ? -1 : 1; /* more reliable first */
    return a->j - b->j;
}

/* candidate number idx (enumeration order of step 5) -> its set F (ascending) */
static int osd_subset(int64_t idx, int k, int order, int *F) {
    for (int w = 0; w <= order && w <= k; w++) {
        /* C(k, w) subsets of size w */
        int64_t cnt = 1;
        for (int t = 0; t < w; t++) cnt = cnt * (k - t) / (t + 1);
        if (idx >= cnt) {
            idx -= cnt;
            continue;
        }
        /* the idx-th w-subset in lexicographic order */
        int start = 0;
        for (int t = 0; t < w; t++) {
            for (int v = start; v < k; v++) {
                int64_t rest = 1; /* C(k - v - 1, w - t - 1) */
                for (int q = 0; q < w - t - 1; q++) rest = rest * (k - v - 1 - q) / (q + 1);
                if (idx < rest) {
                    F[t] = v;
                    start = v + 1;
                    break;
                }
                idx -= rest;
            }
        }
        return w;
    }
    return -1;
}

int or_osd(const or_code *c, const double *y, int order, int L, uint8_t *cw_list, double *d_list) {
    int n = c->n, k = c->k;
    uint8_t hd[OR_MAXN];
    rel_pos pos[OR_MAXN];
    for (int j = 0; j < n; j++) {
        hd[j] = y[j] < 0.0 ? 1 : 0;
        pos[j].r = fabs(y[j]);
        pos[j].j = j;
    }
    qsort(pos, (size_t)n, sizeof(rel_pos), rel_cmp);
    /* generator rows (Arikan rows at the non-frozen indices) */
    uint8_t *G = (uint8_t *)malloc((size_t)k * n);
    for (int t = 0; t < k; t++)
        for (int j = 0; j < n; j++) G[(size_t)t * n + j] = c->F[(size_t)c->info[t] * n + j];
    int pivot_row[OR_MAXN], mrb[OR_MAXN], used[OR_MAXN];
    for (int t = 0; t < k; t++) used[t] = 0;
    int found = 0;
    for (int q = 0; q < n && found < k; q++) {
        int p = pos[q].j, r = -1;
        for (int t = 0; t < k; t++)
            if (!used[t] && G[(size_t)t * n + p]) {
                r = t;
                break;
            }
        if (r < 0) continue; /* column dependent on the chosen ones */
        for (int t = 0; t < k; t++)
            if (t != r && G[(size_t)t * n + p])
                for (int j = 0; j < n; j++) G[(size_t)t * n + j] ^= G[(size_t)r * n + j];
        used[r] = 1;
        pivot_row[found] = r;
        mrb[found] = p;
        found++;
    }
    /* c0 */
    uint8_t c0[OR_MAXN];
    memset(c0, 0, (size_t)n);
    for (int t = 0; t < found; t++)
        if (hd[mrb[t]])
            for (int j = 0; j < n; j++) c0[j] ^= G[(size_t)pivot_row[t] * n + j];
    /* enumerate, score, keep the best */
    int64_t ncand = 0;
    for (int w = 0; w <= order && w <= found; w++) {
        int64_t cnt = 1;
        for (int t = 0; t < w; t++) cnt = cnt * (found - t) / (t + 1);
        ncand += cnt;
    }
    osd_cand *cand = (osd_cand *)malloc(sizeof(osd_cand) * (size_t)ncand);
    int F[OR_MAXN];
    uint8_t cw[OR_MAXN];
    for (int64_t i = 0; i < ncand; i++) {
        int w = osd_subset(i, found, order, F);
        memcpy(cw, c0, (size_t)n);
        for (int t = 0; t < w; t++)
            for (int j = 0; j < n; j++) cw[j] ^= G[(size_t)pivot_row[F[t]] * n + j];
        double d = 0.0;
        for (int j = 0; j < n; j++)
            if (cw[j] != hd[j]) d += fabs(y[j]);
        cand[i].d = d;
        cand[i].idx = i;
    }
    qsort(cand, (size_t)ncand, sizeof(osd_cand), osd_cmp);
    int count = (int)(ncand < L ? ncand : L);
    for (int q = 0; q < count; q++) {
        int w = osd_subset(cand[q].idx, found, order, F);
        uint8_t *out = cw_list + (size_t)q * n;
        memcpy(out, c0, (size_t)n);
        for (int t = 0; t < w; t++)
            for (int j = 0; j < n; j++) out[j] ^= G[(size_t)pivot_row[F[t]] * n + j];
        if (d_list) d_list[q] = cand[q].d;
    }
    free(cand);
    free(G);
    return count;
}

static void pack_bits(const uint8_t *b, int n, uint64_t *w) {
    int W = (n + 63) / 64;
    for (int q = 0; q < W; q++) w[q] = 0;
    for (int j = 0; j < n; j++)
        if (b[j]) w[j >> 6] |= 1ull << (j & 63);
}

/* Decode one frame. Flags: bit0 stage 2 ran, bit1 the output passes the CRC,
 * bits 4..7 outer iterations used by stage 2. */
static void decode_frame(const or_code *c, const double *y, int L, int J, int rule, int aom, int osd_order,
                         uint64_t *cw_out, uint16_t *flags, double *gap, uint8_t *anchors_out, int64_t *evals,
                         int64_t *evals_distinct) {
    int n = c->n;
    uint8_t *ul = (uint8_t *)malloc((size_t)L * n);
    uint8_t *cl = (uint8_t *)malloc((size_t)L * n);
    double *pml = (double *)malloc(sizeof(double) * (size_t)L);
    int count;
    if (osd_order >= 0) {
        /* stage 1 = OSD(osd_order): its list, best discrepancy first, are the anchors */
        count = or_osd(c, y, osd_order, L, cl, pml);
    } else {
        count = or_scl(c, y, L, ul, pml);
        for (int q = 0; q < count; q++) or_encode(c, ul + (size_t)q * n, cl + (size_t)q * n);
    }
    if (anchors_out) {
        memset(anchors_out, 0, (size_t)L * n);
        memcpy(anchors_out, cl, (size_t)count * n);
    }
    uint16_t fl = 0;
    double g = INFINITY;
    int64_t ev = 0, evd = 0;
    uint8_t out[OR_MAXN];
    int use_crc = (c->crc_len > 0) && !aom;
    int done = 0;
    if (use_crc) {
        /* Sec. III-A: the most reliable candidate is checked; TOP1 takes the
         * literal reading (list[0] only); ANY takes the best-PM candidate that
         * passes. */
        int lim = rule == OR_RULE_ANY ? count : 1;
        for (int q = 0; q < lim && !done; q++)
            if (crc_ok_codeword(c, cl + (size_t)q * n)) {
                memcpy(out, cl + (size_t)q * n, (size_t)n);
                done = 1;
            }
    }
    if (!done) {
        wsd_info info;
        mpwsd_frame(c, y, cl, count, J, out, &info);
        fl |= 1;
        int it = info.iters > 15 ? 15 : info.iters;
        fl |= (uint16_t)(it << 4);
        g = info.min_gap;
        ev = info.evals;
        evd = info.evals_distinct;
    }
    if (crc_ok_codeword(c, out) && c->crc_len > 0) fl |= 2;
    pack_bits(out, n, cw_out);
    *flags = fl;
    if (gap) *gap = g;
    if (evals) *evals = ev;
    if (evals_distinct) *evals_distinct = evd;
    free(ul); free(cl); free(pml);
}

static void *batch_worker(void *arg) {
    batch_job *jb = (batch_job *)arg;
    int n = jb->c->n, W = (n + 63) / 64;
    for (;;) {
        pthread_mutex_lock(&jb->lock);
        int64_t f = jb->next++;
        pthread_mutex_unlock(&jb->lock);
        if (f >= jb->B) break;
        decode_frame(jb->c, jb->y + f * n, jb->L, jb->J, jb->rule, jb->aom, jb->osd_order, jb->cw_out + f * W,
                     jb->flags + f,
                     jb->min_gap ? jb->min_gap + f : NULL,
                     jb->anchors_out ? jb->anchors_out + (size_t)f * jb->L * n : NULL,
                     jb->evals ? jb->evals + f : NULL, jb->evals_distinct ? jb->evals_distinct + f : NULL);
    }
    return NULL;
}

/* Decode B frames (y: B x n FP64). Outputs as described above. nthreads <= 0
 * means 1. Returns 0, or -1 on bad arguments. */
int or_decode(const or_code *c, const double *y, int64_t B, int L, int J, int rule, int aom, int osd_order,
              int nthreads, uint64_t *cw_out, uint16_t *flags, double *min_gap, uint8_t *anchors_out,
              int64_t *evals, int64_t *evals_distinct) {
    if (!c || L < 1 || J < 0 || B < 0) return -1;
    if (B == 0) return 0;
    batch_job jb;
    jb.c = c; jb.y = y; jb.B = B; jb.L = L; jb.J = J; jb.rule = rule; jb.aom = aom; jb.osd_order = osd_order;
    jb.cw_out = cw_out; jb.flags = flags; jb.min_gap = min_gap; jb.anchors_out = anchors_out; jb.evals = evals;
    jb.evals_distinct = evals_distinct;
    jb.next = 0;
    pthread_mutex_init(&jb.lock, NULL);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, batch_worker, &jb);
    batch_worker(&jb);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&jb.lock);
    return 0;
}

/* Stage 2 alone on given anchors (count x n bytes), for tests of Algorithm 1. */
void or_mpwsd(const or_code *c, const double *y, const uint8_t *anchors, int count, int J, uint8_t *out,
              int *iters, double *min_gap, int64_t *evals, int *final_k) {
    wsd_info info;
    mpwsd_frame(c, y, anchors, count, J, out, &info);
    *iters = info.iters;
    *min_gap = info.min_gap;
    *evals = info.evals;
    *final_k = info.final_k;
}

/* Correlation gains of Eq. (5) for every pattern around centre cw:
 * G(p) = sum_{j in supp p} -2 y_j xhat_j, xhat = 1 - 2 cw. FP64, exact on the grid. */
void or_gains(const or_code *c, const double *y, const uint8_t *cw, double *G) {
    for (int64_t p = 0; p < c->P; p++) {
        const int *sp = c->pat_supp + (size_t)p * c->n;
        double g = 0.0;
        for (int t = 0; t < c->pat_w[p]; t++) g += -2.0 * y[sp[t]] * (1.0 - 2.0 * cw[sp[t]]);
        G[p] = g;
    }
}

/* Brute-force ML: argmin ||y - x(c)||^2 over all 2^k codewords (ties keep the
 * smallest message integer a, with info bit t at bit t of a). Codewords are
 * formed by XOR of bit-packed generator rows; the distance is computed from
 * the bits directly. */
void or_ml(const or_code *c, const double *y, uint8_t *out, double *ed_out) {
    int n = c->n, k = c->k;
    uint64_t G[64][2];
    for (int t = 0; t < k; t++) {
        G[t][0] = G[t][1] = 0;
        for (int j = 0; j < n; j++)
            if (c->F[c->info[t] * n + j]) G[t][j >> 6] |= 1ull << (j & 63);
    }
    double best = INFINITY;
    uint64_t bw[2] = {0, 0};
    for (uint64_t a = 0; a < (1ull << k); a++) {
        uint64_t cw[2] = {0, 0};
        for (int t = 0; t < k; t++)
            if ((a >> t) & 1ull) { cw[0] ^= G[t][0]; cw[1] ^= G[t][1]; }
        double ed = 0.0;
        for (int j = 0; j < n; j++) {
            double d = y[j] - (((cw[j >> 6] >> (j & 63)) & 1ull) ? -1.0 : 1.0);
            ed += d * d;
        }
        if (ed < best) {
            best = ed;
            bw[0] = cw[0];
            bw[1] = cw[1];
        }
    }
    for (int j = 0; j < n; j++) out[j] = (uint8_t)((bw[j >> 6] >> (j & 63)) & 1ull);
    *ed_out = best;
}
