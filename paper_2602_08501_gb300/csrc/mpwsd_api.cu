// C ABI of libmpwsd (declared in include/mpwsd.h): argument validation, the
// device image of a code (Sec. II-B code model, Sec. II-C pattern set), the
// per-decode workspaces, and the launch sequence of the two-stage decoder
// (Sec. III-A stage 1, Sec. III-B Algorithm 1 stage 2). Host code only;
// every arithmetic step of a decode runs in the CUDA kernels.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <array>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <unordered_set>
#include <vector>

#include "internal.h"

using namespace mpwsd;

namespace {

thread_local std::string g_err;

int fail(int status, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation) return fail(MPWSD_ENOMEM, "%s: %s", what, cudaGetErrorString(e));
    return fail(MPWSD_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Test hook: MPWSD_TEST_FAIL_ALLOC=k makes the k-th device allocation of the
// process (counted from 1) report out-of-memory without allocating.
std::atomic<long> g_alloc_count{0};

cudaError_t dev_alloc(void **p, size_t bytes) {
    const long k = ++g_alloc_count;
    const char *env = getenv("MPWSD_TEST_FAIL_ALLOC");
    if (env && atol(env) == k) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes == 0 ? 16 : bytes);
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }


// Row i of [[1,0],[1,1]]^{(x)m} has ones exactly at the submasks j of i.
inline bool kron_entry(int i, int j) { return (i & j) == j; }

uint16_t f32_to_bf16_bits(float f) {  // exact for 0.0 and 1.0, the only values used
    uint32_t u;
    memcpy(&u, &f, 4);
    return (uint16_t)(u >> 16);
}

}  // namespace

struct mpwsd_workspace {
    Workspace w;
};

// mpwsd_decode_host splits a batch into at most this many chunks, of at least
// kHostChunkFrames frames each, so that the copy of chunk i + 1 overlaps
// stage 1 of chunk i.
constexpr int kHostChunks = 8;
constexpr int64_t kHostChunkFrames = 65536;

struct mpwsd_code {
    CodeDev d;
    std::vector<int> info;  // non-frozen indices, ascending
    mpwsd_workspace *default_ws = nullptr;
    std::atomic<long long> launches{0};
    std::mutex mu;
    // kernel timing (mpwsd_profile_begin / end)
    bool profiling = false;
    std::mutex prof_mu;
    struct Rec {
        int kind;
        cudaEvent_t start, stop;
    };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    // CUDA graphs of decode launch sequences (opts.use_graph)
    struct GraphKey {
        const void *ws, *y, *cw, *fl;
        int64_t ws_B, B;  // workspace layout (base, max_B, max_L) and the call
        int ws_L, L, T, mode, rule, aom, stage1, osd_order;
        const void *hy, *hcw, *hfl;  // host buffers of mpwsd_decode_host (else NULL)
        bool operator==(const GraphKey &o) const {
            return ws == o.ws && ws_B == o.ws_B && ws_L == o.ws_L && y == o.y && cw == o.cw && fl == o.fl &&
                   B == o.B && L == o.L && T == o.T && mode == o.mode && rule == o.rule && aom == o.aom &&
                   stage1 == o.stage1 && osd_order == o.osd_order && hy == o.hy && hcw == o.hcw && hfl == o.hfl;
        }
    };
    struct GraphEnt {
        GraphKey key;
        cudaGraphExec_t exec;
        int kernels;
    };
    std::vector<GraphEnt> graphs;
    cudaStream_t capture_stream = nullptr;
    // mpwsd_decode_host: device staging buffers, the stream that carries the
    // input copies, and the events that order each chunk's stage 1 after its copy.
    // Calls alternate between two input buffers, so the copies of one call can run
    // while the stage 2 of the call before it still reads the other buffer;
    // stage_done[b] marks the end of the last call that used buffer b.
    float *stage_y = nullptr;
    float *stage_y2 = nullptr;
    int stage_next = 0;
    cudaEvent_t stage_done[2] = {};
    bool stage_used[2] = {};
    uint64_t *stage_cw = nullptr;
    uint16_t *stage_fl = nullptr;
    int64_t stage_B = 0;
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t copy_ev[kHostChunks + 1] = {};
};

namespace {

cudaEvent_t pool_event(mpwsd_code *c) {
    if (!c->pool.empty()) {
        cudaEvent_t e = c->pool.back();
        c->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Launch through `fn`, counting it and, while profiling, bracketing it with
// CUDA events on the launch stream.
thread_local bool t_capturing = false;  // this thread is recording a decode into a graph

template <class Fn>
cudaError_t timed_launch(mpwsd_code *c, int kind, cudaStream_t s, Fn &&fn) {
    if (t_capturing) return fn();  // counted per replay instead
    c->launches++;
    if (!c->profiling) return fn();
    std::lock_guard<std::mutex> lk(c->prof_mu);
    cudaEvent_t a = pool_event(c), b = pool_event(c);
    cudaEventRecord(a, s);
    cudaError_t e = fn();
    cudaEventRecord(b, s);
    c->recs.push_back({kind, a, b});
    return e;
}

}  // namespace

extern "C" const char *mpwsd_strerror(int status) {
    switch (status) {
        case MPWSD_OK: return "MPWSD_OK";
        case MPWSD_EINVAL: return "MPWSD_EINVAL: invalid argument";
        case MPWSD_ENOMEM: return "MPWSD_ENOMEM: out of memory";
        case MPWSD_ECUDA: return "MPWSD_ECUDA: CUDA error";
        case MPWSD_ETIMEOUT: return "MPWSD_ETIMEOUT: device-side wait timed out";
        case MPWSD_EUNSUPPORTED: return "MPWSD_EUNSUPPORTED: not supported by this build";
        default: return "unknown mpwsd status";
    }
}

extern "C" const char *mpwsd_last_error(void) { return g_err.c_str(); }

static void free_code_device(CodeDev &d) {
    cudaFree(d.pat_bits);
    cudaFree(d.pat_supp);
    cudaFree(d.pat_tiles);
    cudaFree(d.flat_w);
    cudaFree(d.flat_idx);
    cudaFree(d.crc_masks);
    cudaFree(d.gen_rows);
    cudaFree(d.osd_sets);
    cudaFree(d.stats);
    d.pat_bits = nullptr;
    d.pat_supp = nullptr;
    d.pat_tiles = nullptr;
    d.flat_w = nullptr;
    d.flat_idx = nullptr;
    d.crc_masks = nullptr;
    d.gen_rows = nullptr;
    d.osd_sets = nullptr;
    d.stats = nullptr;
}

// Flat structure of a pattern set for MPWSD_SCORE_FLATS. Positions j are read
// as m-bit vectors (the binary digits of j, the coordinates of the Arikan
// form). Returns the complement dimension kd (1 or 2) and fills the entries
// (see CodeDev::flat_w / flat_idx) when every pattern is a coset a + V of a
// linear subspace V, all of one dimension m - kd, and every coset of every V
// that occurs is in the set; returns 0 otherwise.
static int flats_table(int n, int m, const uint64_t *patterns, int64_t P, int W, std::vector<uint32_t> &off,
                       std::vector<int32_t> &idx) {
    off.clear();
    idx.clear();
    if (P < 1 || n > 128) return 0;
    auto bit = [&](int64_t p, int j) { return (int)((patterns[p * W + j / 64] >> (j % 64)) & 1ull); };
    auto parity = [](int x) { return __builtin_parity((unsigned)x); };
    int kd = -1;
    std::map<std::vector<int>, int> entry_of;  // complement (its nonzero elements, ascending) -> entry
    std::vector<std::array<int, 2>> basis;
    for (int64_t p = 0; p < P; ++p) {
        std::vector<int> pts;
        for (int j = 0; j < n; ++j)
            if (bit(p, j)) pts.push_back(j);
        const size_t sz = pts.size();
        if (sz == 0 || (sz & (sz - 1))) return 0;
        int dim = 0;
        while ((1u << dim) < sz) ++dim;
        const int a = pts[0];
        std::vector<char> inV((size_t)n, 0);
        for (int x : pts) inV[(size_t)(x ^ a)] = 1;
        for (int x : pts)  // V = pts ^ a is closed under XOR
            for (int y : pts)
                if (!inV[(size_t)(x ^ y)]) return 0;
        const int this_kd = m - dim;
        if (this_kd < 1 || this_kd > 2) return 0;
        if (kd < 0) kd = this_kd;
        if (kd != this_kd) return 0;
        std::vector<int> comp;  // w != 0 orthogonal to every element of V
        for (int w = 1; w < n; ++w) {
            bool ok = true;
            for (int x : pts)
                if (parity(w & (x ^ a))) {
                    ok = false;
                    break;
                }
            if (ok) comp.push_back(w);
        }
        if ((int)comp.size() != (1 << kd) - 1) return 0;
        auto it = entry_of.find(comp);
        int e;
        if (it == entry_of.end()) {
            e = (int)basis.size();
            entry_of.emplace(comp, e);
            basis.push_back({comp[0], kd == 2 ? comp[1] : 0});
            idx.insert(idx.end(), 4, -1);
        } else {
            e = it->second;
        }
        const int c1 = parity(basis[(size_t)e][0] & a), c2 = kd == 2 ? parity(basis[(size_t)e][1] & a) : 0;
        int32_t &slot = idx[(size_t)e * 4 + c1 + 2 * c2];
        if (slot >= 0) return 0;  // the same coset twice
        slot = (int32_t)p;
    }
    for (size_t e = 0; e < basis.size(); ++e)  // every coset present
        for (int c = 0; c < (1 << kd); ++c)
            if (idx[e * 4 + (size_t)c] < 0) return 0;
    for (auto &b : basis) {
        const unsigned w1 = (unsigned)b[0], w2 = (unsigned)b[1];
        off.push_back(w1 | (w2 << 8) | ((w1 ^ w2) << 16));
    }
    return kd;
}

extern "C" int mpwsd_load_code(int n, const uint8_t *G, const uint8_t *frozen, int k_info, uint32_t crc_poly,
                               int crc_len, const uint64_t *patterns, int64_t n_patterns, mpwsd_code **out) {
    if (!out) return fail(MPWSD_EINVAL, "out is NULL");
    *out = nullptr;
    if (n != 32 && n != 64 && n != 128) return fail(MPWSD_EINVAL, "n = %d: must be 32, 64 or 128", n);
    if (!frozen) return fail(MPWSD_EINVAL, "frozen is NULL");
    if (!patterns || n_patterns < 1 || n_patterns > 0x7fffffffLL)
        return fail(MPWSD_EINVAL, "need 1 <= n_patterns < 2^31 and a pattern array");
    if (crc_len < 0 || crc_len > 32) return fail(MPWSD_EINVAL, "crc_len = %d: must be 0..32", crc_len);
    if (crc_len < 32 && (crc_poly >> crc_len) != 0) return fail(MPWSD_EINVAL, "crc_poly has bits above crc_len");
    const int W = (n + 63) / 64;
    int m = 0;
    while ((1 << m) < n) ++m;
    std::vector<int> info;
    for (int i = 0; i < n; ++i) {
        if (frozen[i] > 1) return fail(MPWSD_EINVAL, "frozen[%d] = %d: must be 0 or 1", i, frozen[i]);
        if (!frozen[i]) info.push_back(i);
    }
    const int k = (int)info.size();
    if (k < 1) return fail(MPWSD_EINVAL, "no information positions");
    if (k_info < 1 || k_info + crc_len != k)
        return fail(MPWSD_EINVAL, "k_info (%d) + crc_len (%d) must equal the %d information positions", k_info, crc_len, k);
    if (G) {
        for (int t = 0; t < k; ++t)
            for (int j = 0; j < n; ++j)
                if ((G[(size_t)t * n + j] != 0) != kron_entry(info[t], j))
                    return fail(MPWSD_EINVAL, "G row %d differs from row %d of the Arikan kernel power", t, info[t]);
    }
    // patterns: nonzero, within n bits, codewords (u = p F zero on frozen), distinct
    std::vector<uint8_t> frz(frozen, frozen + n);
    int w_max = 0;
    {
        std::unordered_set<std::string> seen;
        seen.reserve((size_t)n_patterns * 2);
        for (int64_t p = 0; p < n_patterns; ++p) {
            const uint64_t *pw = patterns + p * W;
            if (n < 64 && (pw[0] >> n) != 0) return fail(MPWSD_EINVAL, "pattern %lld has bits beyond n", (long long)p);
            int w = 0;
            for (int q = 0; q < W; ++q) w += __builtin_popcountll(pw[q]);
            if (w == 0) return fail(MPWSD_EINVAL, "pattern %lld is the zero word", (long long)p);
            w_max = std::max(w_max, w);
            // u_i = sum_j c_j F[j][i] = parity of c restricted to supersets of i
            for (int i = 0; i < n; ++i) {
                if (!frz[i]) continue;
                int par = 0;
                for (int q = 0; q < W; ++q) {
                    uint64_t sup = 0;  // positions j (in word q) with i a submask of j
                    for (int b = 0; b < 64 && q * 64 + b < n; ++b)
                        if (kron_entry(q * 64 + b, i)) sup |= 1ull << b;
                    par ^= __builtin_popcountll(pw[q] & sup) & 1;
                }
                if (par) return fail(MPWSD_EINVAL, "pattern %lld is not a codeword (frozen u_%d = 1)", (long long)p, i);
            }
            if (!seen.insert(std::string((const char *)pw, (size_t)W * 8)).second)
                return fail(MPWSD_EINVAL, "pattern %lld repeats an earlier pattern", (long long)p);
        }
    }

    mpwsd_code *c = new (std::nothrow) mpwsd_code();
    if (!c) return fail(MPWSD_ENOMEM, "host allocation");
    CodeDev &d = c->d;
    c->info = info;
    d.n = n;
    d.W = W;
    d.m = m;
    d.k = k;
    d.k_info = k_info;
    d.crc_len = crc_len;
    d.crc_poly = crc_poly;
    d.P = n_patterns;
    for (int i = 0; i < n; ++i)
        if (frozen[i]) {
            if (i < 64)
                d.frozen_lo |= 1ull << i;
            else
                d.frozen_hi |= 1ull << (i - 64);
        }
    d.rm_spec = rm_specialisation(n, d.frozen_lo, d.frozen_hi);
    if (const char *st = getenv("MPWSD_TEST_TC_STALL")) {
        if (atoi(st) > 0) {  // test hook: see CodeDev::test_stall
            d.test_stall = 1;
            d.wait_limit_ns = 20000000ull;
        }
    }
    d.trailing_frozen = info.back() != n - 1;
    d.w_max = w_max;
    d.wq_max = (w_max + 3) / 4;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaGetDevice");
    }
    e = cudaDeviceGetAttribute(&d.num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        delete c;
        return cuda_fail(e, "cudaDeviceGetAttribute");
    }
    d.split_items = d.num_sms / 2;

    // host images
    std::vector<uint32_t> supp((size_t)n_patterns * d.wq_max, 0);
    d.supp_dense = true;
    for (int64_t p = 0; p < n_patterns; ++p) {
        uint8_t idx[128];
        int w = 0;
        for (int j = 0; j < n; ++j)
            if ((patterns[p * W + j / 64] >> (j % 64)) & 1ull) idx[w++] = (uint8_t)j;
        if (w != d.wq_max * 4) d.supp_dense = false;
        for (; w < d.wq_max * 4; ++w) idx[w] = (uint8_t)n;  // pad: reads the zero slot
        for (int q = 0; q < d.wq_max; ++q)
            supp[(size_t)p * d.wq_max + q] = (uint32_t)idx[4 * q] | ((uint32_t)idx[4 * q + 1] << 8) |
                                             ((uint32_t)idx[4 * q + 2] << 16) | ((uint32_t)idx[4 * q + 3] << 24);
    }
    // bf16 0/1 pattern tiles, tc_patterns_per_tile(n) patterns x n per tile, laid
    // out as the shared memory image a K-major 128-byte-swizzled UMMA operand
    // expects: for each 64-element K chunk, rows of 128 B grouped in 1024-B
    // atoms, 16-B unit u of row r stored at unit u ^ (r % 8).
    const int TP = tc_patterns_per_tile(n);
    d.n_tiles = (n_patterns + TP - 1) / TP;
    const int kchunks = n / 64 > 0 ? n / 64 : 1;
    const size_t tile_elems = (size_t)TP * kchunks * 64;
    std::vector<uint16_t> tiles;
    if (n >= 64) {
        tiles.assign((size_t)d.n_tiles * tile_elems, 0);
        const uint16_t one = f32_to_bf16_bits(1.0f);
        for (int64_t p = 0; p < n_patterns; ++p) {
            const int64_t tile = p / TP;
            const int r = (int)(p % TP);
            for (int j = 0; j < n; ++j) {
                if (!((patterns[p * W + j / 64] >> (j % 64)) & 1ull)) continue;
                const int kc = j / 64, e64 = j % 64;
                const int unit = e64 / 8, within = e64 % 8;
                const size_t off = (size_t)tile * tile_elems + (size_t)kc * TP * 64 + (size_t)r * 64 +
                                   (size_t)((unit ^ (r % 8)) * 8 + within);
                tiles[off] = one;
            }
        }
    }
    // CRC: parity matrix by long division of the unit messages, then the
    // syndrome masks moved to the codeword domain (u = c F, F an involution).
    std::vector<uint64_t> masks((size_t)std::max(crc_len, 1) * W, 0);
    for (int b = 0; b < crc_len; ++b) {
        std::vector<uint8_t> inset(n, 0);  // M_b over u indices
        for (int t = 0; t < k_info; ++t) {
            // remainder of x^(k_info - 1 - t + crc_len) mod g(x)
            uint64_t val = 1;
            const uint64_t top = 1ull << crc_len;
            for (int s = 0; s < k_info - 1 - t + crc_len; ++s) {
                val <<= 1;
                if (val & top) val ^= top | crc_poly;
            }
            if ((val >> (crc_len - 1 - b)) & 1ull) inset[info[t]] = 1;
        }
        inset[info[k_info + b]] = 1;
        for (int j = 0; j < n; ++j) {
            int par = 0;
            for (int i = 0; i < n; ++i)
                if (inset[i] && kron_entry(j, i)) par ^= 1;
            if (par) masks[(size_t)b * W + j / 64] |= 1ull << (j % 64);
        }
    }
    // generator rows for OSD: row t = row info[t] of the Arikan kernel power
    std::vector<uint64_t> gen((size_t)k * W, 0);
    for (int t = 0; t < k; ++t)
        for (int j = 0; j < n; ++j)
            if (kron_entry(info[t], j)) gen[(size_t)t * W + j / 64] |= 1ull << (j % 64);
    // OSD candidate row sets in number order: by size, then lexicographic (k <= 32 only)
    std::vector<uint32_t> osd_sets;
    if (k <= 32) {
        osd_sets.reserve((size_t)osd_candidates(k, kOsdMaxOrder));
        for (int w = 0; w <= kOsdMaxOrder && w <= k; ++w) {
            int sel[kOsdMaxOrder];
            for (int t = 0; t < w; ++t) sel[t] = t;
            for (;;) {
                uint32_t v = (uint32_t)w << 20;
                for (int t = 0; t < w; ++t) v |= (uint32_t)sel[t] << (5 * t);
                osd_sets.push_back(v);
                int t = w - 1;  // next w-subset in lexicographic order
                while (t >= 0 && sel[t] == k - w + t) --t;
                if (t < 0) break;
                ++sel[t];
                for (int u = t + 1; u < w; ++u) sel[u] = sel[u - 1] + 1;
            }
        }
    }
    // flat structure of the pattern set (MPWSD_SCORE_FLATS)
    std::vector<uint32_t> flat_w;
    std::vector<int32_t> flat_idx;
    d.flat_kd = flats_table(n, m, patterns, n_patterns, W, flat_w, flat_idx);
    d.n_flat = d.flat_kd ? (int)flat_w.size() : 0;
    // device images
    struct Up {
        void **dst;
        const void *src;
        size_t bytes;
    } ups[] = {
        {(void **)&d.flat_w, flat_w.data(), flat_w.size() * 4},
        {(void **)&d.flat_idx, flat_idx.data(), flat_idx.size() * 4},
        {(void **)&d.pat_bits, patterns, (size_t)n_patterns * W * 8},
        {(void **)&d.pat_supp, supp.data(), supp.size() * 4},
        {(void **)&d.pat_tiles, tiles.data(), tiles.size() * 2},
        {(void **)&d.crc_masks, masks.data(), masks.size() * 8},
        {(void **)&d.gen_rows, gen.data(), gen.size() * 8},
        {(void **)&d.osd_sets, osd_sets.data(), osd_sets.size() * 4},
    };
    for (auto &u : ups) {
        e = dev_alloc(u.dst, u.bytes);
        if (e == cudaSuccess && u.bytes) e = cudaMemcpy(*u.dst, u.src, u.bytes, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            free_code_device(d);
            delete c;
            return cuda_fail(e, "uploading the code");
        }
    }
    e = dev_alloc((void **)&d.stats, sizeof(DevStats));
    if (e == cudaSuccess) e = cudaMemset(d.stats, 0, sizeof(DevStats));
    if (e != cudaSuccess) {
        free_code_device(d);
        delete c;
        return cuda_fail(e, "allocating counters");
    }
    *out = c;
    return MPWSD_OK;
}

extern "C" int mpwsd_code_info(const mpwsd_code *code, int *n, int *k, int64_t *n_patterns, int *max_w) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    if (n) *n = code->d.n;
    if (k) *k = code->d.k;
    if (n_patterns) *n_patterns = code->d.P;
    if (max_w) *max_w = code->d.w_max;
    return MPWSD_OK;
}

// ---- workspaces -------------------------------------------------------------

static size_t ws_layout(const CodeDev &d, int64_t max_B, int max_L, Workspace *w) {
    const int64_t M = max_B * max_L;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off += align256(bytes);
        return o;
    };
    const size_t o_cnt = take(64 * sizeof(int));
    const size_t o_sf = take((size_t)max_B * sizeof(int));
    const size_t o_l1 = take((size_t)max_B * sizeof(float));
    const size_t o_yhl = take((size_t)max_B * d.n * 4);
    const size_t o_cw = take((size_t)M * d.W * 8);
    const size_t o_D = take((size_t)M * 8);
    const size_t o_st = take((size_t)M * 4);
    const size_t o_a0 = take((size_t)M * 4);
    const size_t o_a1 = take((size_t)M * 4);
    const size_t o_rs = take((size_t)M * 4);
    const size_t o_tv = take((size_t)M * kTopK * 4);
    const size_t o_ti = take((size_t)M * kTopK * 4);
    if (w && w->base) {
        char *b = (char *)w->base;
        w->counters = (int *)(b + o_cnt);
        w->slot_frame = (int *)(b + o_sf);
        w->slot_l1 = (float *)(b + o_l1);
        w->slot_yhl = (uint32_t *)(b + o_yhl);
        w->traj_cw = (uint64_t *)(b + o_cw);
        w->traj_D = (double *)(b + o_D);
        w->traj_state = (uint32_t *)(b + o_st);
        w->act[0] = (int *)(b + o_a0);
        w->act[1] = (int *)(b + o_a1);
        w->rescan_rows = (int *)(b + o_rs);
        w->topk_val = (float *)(b + o_tv);
        w->topk_idx = (int *)(b + o_ti);
    }
    return off;
}

extern "C" int mpwsd_workspace_bytes(const mpwsd_code *code, int64_t max_B, int max_L, size_t *bytes) {
    if (!code || !bytes) return fail(MPWSD_EINVAL, "NULL argument");
    if (max_B < 1 || max_L < 1 || max_L > MPWSD_MAX_L) return fail(MPWSD_EINVAL, "need max_B >= 1, 1 <= max_L <= 32");
    if (max_B * max_L > 0x7fffffffLL) return fail(MPWSD_EINVAL, "max_B * max_L must stay below 2^31");
    *bytes = ws_layout(code->d, max_B, max_L, nullptr);
    return MPWSD_OK;
}

extern "C" int mpwsd_workspace_create(const mpwsd_code *code, int64_t max_B, int max_L, mpwsd_workspace **out) {
    if (!out) return fail(MPWSD_EINVAL, "out is NULL");
    *out = nullptr;
    size_t bytes = 0;
    int st = mpwsd_workspace_bytes(code, max_B, max_L, &bytes);
    if (st) return st;
    mpwsd_workspace *ws = new (std::nothrow) mpwsd_workspace();
    if (!ws) return fail(MPWSD_ENOMEM, "host allocation");
    // tail: buffers of the pattern split of the tensor-core scoring kernel
    const size_t split_items = (size_t)kSplitItemsPerSm * std::max(code->d.num_sms, 1);
    const size_t split_entries = split_items * 256 * kTopK;
    const size_t split_bytes = align256(split_entries * 4) * 2 + align256(split_items * sizeof(int));
    cudaError_t e = dev_alloc(&ws->w.base, bytes + split_bytes);
    if (e != cudaSuccess) {
        delete ws;
        cudaGetLastError();  // clear the sticky-free allocation error
        return cuda_fail(e, "workspace allocation");
    }
    ws->w.bytes = bytes + split_bytes;
    ws->w.max_B = max_B;
    ws->w.max_L = max_L;
    cudaGetDevice(&ws->w.device);
    ws_layout(code->d, max_B, max_L, &ws->w);
    char *tail = (char *)ws->w.base + bytes;
    ws->w.split_val = (float *)tail;
    ws->w.split_idx = (int *)(tail + align256(split_entries * 4));
    ws->w.unit_done = (int *)(tail + 2 * align256(split_entries * 4));
    e = cudaMemset(ws->w.unit_done, 0, split_items * sizeof(int));
    if (e != cudaSuccess) {
        cudaFree(ws->w.base);
        delete ws;
        return cuda_fail(e, "workspace initialisation");
    }
    *out = ws;
    return MPWSD_OK;
}

extern "C" void mpwsd_workspace_free(mpwsd_workspace *ws) {
    if (!ws) return;
    cudaDeviceSynchronize();
    cudaFree(ws->w.base);
    delete ws;
}

extern "C" void mpwsd_free_code(mpwsd_code *code) {
    if (!code) return;
    cudaDeviceSynchronize();
    for (auto &r : code->recs) {
        cudaEventDestroy(r.start);
        cudaEventDestroy(r.stop);
    }
    for (auto e : code->pool) cudaEventDestroy(e);
    for (auto &g : code->graphs) cudaGraphExecDestroy(g.exec);
    if (code->capture_stream) cudaStreamDestroy(code->capture_stream);
    if (code->copy_stream) cudaStreamDestroy(code->copy_stream);
    for (auto e : code->copy_ev)
        if (e) cudaEventDestroy(e);
    for (auto e : code->stage_done)
        if (e) cudaEventDestroy(e);
    cudaFree(code->stage_y);
    cudaFree(code->stage_y2);
    cudaFree(code->stage_cw);
    cudaFree(code->stage_fl);
    mpwsd_workspace_free(code->default_ws);
    free_code_device(code->d);
    delete code;
}

// ---- decode -----------------------------------------------------------------

static int check_opts(const mpwsd_opts *opts, mpwsd_opts *o) {
    memset(o, 0, sizeof(*o));
    if (!opts) return MPWSD_OK;
    *o = *opts;
    if (o->score_mode != MPWSD_SCORE_BF16X2 && o->score_mode != MPWSD_SCORE_FP32 &&
        o->score_mode != MPWSD_SCORE_FLATS)
        return fail(MPWSD_EINVAL, "score_mode = %d", o->score_mode);
    if (o->stage1_rule != MPWSD_RULE_TOP1 && o->stage1_rule != MPWSD_RULE_ANY)
        return fail(MPWSD_EINVAL, "stage1_rule = %d", o->stage1_rule);
    if (o->stage1 != MPWSD_STAGE1_SCL && o->stage1 != MPWSD_STAGE1_OSD)
        return fail(MPWSD_EINVAL, "stage1 = %d", o->stage1);
    if (o->stage1 == MPWSD_STAGE1_OSD && (o->osd_order < 0 || o->osd_order > MPWSD_MAX_OSD_ORDER))
        return fail(MPWSD_EINVAL, "osd_order = %d: must be 0..%d", o->osd_order, MPWSD_MAX_OSD_ORDER);
    if (o->stage1 == MPWSD_STAGE1_SCL && o->osd_order != 0)
        return fail(MPWSD_EINVAL, "osd_order is for MPWSD_STAGE1_OSD");
    for (int i = 0; i < 2; ++i)
        if (o->reserved[i]) return fail(MPWSD_EINVAL, "reserved option fields must be zero");
    return MPWSD_OK;
}

static int check_device(const mpwsd_code *code) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    (void)code;
    return MPWSD_OK;
}

static cudaError_t launch_score(mpwsd_code *code, int mode, const ScoreArgs &a, cudaStream_t s) {
    if (mode == MPWSD_SCORE_FP32)
        return timed_launch(code, MPWSD_KERNEL_SCORE_FP32, s, [&] { return launch_score_fp32(code->d, a, s); });
    if (mode == MPWSD_SCORE_FLATS)
        return timed_launch(code, MPWSD_KERNEL_SCORE_FLATS, s, [&] { return launch_score_flats(code->d, a, s); });
    // tensor cores keep candidate groups; their exact argmin follows in its own kernel
    cudaError_t e = timed_launch(code, MPWSD_KERNEL_SCORE_TC, s, [&] { return launch_score_tc(code->d, a, s); });
    if (e != cudaSuccess) return e;
    return timed_launch(code, MPWSD_KERNEL_RESOLVE, s,
                        [&] { return launch_resolve_groups(code->d, a, nullptr, 0, s); });
}

// One scoring step of stage 2 and the re-rank / hop decision of its rows
// (iteration `iter` of a decode, or a pool step): with tensor-core scoring the
// group resolution takes the decisions itself; the other forms leave their
// lists to the hop kernel.
static cudaError_t score_and_hop(mpwsd_code *code, int mode, const ScoreArgs &a, const Workspace &ws, int iter, int L,
                                 const float *y, cudaStream_t s) {
    if (mode == MPWSD_SCORE_BF16X2) {
        cudaError_t e = timed_launch(code, MPWSD_KERNEL_SCORE_TC, s, [&] { return launch_score_tc(code->d, a, s); });
        if (e != cudaSuccess) return e;
        return timed_launch(code, MPWSD_KERNEL_RESOLVE, s,
                            [&] { return launch_resolve_groups(code->d, a, &ws, iter, s); });
    }
    cudaError_t e = launch_score(code, mode, a, s);
    if (e != cudaSuccess) return e;
    return timed_launch(code, MPWSD_KERNEL_HOP, s, [&] { return launch_hop(code->d, ws, iter, L, y, s); });
}

// Host buffers of mpwsd_decode_host: y is copied in chunk by chunk on the copy
// stream, and the results are copied back on the decode stream at the end.
struct HostIO {
    const float *y = nullptr;
    uint64_t *cw = nullptr;
    uint16_t *fl = nullptr;
    int buf = 0;  // which of the two staging input buffers y_dev is
};

static cudaError_t stage1_launch(mpwsd_code *code, Workspace &ws, const float *y_dev, int64_t f0, int64_t B, int L,
                                 const mpwsd_opts &o, uint64_t *cw_dev, uint16_t *flags_dev, cudaStream_t s,
                                 int32_t *done_dev = nullptr, int submit_id = 0) {
    CodeDev &d = code->d;
    const int W = d.W;
    if (o.stage1 == MPWSD_STAGE1_OSD) {
        OsdArgs oa{};
        oa.y = y_dev + f0 * d.n;
        oa.B = B;
        oa.f0 = f0;
        oa.L = L;
        oa.order = o.osd_order;
        oa.ncand = osd_candidates(d.k, o.osd_order);
        oa.mode = 0;
        oa.rule = o.stage1_rule;
        oa.use_crc = d.crc_len > 0 && !o.always_on;
        oa.write_yhl = o.score_mode == MPWSD_SCORE_BF16X2;
        oa.cw_out = cw_dev + f0 * W;
        oa.flags_out = flags_dev + f0;
        oa.done_out = done_dev ? done_dev + f0 : nullptr;
        oa.submit_id = submit_id;
        oa.ws = ws;
        return timed_launch(code, MPWSD_KERNEL_OSD, s, [&] { return launch_osd(d, oa, s); });
    }
    SclArgs sa{};
    sa.y = y_dev + f0 * d.n;
    sa.B = B;
    sa.f0 = f0;
    sa.L = L;
    sa.mode = 0;
    sa.rule = o.stage1_rule;
    sa.use_crc = d.crc_len > 0 && !o.always_on;
    sa.cw_out = cw_dev + f0 * W;
    sa.flags_out = flags_dev + f0;
    sa.done_out = done_dev ? done_dev + f0 : nullptr;
    sa.submit_id = submit_id;
    sa.ws = ws;
    sa.write_yhl = o.score_mode == MPWSD_SCORE_BF16X2;
    return timed_launch(code, MPWSD_KERNEL_SCL, s, [&] { return launch_scl(d, sa, s); });
}

static int decode_impl(mpwsd_code *code, Workspace &ws, const float *y_dev, int64_t B, int L, int T,
                       const mpwsd_opts &o, uint64_t *cw_dev, uint16_t *flags_dev, cudaStream_t s,
                       const HostIO *host = nullptr) {
    CodeDev &d = code->d;
    cudaError_t e = cudaMemsetAsync(ws.counters, 0, 64 * sizeof(int), s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMemsetAsync");
    if (!host) {
        e = stage1_launch(code, ws, y_dev, 0, B, L, o, cw_dev, flags_dev, s);
    } else {
        // chunk i is copied on the copy stream, then its stage 1 runs on s. The
        // copies start after the last call that used this staging buffer (the call
        // before this one used the other buffer, and its stage 2 may still run);
        // inside a graph capture they start after everything already on s
        const int nch = (int)std::max<int64_t>(1, std::min<int64_t>(kHostChunks, B / kHostChunkFrames));
        if (t_capturing) {
            cudaEvent_t fork = code->copy_ev[kHostChunks];
            e = cudaEventRecord(fork, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(code->copy_stream, fork, 0);
        } else if (code->stage_used[host->buf]) {
            e = cudaStreamWaitEvent(code->copy_stream, code->stage_done[host->buf], 0);
        }
        for (int i = 0; i < nch && e == cudaSuccess; ++i) {
            const int64_t a = B * i / nch, b = B * (i + 1) / nch;
            e = cudaMemcpyAsync((void *)(y_dev + a * d.n), host->y + a * d.n, (size_t)(b - a) * d.n * sizeof(float),
                                cudaMemcpyHostToDevice, code->copy_stream);
            if (e == cudaSuccess) e = cudaEventRecord(code->copy_ev[i], code->copy_stream);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, code->copy_ev[i], 0);
            if (e == cudaSuccess) e = stage1_launch(code, ws, y_dev, a, b - a, L, o, cw_dev, flags_dev, s);
        }
    }
    if (e != cudaSuccess) return cuda_fail(e, "stage-1 launch");
    for (int it = 0; it < T; ++it) {
        ScoreArgs a{};
        a.y = y_dev;
        a.rows = ws.act[0];
        a.n_rows_dev = ws.counters + 1 + it;
        a.cw = ws.traj_cw;
        a.slot_frame = ws.slot_frame;
        a.L = L;
        a.topk_val = ws.topk_val;
        a.topk_idx = ws.topk_idx;
        a.yhl = ws.slot_yhl;
        a.l1 = ws.slot_l1;
        a.split_val = ws.split_val;
        a.split_idx = ws.split_idx;
        a.unit_done = ws.unit_done;
        a.split_items = d.split_items;
        e = score_and_hop(code, o.score_mode, a, ws, it, L, y_dev, s);
        if (e != cudaSuccess) return cuda_fail(e, "scoring / hop launch");
        e = timed_launch(code, MPWSD_KERNEL_RESCAN, s, [&] { return launch_rescan(d, ws, it, L, y_dev, s); });
        if (e != cudaSuccess) return cuda_fail(e, "rescan launch");
        if (it + 1 < T) {
            // the next iteration's rows: those that hopped, without duplicates of a
            // lower-numbered trajectory of the same frame (counted with the hop class)
            e = timed_launch(code, MPWSD_KERNEL_HOP, s, [&] { return launch_dedup(d, ws, it, L, s); });
            if (e != cudaSuccess) return cuda_fail(e, "dedup launch");
        }
    }
    e = timed_launch(code, MPWSD_KERNEL_FINAL, s, [&] { return launch_final(d, ws, L, T, B, cw_dev, flags_dev, s); });
    if (e != cudaSuccess) return cuda_fail(e, "final launch");
    if (host) {
        e = cudaMemcpyAsync(host->cw, cw_dev, (size_t)B * d.W * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(host->fl, flags_dev, (size_t)B * sizeof(uint16_t), cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "copying the results to the host");
    }
    return MPWSD_OK;
}

// Kernel nodes of a captured graph (each replay launches that many kernels).
static int graph_kernel_nodes(cudaGraph_t graph) {
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    std::vector<cudaGraphNode_t> list(nodes);
    if (nodes) cudaGraphGetNodes(graph, list.data(), &nodes);
    int kernels = 0;
    for (auto nd : list) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++kernels;
    }
    return kernels;
}

// Decode through a cached CUDA graph of the launch sequence: on a miss the
// sequence is captured on the handle's private stream (nothing runs) and
// instantiated; every call then launches the graph on the caller's stream.
static int decode_graph(mpwsd_code *code, Workspace &ws, const float *y_dev, int64_t B, int L, int T,
                        const mpwsd_opts &o, uint64_t *cw_dev, uint16_t *flags_dev, cudaStream_t s,
                        const HostIO *host) {
    mpwsd_code::GraphKey key{ws.base,  y_dev, cw_dev, flags_dev,     ws.max_B,      B,
                             ws.max_L, L,     T,      o.score_mode, o.stage1_rule, o.always_on,
                             o.stage1, o.osd_order, host ? (const void *)host->y : nullptr,
                             host ? (const void *)host->cw : nullptr, host ? (const void *)host->fl : nullptr};
    std::lock_guard<std::mutex> lk(code->mu);
    for (auto &g : code->graphs)
        if (g.key == key) {
            cudaError_t e = cudaGraphLaunch(g.exec, s);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
            code->launches += g.kernels;
            return MPWSD_OK;
        }
    cudaError_t e = cudaSuccess;
    if (!code->capture_stream) e = cudaStreamCreateWithFlags(&code->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return cuda_fail(e, "creating the capture stream");
    e = cudaStreamBeginCapture(code->capture_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamBeginCapture");
    t_capturing = true;
    int st = decode_impl(code, ws, y_dev, B, L, T, o, cw_dev, flags_dev, code->capture_stream, host);
    t_capturing = false;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(code->capture_stream, &graph);
    if (st) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
    const int kernels = graph_kernel_nodes(graph);
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
    if (code->graphs.size() >= 256) {
        cudaGraphExecDestroy(code->graphs.front().exec);
        code->graphs.erase(code->graphs.begin());
    }
    code->graphs.push_back({key, exec, kernels});
    e = cudaGraphLaunch(exec, s);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
    code->launches += kernels;
    return MPWSD_OK;
}

static int run_decode(mpwsd_code *code, Workspace &ws, const float *y_dev, int64_t B, int L, int T,
                      const mpwsd_opts &o, uint64_t *cw_dev, uint16_t *flags_dev, cudaStream_t s,
                      const HostIO *host = nullptr) {
    if (o.use_graph && !code->profiling) return decode_graph(code, ws, y_dev, B, L, T, o, cw_dev, flags_dev, s, host);
    return decode_impl(code, ws, y_dev, B, L, T, o, cw_dev, flags_dev, s, host);
}

static int check_decode_args(mpwsd_code *code, const float *y_dev, int64_t B, int L, int T, const mpwsd_opts *opts,
                             uint64_t *cw_dev, uint16_t *flags_dev, mpwsd_opts *o) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    if (B < 0) return fail(MPWSD_EINVAL, "B < 0");
    if (L < 1 || L > MPWSD_MAX_L) return fail(MPWSD_EINVAL, "L = %d: must be 1..%d", L, MPWSD_MAX_L);
    if (T < 1 || T > MPWSD_MAX_T) return fail(MPWSD_EINVAL, "T = %d: must be 1..%d", T, MPWSD_MAX_T);
    if (B > 0 && (!y_dev || !cw_dev || !flags_dev)) return fail(MPWSD_EINVAL, "NULL buffer");
    if (B > 0x7fffffffLL / L) return fail(MPWSD_EINVAL, "B * L must stay below 2^31");
    int st = check_opts(opts, o);
    if (st) return st;
    if (o->score_mode == MPWSD_SCORE_BF16X2 && !score_tc_supported(code->d))
        return fail(MPWSD_EUNSUPPORTED, "BF16X2 tensor-core scoring needs n = 64 or 128");
    if (o->score_mode == MPWSD_SCORE_FLATS && code->d.n_flat == 0)
        return fail(MPWSD_EUNSUPPORTED, "FLATS scoring needs a pattern set made of all cosets of subspaces whose "
                                        "complements have dimension 1 or 2");
    if (o->stage1 == MPWSD_STAGE1_OSD && code->d.k > 32)
        return fail(MPWSD_EUNSUPPORTED, "OSD stage 1 needs k <= 32 (k = %d)", code->d.k);
    return check_device(code);
}

extern "C" int mpwsd_decode_ws(mpwsd_code *code, mpwsd_workspace *ws, const float *y_dev, int64_t B, int L, int T,
                               const mpwsd_opts *opts, uint64_t *cw_dev, uint16_t *flags_dev, void *stream) {
    mpwsd_opts o;
    int st = check_decode_args(code, y_dev, B, L, T, opts, cw_dev, flags_dev, &o);
    if (st) return st;
    if (!ws) return fail(MPWSD_EINVAL, "workspace is NULL");
    if (B > ws->w.max_B || L > ws->w.max_L)
        return fail(MPWSD_EINVAL, "B = %lld, L = %d exceed the workspace (%lld, %d)", (long long)B, L,
                    (long long)ws->w.max_B, ws->w.max_L);
    if (B == 0) return MPWSD_OK;
    return run_decode(code, ws->w, y_dev, B, L, T, o, cw_dev, flags_dev, (cudaStream_t)stream);
}

// The handle's own workspace, grown to (B, L) if needed. Caller holds code->mu.
static int default_workspace(mpwsd_code *code, int64_t B, int L, mpwsd_workspace **out) {
    mpwsd_workspace *ws = code->default_ws;
    if (!ws || ws->w.max_B < B || ws->w.max_L < L) {
        const int64_t nb = std::max<int64_t>(B, ws ? ws->w.max_B : 0);
        const int nl = std::max(L, ws ? ws->w.max_L : 0);
        mpwsd_workspace *nw = nullptr;
        int st = mpwsd_workspace_create(code, nb, nl, &nw);
        if (st) return st;
        // graphs recorded on the old workspace go with it
        for (auto it = code->graphs.begin(); it != code->graphs.end();)
            if (ws && it->key.ws == ws->w.base) {
                cudaGraphExecDestroy(it->exec);
                it = code->graphs.erase(it);
            } else {
                ++it;
            }
        mpwsd_workspace_free(ws);
        code->default_ws = ws = nw;
    }
    *out = ws;
    return MPWSD_OK;
}

extern "C" int mpwsd_decode(mpwsd_code *code, const float *y_dev, int64_t B, int L, int T, const mpwsd_opts *opts,
                            uint64_t *cw_dev, uint16_t *flags_dev, void *stream) {
    mpwsd_opts o;
    int st = check_decode_args(code, y_dev, B, L, T, opts, cw_dev, flags_dev, &o);
    if (st) return st;
    if (B == 0) return MPWSD_OK;
    mpwsd_workspace *ws;
    {
        std::lock_guard<std::mutex> lk(code->mu);
        st = default_workspace(code, B, L, &ws);
        if (st) return st;
    }
    return run_decode(code, ws->w, y_dev, B, L, T, o, cw_dev, flags_dev, (cudaStream_t)stream);
}

extern "C" int mpwsd_decode_host(mpwsd_code *code, const float *y_host, int64_t B, int L, int T,
                                 const mpwsd_opts *opts, uint64_t *cw_host, uint16_t *flags_host, void *stream) {
    mpwsd_opts o;
    int st = check_decode_args(code, y_host, B, L, T, opts, cw_host, flags_host, &o);
    if (st) return st;
    if (B == 0) return MPWSD_OK;
    mpwsd_workspace *ws;
    HostIO io;
    io.y = y_host;
    io.cw = cw_host;
    io.fl = flags_host;
    {
        std::lock_guard<std::mutex> lk(code->mu);
        st = default_workspace(code, B, L, &ws);
        if (st) return st;
        cudaError_t e = cudaSuccess;
        if (!code->copy_stream) e = cudaStreamCreateWithFlags(&code->copy_stream, cudaStreamNonBlocking);
        for (auto &ev : code->copy_ev)
            if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        for (auto &ev : code->stage_done)
            if (e == cudaSuccess && !ev) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e, "creating the copy stream");
        if (code->stage_B < B) {
            // a growth waits for the device (cudaFree); graphs keyed on the old buffers never match again
            cudaFree(code->stage_y);
            cudaFree(code->stage_y2);
            cudaFree(code->stage_cw);
            cudaFree(code->stage_fl);
            code->stage_y = nullptr;
            code->stage_y2 = nullptr;
            code->stage_cw = nullptr;
            code->stage_fl = nullptr;
            code->stage_B = 0;
            code->stage_used[0] = code->stage_used[1] = false;  // cudaFree waited for every use
            e = dev_alloc((void **)&code->stage_y, (size_t)B * code->d.n * sizeof(float));
            if (e == cudaSuccess) e = dev_alloc((void **)&code->stage_y2, (size_t)B * code->d.n * sizeof(float));
            if (e == cudaSuccess) e = dev_alloc((void **)&code->stage_cw, (size_t)B * code->d.W * sizeof(uint64_t));
            if (e == cudaSuccess) e = dev_alloc((void **)&code->stage_fl, (size_t)B * sizeof(uint16_t));
            if (e != cudaSuccess) return cuda_fail(e, "allocating the staging buffers");
            code->stage_B = B;
        }
        io.buf = code->stage_next;
        code->stage_next ^= 1;
    }
    st = run_decode(code, ws->w, io.buf ? code->stage_y2 : code->stage_y, B, L, T, o, code->stage_cw, code->stage_fl,
                    (cudaStream_t)stream, &io);
    if (st) return st;
    // everything this call does is on the stream now: the end of its use of the input buffer
    cudaError_t e = cudaEventRecord(code->stage_done[io.buf], (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "recording the end of the call");
    code->stage_used[io.buf] = true;
    return MPWSD_OK;
}

extern "C" int mpwsd_stage1_list(mpwsd_code *code, const float *y_dev, int64_t B, int L, uint64_t *list_cw_dev,
                                 int64_t *list_pm_dev, void *stream) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    if (B < 0 || L < 1 || L > MPWSD_MAX_L) return fail(MPWSD_EINVAL, "need B >= 0 and 1 <= L <= 32");
    if (B > 0 && (!y_dev || !list_cw_dev || !list_pm_dev)) return fail(MPWSD_EINVAL, "NULL buffer");
    if (B == 0) return MPWSD_OK;
    SclArgs sa{};
    sa.y = y_dev;
    sa.B = B;
    sa.L = L;
    sa.mode = 1;
    sa.list_cw = list_cw_dev;
    sa.list_pm = list_pm_dev;
    cudaError_t e = timed_launch(code, MPWSD_KERNEL_SCL, (cudaStream_t)stream,
                                 [&] { return launch_scl(code->d, sa, (cudaStream_t)stream); });
    if (e != cudaSuccess) return cuda_fail(e, "stage-1 launch");
    return MPWSD_OK;
}

static_assert(MPWSD_MAX_OSD_ORDER == kOsdMaxOrder, "the OSD set table covers every allowed order");

extern "C" int mpwsd_osd_list(mpwsd_code *code, const float *y_dev, int64_t B, int order, int L, uint64_t *list_cw_dev,
                              int64_t *list_d_dev, void *stream) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    if (B < 0 || L < 1 || L > MPWSD_MAX_L) return fail(MPWSD_EINVAL, "need B >= 0 and 1 <= L <= 32");
    if (order < 0 || order > MPWSD_MAX_OSD_ORDER) return fail(MPWSD_EINVAL, "order = %d: must be 0..%d", order,
                                                              MPWSD_MAX_OSD_ORDER);
    if (code->d.k > 32) return fail(MPWSD_EUNSUPPORTED, "OSD needs k <= 32 (k = %d)", code->d.k);
    if (B > 0 && (!y_dev || !list_cw_dev || !list_d_dev)) return fail(MPWSD_EINVAL, "NULL buffer");
    if (B == 0) return MPWSD_OK;
    OsdArgs oa{};
    oa.y = y_dev;
    oa.B = B;
    oa.L = L;
    oa.order = order;
    oa.ncand = osd_candidates(code->d.k, order);
    oa.mode = 1;
    oa.list_cw = list_cw_dev;
    oa.list_d = list_d_dev;
    cudaError_t e = timed_launch(code, MPWSD_KERNEL_OSD, (cudaStream_t)stream,
                                 [&] { return launch_osd(code->d, oa, (cudaStream_t)stream); });
    if (e != cudaSuccess) return cuda_fail(e, "OSD launch");
    return MPWSD_OK;
}

extern "C" int mpwsd_score_topk(mpwsd_code *code, int score_mode, const float *y_dev, int64_t B,
                                const int32_t *frame_dev, const uint64_t *cw_dev, int64_t M, float *topk_val_dev,
                                int32_t *topk_idx_dev, void *stream) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    if (score_mode != MPWSD_SCORE_BF16X2 && score_mode != MPWSD_SCORE_FP32 && score_mode != MPWSD_SCORE_FLATS)
        return fail(MPWSD_EINVAL, "score_mode = %d", score_mode);
    if (score_mode == MPWSD_SCORE_BF16X2 && !score_tc_supported(code->d))
        return fail(MPWSD_EUNSUPPORTED, "BF16X2 tensor-core scoring needs n = 64 or 128");
    if (score_mode == MPWSD_SCORE_FLATS && code->d.n_flat == 0)
        return fail(MPWSD_EUNSUPPORTED, "FLATS scoring needs a pattern set of whole cosets of subspaces");
    if (M < 0 || B < 0 || M > 0x7fffffffLL || (M > 0 && B == 0)) return fail(MPWSD_EINVAL, "bad sizes");
    if (M > 0 && (!y_dev || !frame_dev || !cw_dev || !topk_val_dev || !topk_idx_dev))
        return fail(MPWSD_EINVAL, "NULL buffer");
    if (M == 0) return MPWSD_OK;
    ScoreArgs a{};
    a.y = y_dev;
    a.rows = nullptr;
    a.n_rows_dev = nullptr;
    a.n_rows = M;
    a.cw = cw_dev;
    a.row_frame = frame_dev;
    a.L = 1;
    a.topk_val = topk_val_dev;
    a.topk_idx = topk_idx_dev;
    const cudaStream_t s = (cudaStream_t)stream;
    void *prep = nullptr;
    if (score_mode == MPWSD_SCORE_BF16X2) {
        // stream-ordered scratch for y in split form: B x n words, then B norms
        const size_t yhl_bytes = align256((size_t)B * code->d.n * 4);
        cudaError_t e = cudaMallocAsync(&prep, yhl_bytes + (size_t)B * 4, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMallocAsync");
        a.yhl = (const uint32_t *)prep;
        a.l1 = (const float *)((char *)prep + yhl_bytes);
        e = launch_split_prep(code->d, y_dev, B, (uint32_t *)prep, (float *)((char *)prep + yhl_bytes), s);
        if (e != cudaSuccess) {
            cudaFreeAsync(prep, s);
            return cuda_fail(e, "split launch");
        }
    }
    cudaError_t e = launch_score(code, score_mode, a, s);
    if (prep) {
        const cudaError_t ef = cudaFreeAsync(prep, s);
        if (e == cudaSuccess) e = ef;
    }
    if (e != cudaSuccess) return cuda_fail(e, "scoring launch");
    return MPWSD_OK;
}

extern "C" int mpwsd_sync(mpwsd_code *code, void *stream) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
    unsigned long long err = 0;
    e = cudaMemcpy(&err, &code->d.stats->error, sizeof(err), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading the error word");
    if (err) {
        cudaMemset(&code->d.stats->error, 0, sizeof(err));
        return fail(MPWSD_ETIMEOUT, "a bounded device-side wait gave up (code %llu)", err);
    }
    return MPWSD_OK;
}

extern "C" int mpwsd_stats_get(mpwsd_code *code, mpwsd_stats *out) {
    if (!code || !out) return fail(MPWSD_EINVAL, "NULL argument");
    cudaError_t e = cudaDeviceSynchronize();
    DevStats ds;
    if (e == cudaSuccess) e = cudaMemcpy(&ds, code->d.stats, sizeof(ds), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "reading counters");
    out->frames = (int64_t)ds.frames;
    out->stage2_frames = (int64_t)ds.stage2_frames;
    out->trajectories = (int64_t)ds.trajectories;
    out->pattern_evals = (int64_t)ds.pattern_evals;
    out->rerank_candidates = (int64_t)ds.rerank_candidates;
    out->rescans = (int64_t)ds.rescans;
    out->hops = (int64_t)ds.hops;
    out->kernel_launches = code->launches.load();
    return MPWSD_OK;
}

extern "C" int mpwsd_profile_begin(mpwsd_code *code) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    std::lock_guard<std::mutex> lk(code->prof_mu);
    for (auto &r : code->recs) {
        code->pool.push_back(r.start);
        code->pool.push_back(r.stop);
    }
    code->recs.clear();
    code->profiling = true;
    return MPWSD_OK;
}

extern "C" int mpwsd_profile_end(mpwsd_code *code, mpwsd_kernel_time *out) {
    if (!code || !out) return fail(MPWSD_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(code->prof_mu);
    code->profiling = false;
    for (int k = 0; k < MPWSD_KERNEL_KINDS; ++k) {
        out[k].launches = 0;
        out[k].ms = 0.0;
    }
    int status = MPWSD_OK;
    for (auto &r : code->recs) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.stop);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.start, r.stop);
        if (e != cudaSuccess && status == MPWSD_OK) status = cuda_fail(e, "reading kernel timers");
        out[r.kind].launches += 1;
        out[r.kind].ms += ms;
        code->pool.push_back(r.start);
        code->pool.push_back(r.stop);
    }
    code->recs.clear();
    return status;
}

extern "C" int mpwsd_tune_set(mpwsd_code *code, int knob, int value) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    if (knob == MPWSD_TUNE_SPLIT_ITEMS) {
        // units x chunks stays below kSplitItemsPerSm x SMs, the size of the split buffers
        const int cap = kSplitItemsPerSm / 2 * code->d.num_sms;
        if (value < 0 || value > cap) return fail(MPWSD_EINVAL, "split items %d outside 0..%d", value, cap);
    } else if (knob == MPWSD_TUNE_TC_SHAPE) {
        if (!tc_shape_valid(code->d.n, value))
            return fail(MPWSD_EINVAL, "scoring shape %d is not instantiated for n = %d", value, code->d.n);
    } else {
        return fail(MPWSD_EINVAL, "unknown knob %d", knob);
    }
    std::lock_guard<std::mutex> lk(code->mu);
    if (knob == MPWSD_TUNE_SPLIT_ITEMS) code->d.split_items = value;
    else code->d.tc_shape = value;
    for (auto &g : code->graphs) cudaGraphExecDestroy(g.exec);  // recorded with the old value
    code->graphs.clear();
    return MPWSD_OK;
}

extern "C" int mpwsd_tune_get(const mpwsd_code *code, int knob, int *value) {
    if (!code || !value) return fail(MPWSD_EINVAL, "NULL argument");
    if (knob == MPWSD_TUNE_SPLIT_ITEMS) *value = code->d.split_items;
    else if (knob == MPWSD_TUNE_TC_SHAPE) *value = code->d.tc_shape;
    else return fail(MPWSD_EINVAL, "unknown knob %d", knob);
    return MPWSD_OK;
}

extern "C" int mpwsd_stats_reset(mpwsd_code *code) {
    if (!code) return fail(MPWSD_EINVAL, "code is NULL");
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemset(code->d.stats, 0, sizeof(DevStats));
    if (e != cudaSuccess) return cuda_fail(e, "resetting counters");
    code->launches = 0;
    return MPWSD_OK;
}

// ---- host pattern enumeration ------------------------------------------------

extern "C" int mpwsd_enumerate_codewords(int n, const uint8_t *frozen, const int *weights, int n_weights,
                                         uint64_t *out, int64_t max_out, int64_t *count) {
    if (n != 32 && n != 64 && n != 128) return fail(MPWSD_EINVAL, "n = %d: must be 32, 64 or 128", n);
    if (!frozen || !weights || n_weights < 1 || !count) return fail(MPWSD_EINVAL, "NULL argument");
    for (int i = 0; i < n_weights; ++i) {
        if (weights[i] < 1 || weights[i] > n) return fail(MPWSD_EINVAL, "weight %d out of range", weights[i]);
        if (i && weights[i] <= weights[i - 1]) return fail(MPWSD_EINVAL, "weights must be strictly ascending");
    }
    std::vector<int> info;
    for (int i = 0; i < n; ++i)
        if (!frozen[i]) info.push_back(i);
    const int k = (int)info.size();
    if (k < 1 || k > 40) return fail(MPWSD_EINVAL, "k = %d: enumeration supports 1..40", k);
    const int W = (n + 63) / 64;
    // Gray-code walk: bit b of the message integer a is information index
    // info[k-1-b] (lowest index = most significant bit); each step XORs one row.
    std::vector<uint64_t> row((size_t)k * 2, 0);
    for (int b = 0; b < k; ++b) {
        const int i = info[k - 1 - b];
        for (int j = 0; j < n; ++j)
            if (kron_entry(i, j)) row[(size_t)b * 2 + j / 64] |= 1ull << (j % 64);
    }
    int wclass[129];
    for (int w = 0; w <= 128; ++w) wclass[w] = -1;
    for (int i = 0; i < n_weights; ++i) wclass[weights[i]] = i;
    struct Rec {
        int cls;
        uint64_t a;
        uint64_t c0, c1;
    };
    std::vector<Rec> recs;
    uint64_t c0 = 0, c1 = 0;
    const uint64_t total = 1ull << k;
    for (uint64_t s = 1; s < total; ++s) {
        const int b = __builtin_ctzll(s);
        c0 ^= row[(size_t)b * 2];
        c1 ^= row[(size_t)b * 2 + 1];
        const int w = __builtin_popcountll(c0) + __builtin_popcountll(c1);
        if (wclass[w] >= 0) recs.push_back({wclass[w], s ^ (s >> 1), c0, c1});
    }
    std::sort(recs.begin(), recs.end(), [](const Rec &x, const Rec &y) {
        return x.cls != y.cls ? x.cls < y.cls : x.a < y.a;
    });
    *count = (int64_t)recs.size();
    if (!out) return MPWSD_OK;
    if ((int64_t)recs.size() > max_out) return fail(MPWSD_EINVAL, "%lld codewords do not fit in max_out", (long long)recs.size());
    for (size_t i = 0; i < recs.size(); ++i) {
        out[i * W] = recs[i].c0;
        if (W > 1) out[i * W + 1] = recs[i].c1;
    }
    return MPWSD_OK;
}

// ---- allocation-free decode ---------------------------------------------------
//
// Some callers cannot allocate device memory at decode time: serving threads
// that must not touch the allocator once warmed up, and hosts whose device
// memory is owned by another allocator that the library must not bypass. For
// them, mpwsd_decode_noalloc runs the same decode with its scratch in one
// file-scope device array of fixed size. The array holds the workspace layout
// only; the pattern split of the scoring kernel has no buffers there, so this
// path scores without it (same results).

namespace {

constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;  // 4 MiB per device, held until process exit
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
void *g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device, looked up once
// per device (with that device current). In host code the array's name is
// only a host-side handle, never a device address.
int noalloc_scratch(void **out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return fail(MPWSD_EUNSUPPORTED, "device %d beyond %d", dev, kMaxDevices);
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress of the scratch array");
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return MPWSD_OK;
}

}  // namespace

extern "C" int mpwsd_decode_noalloc(mpwsd_code *code, const float *y_dev, int64_t B, int L, int T,
                                    const mpwsd_opts *opts, uint64_t *cw_dev, uint16_t *flags_dev, void *stream) {
    mpwsd_opts o;
    int st = check_decode_args(code, y_dev, B, L, T, opts, cw_dev, flags_dev, &o);
    if (st) return st;
    if (code->profiling)
        return fail(MPWSD_EINVAL, "kernel timing is on for this handle (it creates CUDA events); "
                                  "call mpwsd_profile_end first");
    const size_t need = ws_layout(code->d, std::max<int64_t>(B, 1), L, nullptr);
    if (need > kNoAllocScratchBytes)
        return fail(MPWSD_EINVAL,
                    "B = %lld frames with L = %d need %zu bytes of scratch; the allocation-free entry point has %zu "
                    "(about %lld trajectories B*L for n = %d)",
                    (long long)B, L, need, kNoAllocScratchBytes,
                    (long long)(kNoAllocScratchBytes / (need / std::max<int64_t>((int64_t)B * L, 1))), code->d.n);
    if (B == 0) return MPWSD_OK;
    void *base = nullptr;
    st = noalloc_scratch(&base);
    if (st) return st;
    Workspace ws;
    ws.base = base;
    ws.bytes = need;
    ws.max_B = B;
    ws.max_L = L;
    cudaGetDevice(&ws.device);
    ws_layout(code->d, B, L, &ws);
    return decode_impl(code, ws, y_dev, B, L, T, o, cw_dev, flags_dev, (cudaStream_t)stream);
}

// ---- continuous stage-2 batching (pools) ---------------------------------------
//
// A pool keeps the stage-2 state of one code across calls. mpwsd_pool_submit
// runs stage 1 on a batch; its CRC-failing frames take slots of the pool and
// their trajectories join the rows of the next step. mpwsd_pool_step runs one
// iteration of Algorithm 1 (score, exact re-rank, hop, twin retirement) on
// every live row, whatever submission it came from, then writes the results of
// the frames that finished and frees their slots. Every trajectory ends after
// at most T steps, so a submission's frames are all done T steps after it: the
// host bounds the frames in flight by the submissions of the last T steps and
// needs no read-back.

struct mpwsd_pool {
    mpwsd_code *code = nullptr;
    Workspace w;
    int L = 0, T = 0;
    mpwsd_opts o{};
    int64_t cap = 0;
    int64_t steps = 0, submits = 0, in_flight = 0;
    std::deque<std::pair<int64_t, int64_t>> recent;  // (steps before the submission, frames)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    int graph_kernels = 0;
};

static int pool_step_launches(mpwsd_pool *p, cudaStream_t s) {
    mpwsd_code *code = p->code;
    CodeDev &d = code->d;
    Workspace &ws = p->w;
    ScoreArgs a{};
    a.y = ws.pool.slot_y;
    a.rows = ws.act[0];
    a.n_rows_dev = ws.counters + 1;
    a.cw = ws.traj_cw;
    a.slot_frame = ws.slot_frame;
    a.L = p->L;
    a.topk_val = ws.topk_val;
    a.topk_idx = ws.topk_idx;
    a.yhl = ws.slot_yhl;
    a.l1 = ws.slot_l1;
    a.split_val = ws.split_val;
    a.split_idx = ws.split_idx;
    a.unit_done = ws.unit_done;
    a.split_items = d.split_items;
    const float *y = ws.pool.slot_y;
    const int L = p->L;
    cudaError_t e = score_and_hop(code, p->o.score_mode, a, ws, 0, L, y, s);
    if (e != cudaSuccess) return cuda_fail(e, "scoring / hop launch");
    e = timed_launch(code, MPWSD_KERNEL_RESCAN, s, [&] { return launch_rescan(d, ws, 0, L, y, s); });
    if (e == cudaSuccess) e = timed_launch(code, MPWSD_KERNEL_HOP, s, [&] { return launch_dedup(d, ws, 0, L, s); });
    if (e == cudaSuccess) e = timed_launch(code, MPWSD_KERNEL_FINAL, s, [&] { return launch_pool_final(d, ws, L, s); });
    if (e == cudaSuccess) e = timed_launch(code, MPWSD_KERNEL_FINAL, s, [&] { return launch_pool_end(d, ws, s); });
    if (e != cudaSuccess) return cuda_fail(e, "pool step launch");
    return MPWSD_OK;
}

// Device layout of a pool: the workspace arrays for (max_frames, L), the
// buffers of the scoring kernel's pattern split, and the pool's own arrays.
struct PoolLayout {
    size_t sv, si, ud, ctr, ring, live, comp, dst, y, total;
    size_t split_items;
};
static PoolLayout pool_layout(const CodeDev &d, int64_t max_frames, int L) {
    PoolLayout l{};
    size_t off = ws_layout(d, max_frames, L, nullptr);
    auto take = [&](size_t bytes) {
        size_t r = off;
        off += align256(bytes);
        return r;
    };
    l.split_items = (size_t)kSplitItemsPerSm * std::max(d.num_sms, 1);
    const size_t split_entries = l.split_items * 256 * kTopK;
    l.sv = take(split_entries * 4);
    l.si = take(split_entries * 4);
    l.ud = take(l.split_items * 4);
    l.ctr = take(64 * 4);
    l.ring = take((size_t)max_frames * 4);
    l.live = take((size_t)max_frames * 4);
    l.comp = take((size_t)max_frames * 4);
    l.dst = take((size_t)max_frames * 3 * 8);
    l.y = take((size_t)max_frames * d.n * 4);
    l.total = off;
    return l;
}

extern "C" int mpwsd_pool_bytes(const mpwsd_code *code, int64_t max_frames, int L, size_t *bytes) {
    if (!code || !bytes) return fail(MPWSD_EINVAL, "NULL argument");
    if (L < 1 || L > MPWSD_MAX_L) return fail(MPWSD_EINVAL, "L = %d: must be 1..%d", L, MPWSD_MAX_L);
    if (max_frames < 1 || max_frames * L > 0x7fffffffLL)
        return fail(MPWSD_EINVAL, "max_frames = %lld: need 1 <= max_frames and max_frames * L < 2^31", (long long)max_frames);
    *bytes = pool_layout(code->d, max_frames, L).total;
    return MPWSD_OK;
}

extern "C" int mpwsd_pool_create(mpwsd_code *code, int64_t max_frames, int L, int T, const mpwsd_opts *opts,
                                 mpwsd_pool **out) {
    if (!out) return fail(MPWSD_EINVAL, "out is NULL");
    *out = nullptr;
    mpwsd_opts o;
    int st = check_decode_args(code, nullptr, 0, L, T, opts, nullptr, nullptr, &o);
    if (st) return st;
    if (max_frames < 1 || max_frames * L > 0x7fffffffLL)
        return fail(MPWSD_EINVAL, "max_frames = %lld: need 1 <= max_frames and max_frames * L < 2^31", (long long)max_frames);
    const CodeDev &d = code->d;
    const PoolLayout lay = pool_layout(d, max_frames, L);
    const size_t o_sv = lay.sv, o_si = lay.si, o_ud = lay.ud, o_ctr = lay.ctr, o_ring = lay.ring, o_live = lay.live;
    const size_t o_comp = lay.comp, o_dst = lay.dst, o_y = lay.y, off = lay.total;
    const size_t split_items = lay.split_items;
    mpwsd_pool *p = new (std::nothrow) mpwsd_pool();
    if (!p) return fail(MPWSD_ENOMEM, "host allocation");
    p->code = code;
    p->L = L;
    p->T = T;
    p->o = o;
    p->cap = max_frames;
    cudaError_t e = dev_alloc(&p->w.base, off);
    if (e != cudaSuccess) {
        delete p;
        cudaGetLastError();
        return cuda_fail(e, "pool allocation");
    }
    p->w.bytes = off;
    p->w.max_B = max_frames;
    p->w.max_L = L;
    cudaGetDevice(&p->w.device);
    ws_layout(d, max_frames, L, &p->w);
    char *b = (char *)p->w.base;
    p->w.split_val = (float *)(b + o_sv);
    p->w.split_idx = (int *)(b + o_si);
    p->w.unit_done = (int *)(b + o_ud);
    PoolDev &pd = p->w.pool;
    pd.cap = (int)max_frames;
    pd.T = T;
    pd.ctr = (int *)(b + o_ctr);
    pd.free_ring = (int *)(b + o_ring);
    pd.live = (int *)(b + o_live);
    pd.completed = (int *)(b + o_comp);
    pd.dst = (unsigned long long *)(b + o_dst);
    pd.slot_y = (float *)(b + o_y);
    // every slot free; no rows; counters at zero
    std::vector<int> ring((size_t)max_frames);
    for (int64_t i = 0; i < max_frames; ++i) ring[(size_t)i] = (int)i;
    int ctr[64] = {0};
    ctr[kPoolPush] = (int)max_frames;
    e = cudaMemset(p->w.counters, 0, 64 * sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->w.unit_done, 0, split_items * sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpy(pd.ctr, ctr, sizeof(ctr), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(pd.free_ring, ring.data(), ring.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->w.base);
        delete p;
        return cuda_fail(e, "pool initialisation");
    }
    *out = p;
    return MPWSD_OK;
}

extern "C" void mpwsd_pool_free(mpwsd_pool *p) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->graph) cudaGraphExecDestroy(p->graph);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    cudaFree(p->w.base);
    delete p;
}

extern "C" int mpwsd_pool_free_frames(const mpwsd_pool *p, int64_t *frames) {
    if (!p || !frames) return fail(MPWSD_EINVAL, "NULL argument");
    *frames = p->cap - p->in_flight;
    return MPWSD_OK;
}

extern "C" int mpwsd_pool_submit(mpwsd_pool *p, const float *y_dev, int64_t B, uint64_t *cw_dev, uint16_t *flags_dev,
                                 int32_t *done_dev, void *stream) {
    if (!p) return fail(MPWSD_EINVAL, "pool is NULL");
    if (B < 0) return fail(MPWSD_EINVAL, "B < 0");
    if (B > 0 && (!y_dev || !cw_dev || !flags_dev)) return fail(MPWSD_EINVAL, "NULL buffer");
    if (B > p->cap - p->in_flight)
        return fail(MPWSD_ENOMEM, "pool full: %lld frames submitted, %lld free until earlier frames finish",
                    (long long)B, (long long)(p->cap - p->in_flight));
    if (B == 0) return MPWSD_OK;
    cudaError_t e = stage1_launch(p->code, p->w, y_dev, 0, B, p->L, p->o, cw_dev, flags_dev, (cudaStream_t)stream,
                                  done_dev, (int)p->submits);
    if (e != cudaSuccess) return cuda_fail(e, "stage-1 launch");
    p->submits++;
    p->in_flight += B;
    p->recent.emplace_back(p->steps, B);
    return MPWSD_OK;
}

extern "C" int mpwsd_pool_step(mpwsd_pool *p, void *stream) {
    if (!p) return fail(MPWSD_EINVAL, "pool is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    mpwsd_code *code = p->code;
    int st = MPWSD_OK;
    if (p->o.use_graph && !code->profiling) {
        if (!p->graph) {
            cudaError_t e = cudaSuccess;
            if (!p->cap_stream) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed);
            if (e != cudaSuccess) return cuda_fail(e, "capturing the pool step");
            t_capturing = true;
            st = pool_step_launches(p, p->cap_stream);
            t_capturing = false;
            cudaGraph_t graph = nullptr;
            e = cudaStreamEndCapture(p->cap_stream, &graph);
            if (st) {
                if (graph) cudaGraphDestroy(graph);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture");
            p->graph_kernels = graph_kernel_nodes(graph);
            e = cudaGraphInstantiate(&p->graph, graph, 0);
            cudaGraphDestroy(graph);
            if (e != cudaSuccess) return cuda_fail(e, "cudaGraphInstantiate");
        }
        cudaError_t e = cudaGraphLaunch(p->graph, s);
        if (e != cudaSuccess) return cuda_fail(e, "cudaGraphLaunch");
        code->launches += p->graph_kernels;
    } else {
        st = pool_step_launches(p, s);
        if (st) return st;
    }
    p->steps++;
    // a submission made before step k is done after step k + T - 1
    while (!p->recent.empty() && p->recent.front().first + p->T <= p->steps) {
        p->in_flight -= p->recent.front().second;
        p->recent.pop_front();
    }
    return MPWSD_OK;
}
