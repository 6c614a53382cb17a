// Stage 1 by ordered-statistics decoding, OSD(order): the anchor list of the
// RM experiment (Sec. IV-C; the paper names OSD without details, this is the
// standard construction). For each frame:
//   1. hard decisions hd_j = [y_j < 0], reliabilities |y_j| on the 2^-19 grid;
//   2. positions in decreasing reliability, ties to the lower index;
//   3. the most reliable basis: walking the positions in that order, a
//      position joins when its generator column is independent of the ones
//      chosen so far; Gauss-Jordan makes row t of G_sys the codeword that is 1
//      at the t-th chosen position and 0 at the others;
//   4. c0 = XOR of the rows t whose basis position has hd = 1;
//   5. candidates c0 XOR (rows of F) for every set F of at most `order` rows,
//      numbered by |F|, then lexicographically;
//   6. discrepancy D(c) = sum_j |y_j| [c_j != hd_j] (ED(c) = ||y||^2 + n -
//      2 sum |y| + 4 D(c)): exact integers;
//   7. the min(L, #candidates) smallest (D, number), ascending.
// GPU mapping: one warp per frame. Element j of the frame sits in lane j % 32
// (so a ballot over lanes gives 32 consecutive bits of a bit vector); the
// generator rows sit one per lane (k <= 32) for the elimination; D of a
// candidate is sum_b popc(e & plane_b) << b over the bit planes of |y|, no
// data-dependent loops; the running list lives one entry per lane, and a
// candidate that beats its last entry is inserted with a ballot and one
// shuffle. The decode tail (CRC early exit, slots, trajectories) matches the
// SC-list kernel's.
#include <cuda_bf16.h>

#include "common.cuh"

namespace mpwsd {
namespace {

constexpr int kOsdWarps = 4;
constexpr unsigned kAll = 0xffffffffu;

__device__ __forceinline__ uint32_t binom(int n, int r) {  // C(n, r) for 0 <= r <= 4
    if (n < r || n < 0) return 0;
    switch (r) {
        case 0: return 1;
        case 1: return (uint32_t)n;
        case 2: return (uint32_t)(n * (n - 1) / 2);
        case 3: return (uint32_t)(n * (n - 1) * (n - 2) / 6);
        default: return (uint32_t)((n * (n - 1) * (n - 2) / 6) * (n - 3) / 4);
    }
}

// number of a candidate: sets of fewer rows first, then the lexicographic rank
// of the sorted set (c[0] < ... < c[w-1]) among the w-subsets of k rows
__device__ __forceinline__ uint32_t cand_number(int k, int w, const int (&c)[4]) {
    uint32_t base = 0;
    for (int v = 0; v < w; ++v) base += binom(k, v);
    uint32_t r = binom(k, w) - 1;
    for (int t = 0; t < w; ++t) r -= binom(k - 1 - c[t], w - t);
    return base + r;
}

// inverse of cand_number
__device__ __forceinline__ int cand_set(int k, uint32_t idx, int (&c)[4]) {
    int w = 0;
    while (w < 4 && idx >= binom(k, w)) idx -= binom(k, w++);
    int start = 0;
    for (int t = 0; t < w; ++t) {
        for (int v = start; v < k; ++v) {
            const uint32_t rest = binom(k - v - 1, w - t - 1);
            if (idx < rest) {
                c[t] = v;
                start = v + 1;
                break;
            }
            idx -= rest;
        }
    }
    return w;
}

template <int N>
struct OsdSmem {
    static constexpr int W = (N + 63) / 64;
    int g[kOsdWarps][N];              // round(y 2^19)
    uint32_t key[kOsdWarps][N];       // |g| << 8 | (255 - j): larger = more reliable
    uint8_t perm[kOsdWarps][N];       // positions by decreasing reliability
    uint8_t mrb[kOsdWarps][32];       // basis position of pivot t
    uint64_t gs[kOsdWarps][32][W];    // G_sys rows by pivot order
    uint64_t plane[kOsdWarps][24][W]; // bit planes of |g|
};

template <int N>
__device__ __forceinline__ uint32_t discrepancy(const uint64_t (&e)[(N + 63) / 64], const uint64_t (*plane)[(N + 63) / 64],
                                                int nb) {
    constexpr int W = (N + 63) / 64;
    uint32_t d = 0;
    for (int b = 0; b < nb; ++b) {
        int cnt = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) cnt += __popcll(e[w] & plane[b][w]);
        d += (uint32_t)cnt << b;
    }
    return d;
}

template <int N>
__global__ void __launch_bounds__(kOsdWarps * 32) osd_kernel(const OsdArgs a, const CodeDev c) {
    constexpr int W = (N + 63) / 64;
    constexpr int EPL = N / 32;  // elements per lane: element j = lane + 32 e
    __shared__ OsdSmem<N> sm;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int k = c.k;
    const int L = a.L;
    for (int64_t f = (int64_t)blockIdx.x * kOsdWarps + warp; f < a.B; f += (int64_t)gridDim.x * kOsdWarps) {
        // ---- 1. hard decisions, reliabilities, bit planes ----
        int g[EPL];
        uint32_t hdh[EPL];  // 32-bit halves of hd: half e holds elements 32e .. 32e+31
        int asum = 0;
        uint32_t amax = 0;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            const int j = lane + 32 * e;
            g[e] = grid_q(a.y[f * N + j]);
            const uint32_t ag = (uint32_t)abs(g[e]);
            asum += (int)ag;
            amax = max(amax, ag);
            sm.g[warp][j] = g[e];
            sm.key[warp][j] = (ag << 8) | (uint32_t)(255 - j);
            hdh[e] = __ballot_sync(kAll, g[e] < 0);
        }
        asum = __reduce_add_sync(kAll, asum);  // sum_j |g_j| < 2^30
        amax = __reduce_max_sync(kAll, amax);
        const int nb = 32 - __clz((int)amax);
        for (int b = 0; b < nb; ++b) {
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint32_t lo = __ballot_sync(kAll, ((uint32_t)abs(g[(2 * w) % EPL]) >> b) & 1u);
                const uint32_t hi = (2 * w + 1 < EPL) ? __ballot_sync(kAll, ((uint32_t)abs(g[(2 * w + 1) % EPL]) >> b) & 1u) : 0u;
                if (lane == 0) sm.plane[warp][b][w] = (uint64_t)lo | ((uint64_t)hi << 32);
            }
        }
        uint64_t hdw[W];
#pragma unroll
        for (int w = 0; w < W; ++w)
            hdw[w] = (uint64_t)hdh[(2 * w) % EPL] | ((2 * w + 1 < EPL) ? (uint64_t)hdh[(2 * w + 1) % EPL] << 32 : 0ull);
        __syncwarp();
        // ---- 2. positions by decreasing reliability (rank by counting; keys are distinct) ----
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            const int j = lane + 32 * e;
            const uint32_t kj = sm.key[warp][j];
            int r = 0;
            for (int i = 0; i < N; ++i) r += sm.key[warp][i] > kj;
            sm.perm[warp][r] = (uint8_t)j;
        }
        __syncwarp();
        // ---- 3. Gauss-Jordan with pivots in reliability order ----
        uint64_t row[W];
#pragma unroll
        for (int w = 0; w < W; ++w) row[w] = lane < k ? c.gen_rows[lane * W + w] : 0ull;
        bool used = lane >= k;
        int piv = 0, found = 0;
        for (int q = 0; q < N && found < k; ++q) {
            const int p = sm.perm[warp][q];
            const bool bit = lane < k && ((row[p >> 6] >> (p & 63)) & 1ull);
            const unsigned m = __ballot_sync(kAll, bit && !used);
            if (!m) continue;  // column dependent on the chosen ones
            const int r = __ffs(m) - 1;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint64_t pw = __shfl_sync(kAll, row[w], r);
                if (bit && lane != r) row[w] ^= pw;
            }
            if (lane == r) {
                used = true;
                piv = found;
            }
            if (lane == 0) sm.mrb[warp][found] = (uint8_t)p;
            ++found;
        }
        __syncwarp();
        // ---- 4. G_sys by pivot order, c0, e0 = c0 xor hd ----
        bool take = false;
        if (lane < k) {
#pragma unroll
            for (int w = 0; w < W; ++w) sm.gs[warp][piv][w] = row[w];
            const int p = sm.mrb[warp][piv];
            take = (hdw[p >> 6] >> (p & 63)) & 1ull;
        }
        uint64_t e0[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t x = take ? row[w] : 0ull;
            const uint32_t lo = __reduce_xor_sync(kAll, (uint32_t)x), hi = __reduce_xor_sync(kAll, (uint32_t)(x >> 32));
            e0[w] = (((uint64_t)hi << 32) | lo) ^ hdw[w];
        }
        __syncwarp();
        // ---- 5-7. candidates, their discrepancy, the running list (one entry per lane) ----
        const uint64_t (*plane)[W] = sm.plane[warp];
        unsigned long long lkey = ~0ull;  // list entry `lane` (D << 32 | number), ascending
        auto offer = [&](bool valid, unsigned long long key) {
            unsigned long long thr = __shfl_sync(kAll, lkey, L - 1);
            unsigned m = __ballot_sync(kAll, valid && key < thr);
            while (m) {
                const int s = __ffs(m) - 1;
                m &= m - 1;
                const unsigned long long x = __shfl_sync(kAll, key, s);
                if (x >= thr) continue;
                const int pos = __popc(__ballot_sync(kAll, lkey < x));
                const unsigned long long prev = __shfl_up_sync(kAll, lkey, 1);
                lkey = lane == pos ? x : (lane > pos ? prev : lkey);
                if (lane >= L) lkey = ~0ull;
                thr = __shfl_sync(kAll, lkey, L - 1);
            }
        };
        auto score = [&](int w, const int (&cs)[4]) {
            uint64_t e[W];
#pragma unroll
            for (int x = 0; x < W; ++x) e[x] = e0[x];
            for (int t = 0; t < w; ++t)
#pragma unroll
                for (int x = 0; x < W; ++x) e[x] ^= sm.gs[warp][cs[t]][x];
            const uint32_t d = discrepancy<N>(e, plane, nb);
            return ((unsigned long long)d << 32) | cand_number(k, w, cs);
        };
        {
            int cs[4] = {0, 0, 0, 0};
            offer(lane == 0, score(0, cs));
        }
        if (a.order >= 1) {
            int cs[4] = {lane, 0, 0, 0};
            offer(lane < k, lane < k ? score(1, cs) : ~0ull);
        }
        if (a.order >= 2)
            for (int i = 0; i + 1 < k; ++i) {
                const int l = i + 1 + lane;
                int cs[4] = {i, l, 0, 0};
                offer(l < k, l < k ? score(2, cs) : ~0ull);
            }
        if (a.order >= 3)
            for (int i = 0; i + 2 < k; ++i)
                for (int i2 = i + 1; i2 + 1 < k; ++i2)
                    for (int l = i2 + 1 + lane; l - lane < k; l += 32) {
                        int cs[4] = {i, i2, l, 0};
                        offer(l < k, l < k ? score(3, cs) : ~0ull);
                    }
        if (a.order >= 4)
            for (int i = 0; i + 3 < k; ++i)
                for (int i2 = i + 1; i2 + 2 < k; ++i2)
                    for (int i3 = i2 + 1; i3 + 1 < k; ++i3) {
                        const int l = i3 + 1 + lane;
                        int cs[4] = {i, i2, i3, l};
                        offer(l < k, l < k ? score(4, cs) : ~0ull);
                    }
        // entry `lane` of the list: its codeword
        const int count = __popc(__ballot_sync(kAll, lkey != ~0ull));
        const bool valid = lane < count;
        uint64_t cw[W];
        uint32_t dval = 0;
        {
            int cs[4] = {0, 0, 0, 0};
            const int w = valid ? cand_set(k, (uint32_t)lkey, cs) : 0;
#pragma unroll
            for (int x = 0; x < W; ++x) cw[x] = e0[x] ^ hdw[x];
            for (int t = 0; t < w; ++t)
#pragma unroll
                for (int x = 0; x < W; ++x) cw[x] ^= sm.gs[warp][cs[t]][x];
            dval = (uint32_t)(lkey >> 32);
        }
        if (a.mode == 1) {
            if (valid) {
#pragma unroll
                for (int x = 0; x < W; ++x) a.list_cw[(f * L + lane) * W + x] = cw[x];
                a.list_d[f * L + lane] = (int64_t)dval;
            }
            __syncwarp();
            continue;
        }
        // ---- decode: CRC early exit (Sec. III-A), else the list becomes the anchors ----
        bool ok = false;
        if (a.use_crc && valid) {
            unsigned syn = 0;
            for (int b = 0; b < c.crc_len; ++b) {
                int p = 0;
#pragma unroll
                for (int x = 0; x < W; ++x) p += __popcll(cw[x] & c.crc_masks[(size_t)b * W + x]);
                syn |= (unsigned)(p & 1);
            }
            ok = syn == 0;
        }
        const unsigned okm = __ballot_sync(kAll, ok && (a.rule == MPWSD_RULE_ANY || lane == 0));
        if (okm) {
            if (lane == __ffs(okm) - 1) {
#pragma unroll
                for (int x = 0; x < W; ++x) a.cw_out[f * W + x] = cw[x];
                a.flags_out[f] = (uint16_t)MPWSD_FLAG_CRC_OK;
            }
            __syncwarp();
            continue;
        }
        int slot = 0, base = 0;
        if (lane == 0) {
            slot = atomicAdd(&a.ws.counters[0], 1);
            base = atomicAdd(&a.ws.counters[1], count);
            a.ws.slot_frame[slot] = (int)f;
            a.ws.slot_l1[slot] = (float)asum * (1.0f / 524288.0f);
        }
        slot = __shfl_sync(kAll, slot, 0);
        base = __shfl_sync(kAll, base, 0);
        if (a.write_yhl) {
            // y in the split form the tensor-core scoring consumes (see the SC-list kernel)
            uint32_t *dst = a.ws.slot_yhl + (int64_t)slot * N;
            for (int w2 = lane; w2 < N / 2; w2 += 32) {
                uint32_t h2 = 0, l2 = 0;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const float v = (float)sm.g[warp][2 * w2 + e] * (1.0f / 524288.0f);
                    const __nv_bfloat16 h = __float2bfloat16_rn(v);
                    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
                    h2 |= (uint32_t)__bfloat16_as_ushort(h) << (16 * e);
                    l2 |= (uint32_t)__bfloat16_as_ushort(l) << (16 * e);
                }
                dst[w2] = h2;
                dst[N / 2 + w2] = l2;
            }
        }
        if (lane < L) {
            const int64_t t = (int64_t)slot * L + lane;
            uint64_t *dst = a.ws.traj_cw + t * W;
            if (valid) {
#pragma unroll
                for (int x = 0; x < W; ++x) dst[x] = cw[x];
                // sum_j g_j x_j = sum |g| - 2 D (a sample agrees in sign with x_j unless it counts in D)
                a.ws.traj_D[t] = ((double)2 * (double)dval - (double)asum) * (1.0 / 524288.0);
                a.ws.traj_state[t] = kTrajValid;
                a.ws.act[0][base + lane] = (int)t;
            } else {
#pragma unroll
                for (int x = 0; x < W; ++x) dst[x] = 0;
                a.ws.traj_D[t] = CUDART_INF;
                a.ws.traj_state[t] = 0;
            }
        }
        __syncwarp();
    }
}

template <int N>
cudaError_t launch_n(const CodeDev &c, const OsdArgs &a, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((a.B + kOsdWarps - 1) / kOsdWarps, (int64_t)c.num_sms * 16);
    if (blocks <= 0) return cudaSuccess;
    osd_kernel<N><<<(unsigned)blocks, kOsdWarps * 32, 0, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_osd(const CodeDev &c, const OsdArgs &a, cudaStream_t s) {
    if (c.k > 32 || a.L < 1 || a.L > 32 || a.order < 0 || a.order > 4) return cudaErrorInvalidValue;
    if (c.n == 32) return launch_n<32>(c, a, s);
    if (c.n == 64) return launch_n<64>(c, a, s);
    if (c.n == 128) return launch_n<128>(c, a, s);
    return cudaErrorNotSupported;
}

}  // namespace mpwsd
