// Stage 1 by ordered-statistics decoding, OSD(order): the anchor list of the
// RM experiment (Sec. IV-A; the paper names OSD without details, this is the
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
// (so a ballot over lanes gives 32 consecutive bits of a bit vector). The
// positions are ranked by a bitonic sort of (|g| << 8 | 255 - j) keys held in
// registers. The generator rows sit one per lane (k <= 32) for the
// elimination and are then moved so that lane t holds row t of G_sys. The
// candidates come from a table of row sets in candidate-number order, 32 per
// step, one per lane; a lane forms its error pattern from the rows by
// shuffles, and D = sum over the bytes of the pattern of a per-frame byte
// table (tab[b][v] = sum of |g_j| over the set bits of v, j = 8b + bit), so a
// candidate costs n/8 lookups. The running list lives one entry per lane; a
// candidate below its last entry is inserted with a ballot and one shuffle.
// The decode tail (CRC early exit, slots, trajectories) matches the SC-list
// kernel's.
#include <cuda_bf16.h>

#include "common.cuh"

namespace mpwsd {
namespace {

constexpr int kOsdWarps = 4;
constexpr unsigned kAll = 0xffffffffu;
constexpr int kMergeMin = 8;  // more entries than this in one step: sort and merge instead of inserting

// The discrepancy tables cut each 64-position word of a pattern into chunks of
// 6 bits (the last one narrower): table t of word x covers positions 64 x + 6 c
// .. + width - 1, and entry v is the sum of |g| over the set bits of v. A table
// has 64 entries (two per shared-memory bank), so the 32 lanes of a lookup
// meet at most two-way bank conflicts, and a warp's tables take 5.5 KB (n =
// 128), which leaves room for 32 warps per SM.
template <int N>
struct OsdGeom {
    static constexpr int W = (N + 63) / 64;
    static constexpr int BITS = N < 64 ? N : 64;  // positions per word
    static constexpr int CPW = (BITS + 5) / 6;    // chunks per word
    static constexpr int NT = W * CPW;            // tables
};

template <int N>
struct OsdWarpSmem {
    uint32_t tab[OsdGeom<N>::NT][64];  // first: 256-byte aligned (see osd_kernel)
    uint32_t a[N];                     // |round(y 2^19)|
    uint8_t perm[N];                   // positions by decreasing reliability
    uint8_t mrb[32];                   // basis position of pivot t
    uint8_t lane_of[32];               // lane that holds the row of pivot t after the elimination
    uint8_t pad[(256 - (N * 5 + 64) % 256) % 256];
};

// bitonic sort of the warp's N keys (element e of lane l is entry 32 e + l),
// descending; keys are distinct
template <int N>
__device__ __forceinline__ void sort_desc(uint32_t (&key)[N / 32], int lane) {
    constexpr int EPL = N / 32;
#pragma unroll
    for (int s = 2; s <= N; s <<= 1) {
#pragma unroll
        for (int d = s >> 1; d > 0; d >>= 1) {
            if (d >= 32) {
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    const int ep = e ^ (d >> 5);
                    if (ep > e) {
                        // entry 32 e + lane is the lower one of the pair
                        const bool desc = ((32 * e + lane) & s) == 0;
                        const uint32_t mx = max(key[e], key[ep]), mn = min(key[e], key[ep]);
                        key[e] = desc ? mx : mn;
                        key[ep] = desc ? mn : mx;
                    }
                }
            } else {
                const bool lower = (lane & d) == 0;
#pragma unroll
                for (int e = 0; e < EPL; ++e) {
                    const uint32_t o = __shfl_xor_sync(kAll, key[e], d);
                    const bool desc = ((32 * e + lane) & s) == 0;
                    key[e] = (lower == desc) ? max(key[e], o) : min(key[e], o);
                }
            }
        }
    }
}

// bit p of a W-word vector, without a dynamically indexed (local-memory) array
template <int W>
__device__ __forceinline__ bool bit_at(const uint64_t (&v)[W], int p) {
    uint64_t x = v[0];
#pragma unroll
    for (int w = 1; w < W; ++w) x = (p >> 6) == w ? v[w] : x;
    return (x >> (p & 63)) & 1ull;
}

// D of the pattern e: one lookup per chunk. tab_base is the shared-window
// address of the warp's tables (256-byte aligned, so the entry offset ORs in).
template <int N>
__device__ __forceinline__ uint32_t discrepancy(const uint64_t (&e)[(N + 63) / 64], uint32_t tab_base) {
    using Gm = OsdGeom<N>;
    uint32_t d[4] = {0u, 0u, 0u, 0u};  // four partial sums: independent add chains
    uint32_t pend = 0u;                 // values are added in pairs (three-input adds)
#pragma unroll
    for (int x = 0; x < Gm::W; ++x) {
        const uint32_t lo = (uint32_t)e[x], hi = (uint32_t)(e[x] >> 32);
#pragma unroll
        for (int cc = 0; cc < Gm::CPW; ++cc) {
            const int s = 6 * cc;
            const int wd = Gm::BITS - s < 6 ? Gm::BITS - s : 6;
            const uint32_t mask4 = ((1u << wd) - 1u) << 2;  // entry v at byte offset 4 v
            uint32_t sh;  // the chunk, shifted so that it starts at bit 2
            if (s == 0) sh = lo << 2;
            else if (s + wd <= 32) sh = lo >> (s - 2);
            else if (s >= 34) sh = hi >> (s - 34);
            else sh = __funnelshift_r(lo, hi, s - 2);
            // table offset as a constant displacement of the load
            const uint32_t addr = ((sh & mask4) | tab_base) + (uint32_t)((x * Gm::CPW + cc) * 256);
            uint32_t v;
            asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(addr));
            const int t = x * Gm::CPW + cc;
            if (t & 1) d[(t >> 1) & 3] += pend + v;
            else pend = v;
        }
    }
    if (Gm::NT & 1) d[0] += pend;
    return (d[0] + d[1]) + (d[2] + d[3]);
}

template <int N>
__global__ void __launch_bounds__(kOsdWarps * 32, 8) osd_kernel(const OsdArgs a, const CodeDev c) {
    constexpr int W = (N + 63) / 64;
    constexpr int EPL = N / 32;  // elements per lane: element j = lane + 32 e
    extern __shared__ __align__(16) unsigned char osd_smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // round the dynamic window up to 256 bytes (the launch adds the slack)
    const uint32_t win = (uint32_t)__cvta_generic_to_shared(osd_smem);
    const uint32_t win256 = (win + 255u) & ~255u;
    OsdWarpSmem<N> &sm = reinterpret_cast<OsdWarpSmem<N> *>(osd_smem + (win256 - win))[warp];
    const uint32_t tab_base = win256 + (uint32_t)(warp * sizeof(OsdWarpSmem<N>));
    const int k = c.k;
    const int L = a.L;
    // lane bit masks for the tables: entries 2 lane and 2 lane + 1 have bits 1..5 = lane
    uint32_t lm[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) lm[i] = 0u - (((uint32_t)lane >> i) & 1u);
    if (a.ws.pool.cap > 0 && blockIdx.x == 0 && threadIdx.x == 0 && a.mode == 0)
        atomicAdd(&c.stats->frames, (unsigned long long)a.B);  // pool: counted per submission
    for (int64_t f = (int64_t)blockIdx.x * kOsdWarps + warp; f < a.B; f += (int64_t)gridDim.x * kOsdWarps) {
        // ---- 1. hard decisions, reliabilities ----
        uint32_t key[EPL];
        uint32_t hdh[EPL];  // 32-bit halves of hd: half e holds elements 32e .. 32e+31
        int asum = 0;
#pragma unroll
        for (int e = 0; e < EPL; ++e) {
            const int j = lane + 32 * e;
            const int g = grid_q(a.y[f * N + j]);
            const uint32_t ag = (uint32_t)abs(g);
            asum += (int)ag;
            sm.a[j] = ag;
            key[e] = (ag << 8) | (uint32_t)(255 - j);
            hdh[e] = __ballot_sync(kAll, g < 0);
        }
        asum = __reduce_add_sync(kAll, asum);  // sum_j |g_j| < 2^30
        uint64_t hdw[W];
#pragma unroll
        for (int w = 0; w < W; ++w)
            hdw[w] = (uint64_t)hdh[(2 * w) % EPL] | ((2 * w + 1 < EPL) ? (uint64_t)hdh[(2 * w + 1) % EPL] << 32 : 0ull);
        __syncwarp();
        // ---- tables of |g| over 6-position chunks ----
        {
            using Gm = OsdGeom<N>;
#pragma unroll
            for (int x = 0; x < Gm::W; ++x)
#pragma unroll
                for (int cc = 0; cc < Gm::CPW; ++cc) {
                    const int p0 = 64 * x + 6 * cc;
                    const int wd = Gm::BITS - 6 * cc < 6 ? Gm::BITS - 6 * cc : 6;
                    uint32_t hi = 0;  // bits 1 .. wd-1 of the entry come from the lane number
#pragma unroll
                    for (int i = 1; i < wd; ++i) hi += sm.a[p0 + i] & lm[i - 1];
                    const uint32_t a0 = sm.a[p0];
                    *reinterpret_cast<uint2 *>(&sm.tab[x * Gm::CPW + cc][2 * lane]) = make_uint2(hi, hi + a0);
                }
        }
        // ---- 2. positions by decreasing reliability ----
        sort_desc<N>(key, lane);
#pragma unroll
        for (int e = 0; e < EPL; ++e) sm.perm[32 * e + lane] = (uint8_t)(255 - (key[e] & 255u));
        __syncwarp();
        // ---- 3. Gauss-Jordan with pivots in reliability order ----
        uint64_t row[W];
#pragma unroll
        for (int w = 0; w < W; ++w) row[w] = lane < k ? c.gen_rows[lane * W + w] : 0ull;
        bool used = lane >= k;
        int piv = 0, found = 0;
        for (int q = 0; q < N && found < k; ++q) {
            const int p = sm.perm[q];
            const bool bit = lane < k && bit_at<W>(row, p);
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
            if (lane == 0) sm.mrb[found] = (uint8_t)p;
            ++found;
        }
        if (lane < k) sm.lane_of[piv] = (uint8_t)lane;
        __syncwarp();
        // ---- 4. lane t takes row t of G_sys; c0; e0 = c0 xor hd ----
        uint64_t rowp[W];
        bool take = false;
        {
            const int src = lane < k ? sm.lane_of[lane] : 0;
#pragma unroll
            for (int w = 0; w < W; ++w) rowp[w] = __shfl_sync(kAll, row[w], src);
            if (lane < k) {
                const int p = sm.mrb[lane];
                take = bit_at<W>(hdw, p);
            } else {
#pragma unroll
                for (int w = 0; w < W; ++w) rowp[w] = 0ull;
            }
        }
        uint64_t e0[W];
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint64_t x = take ? rowp[w] : 0ull;
            const uint32_t lo = __reduce_xor_sync(kAll, (uint32_t)x), hi = __reduce_xor_sync(kAll, (uint32_t)(x >> 32));
            e0[w] = (((uint64_t)hi << 32) | lo) ^ hdw[w];
        }
        // ---- 5-7. candidates, their discrepancy, the running list (one entry per lane) ----
        unsigned long long lkey = ~0ull;  // list entry `lane` (D << 32 | number), ascending
        auto offer = [&](bool valid, unsigned long long key) {
            unsigned long long thr = __shfl_sync(kAll, lkey, L - 1);
            unsigned m = __ballot_sync(kAll, valid && key < thr);
            if (__popc(m) > kMergeMin) {
                // many entries at once: sort the step's keys, then keep the L smallest of
                // the two sorted runs (a bitonic merge); equal to inserting them one by one
                unsigned long long x = (m >> lane) & 1u ? key : ~0ull;
#pragma unroll
                for (int sz = 2; sz <= 32; sz <<= 1)
#pragma unroll
                    for (int d = sz >> 1; d > 0; d >>= 1) {
                        const unsigned long long o = __shfl_xor_sync(kAll, x, d);
                        x = (((lane & d) == 0) == ((lane & sz) == 0)) ? min(x, o) : max(x, o);
                    }
                unsigned long long z = min(lkey, __shfl_sync(kAll, x, 31 - lane));
#pragma unroll
                for (int d = 16; d > 0; d >>= 1) {
                    const unsigned long long o = __shfl_xor_sync(kAll, z, d);
                    z = (lane & d) == 0 ? min(z, o) : max(z, o);
                }
                lkey = lane < L ? z : ~0ull;
                return;
            }
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
        // e ^= rows of the set packed in st (5 bits per row, the size in bits 20..22)
        auto flip_rows = [&](uint64_t (&e)[W], uint32_t st) {
            const int w = (int)(st >> 20);
            const int wmax = (int)__reduce_max_sync(kAll, (unsigned)w);
            for (int t = 0; t < wmax; ++t) {
                const int src = (int)(st >> (5 * t)) & 31;
#pragma unroll
                for (int x = 0; x < W; ++x) {
                    const uint64_t r = __shfl_sync(kAll, rowp[x], src);
                    if (t < w) e[x] ^= r;
                }
            }
        };
        // two steps of 32 candidates at a time: two independent chains of lookups
        for (int base = 0; base < a.ncand; base += 64) {
            const int i0 = base + lane, i1 = base + 32 + lane;
            const bool v0 = i0 < a.ncand, v1 = i1 < a.ncand;
            const uint32_t s0 = v0 ? __ldg(c.osd_sets + i0) : 0u, s1 = v1 ? __ldg(c.osd_sets + i1) : 0u;
            uint64_t e[W], f2[W];
#pragma unroll
            for (int x = 0; x < W; ++x) e[x] = f2[x] = e0[x];
            flip_rows(e, s0);
            flip_rows(f2, s1);
            const uint32_t d0 = discrepancy<N>(e, tab_base), d1 = discrepancy<N>(f2, tab_base);
            offer(v0, ((unsigned long long)d0 << 32) | (unsigned)i0);
            if (__any_sync(kAll, v1)) offer(v1, ((unsigned long long)d1 << 32) | (unsigned)i1);
        }
        // entry `lane` of the list: its codeword
        const int count = __popc(__ballot_sync(kAll, lkey != ~0ull));
        const bool valid = lane < count;
        uint64_t cw[W];
#pragma unroll
        for (int x = 0; x < W; ++x) cw[x] = e0[x] ^ hdw[x];
        flip_rows(cw, valid ? __ldg(c.osd_sets + (uint32_t)lkey) : 0u);
        const uint32_t dval = (uint32_t)(lkey >> 32);
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
                if (a.done_out) a.done_out[f] = -(a.submit_id + 1);
            }
            __syncwarp();
            continue;
        }
        const bool pool = a.ws.pool.cap > 0;
        int slot = 0, base = 0;
        if (lane == 0) {
            slot = pool ? pool_take_slot(a.ws) : atomicAdd(&a.ws.counters[0], 1);
            base = atomicAdd(&a.ws.counters[1], count);
            // a pool slot keeps its own copy of y, so y is read at the slot itself
            a.ws.slot_frame[slot] = pool ? slot : (int)(a.f0 + f);
            a.ws.slot_l1[slot] = (float)asum * (1.0f / 524288.0f);
            if (pool) {
                a.ws.pool.live[slot] = count;
                unsigned long long *d = a.ws.pool.dst + 3 * (int64_t)slot;
                d[0] = (unsigned long long)(a.cw_out + f * W);
                d[1] = (unsigned long long)(a.flags_out + f);
                d[2] = a.done_out ? (unsigned long long)(a.done_out + f) : 0ull;
            }
        }
        slot = __shfl_sync(kAll, slot, 0);
        base = __shfl_sync(kAll, base, 0);
        if (pool)
            for (int j = lane; j < N; j += 32)
                a.ws.pool.slot_y[(int64_t)slot * N + j] =
                    (bit_at<W>(hdw, j) ? -(float)sm.a[j] : (float)sm.a[j]) * (1.0f / 524288.0f);
        if (a.write_yhl) {
            // y in the split form the tensor-core scoring consumes (see the SC-list kernel)
            uint32_t *dst = a.ws.slot_yhl + (int64_t)slot * N;
            for (int w2 = lane; w2 < N / 2; w2 += 32) {
                uint32_t h2 = 0, l2 = 0;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int j = 2 * w2 + e;
                    const float v = (bit_at<W>(hdw, j) ? -(float)sm.a[j] : (float)sm.a[j]) * (1.0f / 524288.0f);
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
    constexpr int smem = kOsdWarps * (int)sizeof(OsdWarpSmem<N>) + 256;  // + slack for the 256-byte alignment
    static_assert(sizeof(OsdWarpSmem<N>) % 256 == 0, "per-warp tables stay 256-byte aligned");
    cudaError_t e = cudaFuncSetAttribute(osd_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = std::min<int64_t>((a.B + kOsdWarps - 1) / kOsdWarps, (int64_t)c.num_sms * 16);
    if (blocks <= 0) return cudaSuccess;
    osd_kernel<N><<<(unsigned)blocks, kOsdWarps * 32, smem, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_osd(const CodeDev &c, const OsdArgs &a, cudaStream_t s) {
    if (c.k > 32 || !c.osd_sets || a.L < 1 || a.L > 32 || a.order < 0 || a.order > 4 ||
        a.ncand != osd_candidates(c.k, a.order))
        return cudaErrorInvalidValue;
    if (c.n == 32) return launch_n<32>(c, a, s);
    if (c.n == 64) return launch_n<64>(c, a, s);
    if (c.n == 128) return launch_n<128>(c, a, s);
    return cudaErrorNotSupported;
}

}  // namespace mpwsd
