// Tensor-core scoring (see score_tc_impl.cuh for the kernel): the launcher
// that picks the instantiated shape, the default shape of each code length,
// and the split preparation of direct scoring calls.
#include "score_tc_impl.cuh"

#include <climits>

namespace mpwsd {
namespace {

// y -> bf16 hi / lo words and the exact ||y||_1 of each frame (one warp per frame)
__global__ void __launch_bounds__(256) split_prep_kernel(const float *y, int64_t B, int n, uint32_t *yhl, float *l1) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t f = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; f < B; f += warps) {
        const float *yr = y + f * n;
        uint32_t *dst = yhl + f * n;
        int acc = 0;
        for (int w = lane; w < n / 2; w += 32) {
            uint32_t h2 = 0, l2 = 0;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const int g = grid_q(yr[2 * w + e]);
                acc += abs(g);
                const float v = (float)g * (1.0f / 524288.0f);
                uint32_t hb, lb;
                split_bf16(v, hb, lb);
                h2 |= hb << (16 * e);
                l2 |= lb << (16 * e);
            }
            dst[w] = h2;
            dst[n / 2 + w] = l2;
        }
        acc = __reduce_add_sync(0xffffffffu, acc);  // exact: |sum| < 2^30
        if (lane == 0) l1[f] = (float)acc * (1.0f / 524288.0f);
    }
}

// Exact resolution of the tensor-core candidate groups (kGroupCols consecutive
// patterns each). Every pattern that can be the exact minimum of a row lies in
// a group whose smallest approximate score is within 2 eps of the row's first
// entry (eps = kEpsScale ||y||_1 bounds |approximate - exact|), so the groups
// in that band are scored exactly: one 8-lane team per row stages the row's z
// = y x(c) as grid integers in shared memory (coalesced loads, one conversion
// per sample), then lane i sums the support of pattern 8g + i of group g from
// there (integer sums on the 2^-19 grid, the numbers the re-rank computes),
// and the team keeps the smallest exact score, lowest pattern index on ties
// (the tie rule of Algorithm 1's argmin). The row's list becomes that one
// pattern with its exact score. A list whose fourth group is also in the band
// may have left candidates out (the re-rank rescans it): it keeps its four
// values, each group replaced by its pattern of smallest exact score, so every
// value stays within eps of its pattern's exact score.
constexpr int kResolveThreads = 256;
constexpr int kResolveTeams = kResolveThreads / kGroupCols;

template <int N>
__global__ void __launch_bounds__(kResolveThreads) resolve_groups_kernel(const ScoreArgs a, const CodeDev c) {
    static_assert(kGroupCols == 8, "one 8-lane team per row");
    constexpr int PER = N / kGroupCols;  // samples each lane stages (8 or 16)
    constexpr int W = (N + 63) / 64;
    __shared__ __align__(16) int zs[kResolveTeams][N + 4];  // z of the team's row; zs[.][N] = 0 (support padding)
    const int nrows = a.n_rows_dev ? *a.n_rows_dev : (int)a.n_rows;
    const int lane = threadIdx.x & 31, sub = lane & 7, tm = threadIdx.x / kGroupCols;
    const unsigned team = 0xffu << (lane & 24);
    const int wq = c.wq_max, P = (int)c.P;
    int *z = zs[tm];
    if (sub == 0) z[N] = 0;
    const int64_t step = (int64_t)gridDim.x * kResolveTeams;
    for (int64_t r = (int64_t)blockIdx.x * kResolveTeams + tm; r < nrows; r += step) {
        const float4 v = reinterpret_cast<const float4 *>(a.topk_val)[r];
        const int4 ix = reinterpret_cast<const int4 *>(a.topk_idx)[r];
        const int t = a.rows ? a.rows[r] : (int)r;
        const int slot = a.row_frame ? a.row_frame[r] : t / a.L;
        const int fr = a.row_frame ? a.row_frame[r] : a.slot_frame[slot];
        // the re-rank's band (same arithmetic as the hop kernel)
        const float thr = __fadd_ru(v.x, __fmul_ru(2.0f, kEpsScale * a.l1[slot]));
        const bool full = ix.w >= 0 && v.w <= thr;
        const int ng = full ? 4 : (ix.x >= 0 && v.x <= thr) + (ix.y >= 0 && v.y <= thr) + (ix.z >= 0 && v.z <= thr);
        if (ng == 0) continue;  // nothing kept (no patterns): the list stays as it is
        // stage z: lane sub converts samples [PER sub, PER sub + PER)
        {
            const uint64_t cwd = a.cw[(int64_t)t * W + (W > 1 ? (sub * PER) >> 6 : 0)];
            const float4 *yr = reinterpret_cast<const float4 *>(a.y + (int64_t)fr * N + sub * PER);
            __syncwarp(team);  // the previous row's sums are done
#pragma unroll
            for (int u = 0; u < PER / 4; ++u) {
                const float4 q = yr[u];
                const float f[4] = {q.x, q.y, q.z, q.w};
                int o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const int j = sub * PER + 4 * u + e;
                    const int g = grid_q(f[e]);
                    o[e] = ((cwd >> (j & 63)) & 1ull) ? -g : g;
                }
                *reinterpret_cast<int4 *>(z + sub * PER + 4 * u) = make_int4(o[0], o[1], o[2], o[3]);
            }
            __syncwarp(team);
        }
        int best = INT_MAX, bp = INT_MAX, gp[4] = {-1, -1, -1, -1};
        for (int q = 0; q < ng; ++q) {
            const int g = q == 0 ? ix.x : q == 1 ? ix.y : q == 2 ? ix.z : ix.w;
            const int p = g * kGroupCols + sub;
            int sum = INT_MAX, pp = INT_MAX;
            if (p < P) {
                const uint32_t *supp = c.pat_supp + (int64_t)p * wq;
                sum = 0;
                for (int q0 = 0; q0 < wq; q0 += 4) {
                    uint32_t wd[4];
                    support_words(supp, wq, q0, wd);
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        const int j = (int)((wd[e >> 2] >> (8 * (e & 3))) & 255u);
                        sum += z[min(j, N)];  // index N (padding) reads 0
                    }
                }
                pp = p;
            }
#pragma unroll
            for (int o = 4; o >= 1; o >>= 1) {
                const int s2 = __shfl_xor_sync(team, sum, o), p2 = __shfl_xor_sync(team, pp, o);
                if (s2 < sum || (s2 == sum && p2 < pp)) {
                    sum = s2;
                    pp = p2;
                }
            }
            gp[q] = pp;
            if (sum < best || (sum == best && pp < bp)) {
                best = sum;
                bp = pp;
            }
        }
        if (sub != 0) continue;
        if (full) {
            reinterpret_cast<int4 *>(a.topk_idx)[r] = make_int4(gp[0], gp[1], gp[2], gp[3]);
        } else {
            reinterpret_cast<float4 *>(a.topk_val)[r] =
                make_float4((float)best * (1.0f / 524288.0f), a.exact_tag ? __int_as_float(best) : CUDART_INF_F,
                            CUDART_INF_F, CUDART_INF_F);
            reinterpret_cast<int4 *>(a.topk_idx)[r] = make_int4(bp, a.exact_tag ? kExactTag : -1, -1, -1);
        }
    }
}

}  // namespace

cudaError_t launch_resolve_groups(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    int64_t grid = (int64_t)c.num_sms * 8;
    if (!a.n_rows_dev) grid = std::min<int64_t>(grid, (a.n_rows + kResolveTeams - 1) / kResolveTeams);
    if (grid <= 0) return cudaSuccess;
    if (c.n == 64)
        resolve_groups_kernel<64><<<(unsigned)grid, kResolveThreads, 0, s>>>(a, c);
    else if (c.n == 128)
        resolve_groups_kernel<128><<<(unsigned)grid, kResolveThreads, 0, s>>>(a, c);
    else
        return cudaErrorNotSupported;
    return cudaGetLastError();
}

cudaError_t launch_split_prep(const CodeDev &c, const float *y, int64_t B, uint32_t *yhl, float *l1, cudaStream_t s) {
    if (B <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((B + 7) / 8, (int64_t)c.num_sms * 16);
    split_prep_kernel<<<(unsigned)blocks, 256, 0, s>>>(y, B, c.n, yhl, l1);
    return cudaGetLastError();
}

bool score_tc_supported(const CodeDev &c) { return (c.n == 64 || c.n == 128) && c.pat_tiles != nullptr; }

bool tc_shape_valid(int n, int shape) {
    if (n == 64) return shape >= 0 && shape < kTcShapes;
    if (n == 128) return shape == 0 || shape == 1;
    return shape == 0;
}

cudaError_t launch_score_tc(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    if (c.tc_shape != 0) return launch_score_tc_alt(c, a, s);
    if (c.n == 64) return launch_shape<64, 256, 2, 2>(c, a, s);
    if (c.n == 128) return launch_shape<128, 128, 2, 2>(c, a, s);
    return cudaErrorNotSupported;
}

}  // namespace mpwsd
