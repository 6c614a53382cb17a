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
// (the tie rule of Algorithm 1's argmin). A list whose fourth group is also
// in the band may have left candidates out and goes to the FP64 rescan.
//
// Mapping: a warp takes 32 rows, one per lane, and loads their lists, ids and
// centres with 32 rows' loads in flight; then eight rounds, in each of which
// its four 8-lane teams resolve one row each (small batches: fewer rows and
// rounds per warp, so that every warp has work).
//
// Two uses. Alone (mpwsd_score_topk), the row's list becomes that one pattern
// with its exact score; a full list keeps its four values, each group replaced
// by its pattern of smallest exact score (so every value stays within eps of
// its pattern's exact score). Inside a decode (HOP) the kernel takes Algorithm
// 1's decision for each row as well, in place of the hop kernel: hop to c xor p
// when the exact S(p) < 0, else stop; a full list goes to the rescan list. A
// row whose smallest approximate score exceeds eps cannot improve and stops
// without a resolution.
//
// A team's row sits in shared memory in sample order, with a zero at index N
// that the support padding (index N, and 255 past a pattern's words, clamped)
// reads; pattern sets without padding skip the clamp.
constexpr int kResolveThreads = 256;
constexpr int kResolveTeams = kResolveThreads / kGroupCols;

template <int N>
struct ResolveShape {
    static constexpr int PER = N / kGroupCols;          // samples per lane (8 or 16)
    static constexpr int STRIDE = N + 8;                 // team region, = 8 (mod 32) ints
    static_assert(STRIDE > N && STRIDE % 32 == 8, "team regions 8 banks apart");
};

// sum of z over 16 support indices (4 words of 4 uint8 indices)
template <int N, bool DENSE>
__device__ __forceinline__ int team_sum16(const int *zb, const uint4 w) {
    const uint32_t wd[4] = {w.x, w.y, w.z, w.w};
    int sum = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        int j = (int)__byte_perm(wd[e >> 2], 0u, 0x4440u + (uint32_t)(e & 3));
        if constexpr (!DENSE) j = min(j, N);
        sum += zb[j];
    }
    return sum;
}

__device__ __forceinline__ uint4 supp_quad(const uint32_t *supp, int wq, int q0) {
    if ((wq & 3) == 0) return __ldg(reinterpret_cast<const uint4 *>(supp + q0));
    uint32_t wd[4];
    support_words(supp, wq, q0, wd);
    return make_uint4(wd[0], wd[1], wd[2], wd[3]);
}

template <int N, bool DENSE, bool HOP>
__global__ void __launch_bounds__(kResolveThreads)
    resolve_groups_kernel(const ScoreArgs a, const CodeDev c, const Workspace ws, int iter) {
    static_assert(kGroupCols == 8, "one 8-lane team per row");
    using S = ResolveShape<N>;
    constexpr int PER = S::PER;
    constexpr int W = (N + 63) / 64;
    __shared__ __align__(16) int zs[kResolveTeams * S::STRIDE];
    const int nrows = a.n_rows_dev ? *a.n_rows_dev : (int)a.n_rows;
    const int lane = threadIdx.x & 31, sub = lane & 7, tq = lane >> 3, tm = threadIdx.x / kGroupCols;
    const unsigned team = 0xffu << (lane & 24);
    const int wq = c.wq_max, P = (int)c.P;
    int *zb = zs + tm * S::STRIDE;
    if (sub == 0) zb[N] = 0;
    unsigned long long my_cand = 0, my_hops = 0;
    // rows per warp pass: 32 when there are enough rows, fewer (a multiple of 4)
    // when a small batch would otherwise leave warps idle while others run eight
    // rounds one after another
    const int64_t nwarps = (int64_t)gridDim.x * (kResolveThreads / 32);
    const int64_t per = (((int64_t)nrows + nwarps - 1) / nwarps + 3) & ~(int64_t)3;
    const int rpw = per < 32 ? (int)per : 32;
    const int64_t wstep = nwarps * rpw;
    for (int64_t base = ((int64_t)blockIdx.x * (kResolveThreads / 32) + (threadIdx.x >> 5)) * rpw; base < nrows;
         base += wstep) {
        // one row per lane: its list, ids and centre (and, with the hop, its D and
        // state), 32 rows' loads in flight
        const int64_t r = lane < rpw ? base + lane : (int64_t)nrows;  // lanes past rpw hold no row
        int4 ix = make_int4(-1, -1, -1, -1);
        int fr = 0, ngf = 0, t = 0;
        uint64_t cw0 = 0, cw1 = 0;
        uint32_t st = 0;
        double D = 0.0;
        if (r < nrows) {
            const float4 v = reinterpret_cast<const float4 *>(a.topk_val)[r];
            ix = reinterpret_cast<const int4 *>(a.topk_idx)[r];
            t = a.rows ? a.rows[r] : (int)r;
            const int slot = a.row_frame ? a.row_frame[r] : t / a.L;
            fr = a.row_frame ? a.row_frame[r] : a.slot_frame[slot];
            cw0 = a.cw[(int64_t)t * W];
            if (W > 1) cw1 = a.cw[(int64_t)t * W + 1];
            if constexpr (HOP) {
                D = ws.traj_D[t];
                st = ws.traj_state[t];
            }
            // the re-rank's band (same arithmetic as the hop kernel)
            const float l1 = a.l1[slot];
            const float thr = __fadd_ru(v.x, __fmul_ru(2.0f, kEpsScale * l1));
            const bool full = ix.w >= 0 && v.w <= thr;
            const int ng = full ? 4 : (ix.x >= 0 && v.x <= thr) + (ix.y >= 0 && v.y <= thr) + (ix.z >= 0 && v.z <= thr);
            ngf = ng | (full ? 8 : 0);
            // with the hop: when even the smallest approximate score exceeds eps, no
            // pattern has a negative exact score (no strict improvement), the row stops
            // and there is nothing to resolve
            if (HOP && !full && v.x > kEpsScale * l1) ngf = 0;
        }
        int my_best = INT_MAX, my_bp = -1;
        // rpw / 4 rounds: team tq resolves the warp's row 4 k + tq
#pragma unroll 1
        for (int k = 0; k < rpw / 4; ++k) {
            const int src = 4 * k + tq;
            const int rngf = __shfl_sync(0xffffffffu, ngf, src);
            const int rfr = __shfl_sync(0xffffffffu, fr, src);
            uint64_t rcw = __shfl_sync(0xffffffffu, cw0, src);
            if constexpr (W > 1) {
                const uint64_t rc1 = __shfl_sync(0xffffffffu, cw1, src);
                if (sub * PER >= 64) rcw = rc1;
            }
            int4 rix;
            rix.x = __shfl_sync(0xffffffffu, ix.x, src);
            rix.y = __shfl_sync(0xffffffffu, ix.y, src);
            rix.z = __shfl_sync(0xffffffffu, ix.z, src);
            rix.w = __shfl_sync(0xffffffffu, ix.w, src);
            const int ng = rngf & 7;
            int best = INT_MAX, bp = INT_MAX, gp[4] = {-1, -1, -1, -1};
            // with the hop, a full list goes to the rescan as it is
            if (ng > 0 && !(HOP && (rngf & 8))) {
                // stage z: lane sub converts samples [PER sub, PER sub + PER)
                const float4 *yr = reinterpret_cast<const float4 *>(a.y + (int64_t)rfr * N + sub * PER);
                float f[PER];
#pragma unroll
                for (int u = 0; u < PER / 4; ++u) {
                    const float4 q = yr[u];
                    f[4 * u] = q.x;
                    f[4 * u + 1] = q.y;
                    f[4 * u + 2] = q.z;
                    f[4 * u + 3] = q.w;
                }
                __syncwarp(team);  // the previous row's sums are done
#pragma unroll
                for (int u = 0; u < PER / 4; ++u) {
                    int o[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int j = sub * PER + 4 * u + e;
                        const int g = grid_q(f[4 * u + e]);
                        o[e] = ((rcw >> (j & 63)) & 1ull) ? -g : g;
                    }
                    *reinterpret_cast<int4 *>(zb + sub * PER + 4 * u) = make_int4(o[0], o[1], o[2], o[3]);
                }
                __syncwarp(team);
                for (int q = 0; q < ng; ++q) {
                    const int g = q == 0 ? rix.x : q == 1 ? rix.y : q == 2 ? rix.z : rix.w;
                    const int p = g * kGroupCols + sub;
                    int sum = INT_MAX, pp = INT_MAX;
                    if (p < P) {
                        const uint32_t *supp = c.pat_supp + (int64_t)p * wq;
                        sum = 0;
                        for (int q0 = 0; q0 < wq; q0 += 4) sum += team_sum16<N, DENSE>(zb, supp_quad(supp, wq, q0));
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
                if (!HOP && sub == 0) {
                    const int64_t rr = base + src;
                    if (rngf & 8) {
                        reinterpret_cast<int4 *>(a.topk_idx)[rr] = make_int4(gp[0], gp[1], gp[2], gp[3]);
                    } else {
                        reinterpret_cast<float4 *>(a.topk_val)[rr] =
                            make_float4((float)best * (1.0f / 524288.0f), CUDART_INF_F, CUDART_INF_F, CUDART_INF_F);
                        reinterpret_cast<int4 *>(a.topk_idx)[rr] = make_int4(bp, -1, -1, -1);
                    }
                }
            }
            if constexpr (HOP) {
                // the team's result goes to the lane that holds the row
                const int from = 8 * ((lane - 4 * k) & 3);
                const int rb = __shfl_sync(0xffffffffu, best, from), rp = __shfl_sync(0xffffffffu, bp, from);
                if ((lane >> 2) == k) {
                    my_best = rb;
                    my_bp = rp == INT_MAX ? -1 : rp;
                }
            }
        }
        if constexpr (HOP) {
            // Algorithm 1's decision for the row (as the hop kernel takes it): hop to
            // c xor p when the exact score S(p) < 0 (a strict ED decrease of 4|S|), else stop
            int outcome = kRowNone;
            if (r < nrows) {
                if (ngf & 8) {
                    outcome = kRowRescan;
                } else {
                    outcome = kRowStop;
                    if (my_bp >= 0) ++my_cand;
                    if (my_bp >= 0 && my_best < 0) {
                        const uint64_t *pb = c.pat_bits + (int64_t)my_bp * W;
                        uint64_t *cwp = ws.traj_cw + (int64_t)t * W;
                        cwp[0] = cw0 ^ pb[0];
                        if (W > 1) cwp[1] = cw1 ^ pb[1];
                        ws.traj_D[t] = D + 2.0 * ((double)my_best * (1.0 / 524288.0));
                        ws.traj_state[t] = st + 1u;  // hops counter in the low byte (<= MPWSD_MAX_T)
                        outcome = kRowHop;
                        ++my_hops;
                    }
                    // pool: a trajectory ends when it stops or has made its T hops
                    if (ws.pool.cap > 0 && (outcome == kRowStop || (int)((st & kTrajHopsMask) + 1u) >= ws.pool.T)) {
                        pool_end_traj(ws, t, a.L);
                        outcome = kRowNone;
                    }
                }
            }
            route_row(ws, iter, outcome, t);
        }
    }
    if constexpr (HOP) {
        const unsigned long long wc = __reduce_add_sync(0xffffffffu, (unsigned)my_cand);
        const unsigned long long wh = __reduce_add_sync(0xffffffffu, (unsigned)my_hops);
        if (lane == 0) {
            if (wc) atomicAdd(&c.stats->rerank_candidates, wc);
            if (wh) atomicAdd(&c.stats->hops, wh);
        }
    }
}

template <int N, bool DENSE, bool HOP>
cudaError_t launch_resolve_n(const CodeDev &c, const ScoreArgs &a, const Workspace *ws, int iter, cudaStream_t s) {
    static int per_sm = 0;  // resident blocks per SM (registers, shared memory)
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, resolve_groups_kernel<N, DENSE, HOP>,
                                                                      kResolveThreads, 0);
        if (e != cudaSuccess) return e;
        per_sm = std::max(per_sm, 1);
    }
    int64_t grid = (int64_t)c.num_sms * per_sm;
    if (!a.n_rows_dev) grid = std::min<int64_t>(grid, (a.n_rows + kResolveThreads - 1) / kResolveThreads);
    if (grid <= 0) return cudaSuccess;
    resolve_groups_kernel<N, DENSE, HOP><<<(unsigned)grid, kResolveThreads, 0, s>>>(a, c, ws ? *ws : Workspace{}, iter);
    return cudaGetLastError();
}

template <int N>
cudaError_t launch_resolve_nd(const CodeDev &c, const ScoreArgs &a, const Workspace *ws, int iter, cudaStream_t s) {
    if (ws) return c.supp_dense ? launch_resolve_n<N, true, true>(c, a, ws, iter, s)
                                : launch_resolve_n<N, false, true>(c, a, ws, iter, s);
    return c.supp_dense ? launch_resolve_n<N, true, false>(c, a, ws, iter, s)
                        : launch_resolve_n<N, false, false>(c, a, ws, iter, s);
}

}  // namespace

cudaError_t launch_resolve_groups(const CodeDev &c, const ScoreArgs &a, const Workspace *ws, int iter,
                                  cudaStream_t s) {
    if (c.n == 64) return launch_resolve_nd<64>(c, a, ws, iter, s);
    if (c.n == 128) return launch_resolve_nd<128>(c, a, ws, iter, s);
    return cudaErrorNotSupported;
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
