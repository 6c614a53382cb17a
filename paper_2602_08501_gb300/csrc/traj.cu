// Stage-2 trajectory kernels (Algorithm 1 after the scoring step):
//   hop_kernel     near-tie re-rank in FP64 of the candidates the scoring kernel
//                  kept, strict-improvement test, hop or deactivate, and
//                  compaction of the rows still active (the only FP64 step);
//   rescan_kernel  exact FP64 scan of every pattern for the rare rows whose
//                  kept candidates could not prove the minimum (near-tie overflow);
//   final_kernel   per failing frame, the trajectory of smallest ED (ties keep
//                  the lowest anchor index), its CRC status and flags.
#include "common.cuh"

namespace mpwsd {
namespace {

constexpr int kHopThreads = 256;

// Re-rank and decision from a top-K written by a scoring kernel (used when the
// scoring kernel did not finish the rows itself).
__global__ void __launch_bounds__(kHopThreads) hop_kernel(const Workspace ws, const CodeDev c, int iter, int L,
                                                          const float *y) {
    const int nrows = ws.counters[1 + iter];
    const int *act_in = ws.act[iter & 1];
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned long long my_cand = 0, my_hops = 0;
    // iterate in whole warps so the aggregated appends see converged lanes
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nrows; base += stride) {
        const int r = base + lane;
        int outcome = kRowNone, t = 0;
        if (r < nrows) {
            t = act_in[r];
            float v[kTopK];
            int ix[kTopK];
#pragma unroll
            for (int q = 0; q < kTopK; ++q) {
                v[q] = ws.topk_val[(int64_t)r * kTopK + q];
                ix[q] = ws.topk_idx[(int64_t)r * kTopK + q];
            }
            outcome = resolve_row(ws, c, t, L, y, v, ix, my_cand);
            my_hops += outcome == kRowHop;
        }
        route_row(ws, iter, outcome, t);
    }
    const unsigned long long wc = __reduce_add_sync(0xffffffffu, (unsigned)my_cand);
    const unsigned long long wh = __reduce_add_sync(0xffffffffu, (unsigned)my_hops);
    if (lane == 0) {
        if (wc) atomicAdd(&c.stats->rerank_candidates, wc);
        if (wh) atomicAdd(&c.stats->hops, wh);
    }
}

// One CTA per overflowing row: exact FP64 score of every pattern, argmin with
// the lowest index on ties, then the same decision as the hop kernel.
__global__ void __launch_bounds__(kHopThreads) rescan_kernel(const Workspace ws, const CodeDev c, int iter, int L,
                                                             const float *y) {
    __shared__ double s_best[kHopThreads / 32];
    __shared__ int s_idx[kHopThreads / 32];
    const int nres = ws.counters[32 + iter];
    int *act_out = ws.act[(iter + 1) & 1];
    int *n_out = ws.counters + 1 + iter + 1;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = blockIdx.x; i < nres; i += gridDim.x) {
        const int t = ws.rescan_rows[i];
        const float *yr = y + (int64_t)ws.slot_frame[t / L] * c.n;
        const uint64_t *cw = ws.traj_cw + (int64_t)t * c.W;
        double best = CUDART_INF;
        int bp = -1;
        for (int p = threadIdx.x; p < (int)c.P; p += blockDim.x) {
            const double s = exact_score(yr, cw, c.W, c.pat_supp + (int64_t)p * c.wq_max, c.wq_max, c.n);
            if (s < best) {
                best = s;
                bp = p;
            }
        }
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
            const double ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int op = __shfl_xor_sync(0xffffffffu, bp, o);
            if (op >= 0 && (ob < best || (ob == best && (bp < 0 || op < bp)))) {
                best = ob;
                bp = op;
            }
        }
        if (lane == 0) {
            s_best[wid] = best;
            s_idx[wid] = bp;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                const int op = s_idx[w];
                if (op >= 0 && (s_best[w] < best || (s_best[w] == best && (bp < 0 || op < bp)))) {
                    best = s_best[w];
                    bp = op;
                }
            }
            ws.traj_state[t] |= kTrajRescan;
            atomicAdd(&c.stats->rescans, 1ull);
            if (apply_decision(ws, c, t, bp, best)) {
                act_out[atomicAdd(n_out, 1)] = t;
                atomicAdd(&c.stats->hops, 1ull);
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kHopThreads) final_kernel(const Workspace ws, const CodeDev c, int L, int T,
                                                            int64_t B, uint64_t *cw_out, uint16_t *flags_out) {
    const int F = ws.counters[0];
    const int W = c.W;
    for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < F; s += gridDim.x * blockDim.x) {
        double best = CUDART_INF;
        int bk = 0;
        unsigned maxh = 0, rescan = 0;
        for (int l = 0; l < L; ++l) {
            const int64_t t = (int64_t)s * L + l;
            const uint32_t st = ws.traj_state[t];
            if (!(st & kTrajValid)) continue;
            const double D = ws.traj_D[t];
            if (D < best) {
                best = D;
                bk = l;
            }
            maxh = max(maxh, st & kTrajHopsMask);
            rescan |= st & kTrajRescan;
        }
        const uint64_t *cw = ws.traj_cw + ((int64_t)s * L + bk) * W;
        const int64_t frame = ws.slot_frame[s];
        unsigned syn = 0;
        for (int b = 0; b < c.crc_len; ++b) {
            int p = 0;
            for (int w = 0; w < W; ++w) p += __popcll(cw[w] & c.crc_masks[b * W + w]);
            syn |= (unsigned)(p & 1);
        }
        const unsigned iters = min((unsigned)T, maxh + 1u);
        uint16_t fl = (uint16_t)(MPWSD_FLAG_STAGE2 | (iters << MPWSD_FLAG_ITERS_SHIFT));
        if (c.crc_len > 0 && syn == 0) fl |= MPWSD_FLAG_CRC_OK;
        if (rescan) fl |= MPWSD_FLAG_RESCAN;
        if (c.stats->error) fl |= MPWSD_FLAG_ERROR;
        for (int w = 0; w < W; ++w) cw_out[frame * W + w] = cw[w];
        flags_out[frame] = fl;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        unsigned long long ev = 0;
        for (int i = 0; i < T; ++i) ev += (unsigned long long)ws.counters[1 + i];
        atomicAdd(&c.stats->frames, (unsigned long long)B);
        atomicAdd(&c.stats->stage2_frames, (unsigned long long)F);
        atomicAdd(&c.stats->trajectories, (unsigned long long)ws.counters[1]);
        atomicAdd(&c.stats->pattern_evals, ev * (unsigned long long)c.P);
    }
}

}  // namespace

cudaError_t launch_hop(const CodeDev &c, const Workspace &ws, int iter, int L, const float *y, cudaStream_t s) {
    hop_kernel<<<c.num_sms * 8, kHopThreads, 0, s>>>(ws, c, iter, L, y);
    return cudaGetLastError();
}

cudaError_t launch_rescan(const CodeDev &c, const Workspace &ws, int iter, int L, const float *y, cudaStream_t s) {
    rescan_kernel<<<c.num_sms * 2, kHopThreads, 0, s>>>(ws, c, iter, L, y);
    return cudaGetLastError();
}

cudaError_t launch_final(const CodeDev &c, const Workspace &ws, int L, int T, int64_t B, uint64_t *cw_out,
                         uint16_t *flags_out, cudaStream_t s) {
    final_kernel<<<c.num_sms * 2, kHopThreads, 0, s>>>(ws, c, L, T, B, cw_out, flags_out);
    return cudaGetLastError();
}

}  // namespace mpwsd
