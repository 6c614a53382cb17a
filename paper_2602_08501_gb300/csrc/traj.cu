// Stage-2 trajectory kernels (Algorithm 1 after the scoring step):
//   hop_kernel     near-tie re-rank in FP64 of the candidates the scoring kernel
//                  kept, strict-improvement test, hop or deactivate, and
//                  compaction of the rows still active (the only FP64 step);
//   rescan_kernel  exact FP64 scan of every pattern for the rare rows whose
//                  kept candidates could not prove the minimum (near-tie overflow);
//   dedup_kernel   retirement of the trajectories that hopped onto the centre
//                  of a lower-numbered trajectory of the same frame, and the
//                  next iteration's active list;
//   final_kernel   per failing frame, the trajectory of smallest ED (ties keep
//                  the lowest anchor index), its CRC status and flags.
#include "common.cuh"

namespace mpwsd {
namespace {

constexpr int kHopThreads = 256;

// Re-rank and decision for each active row, from the list its scoring step
// kept: the candidates are the leading entries within 2 eps of the first
// (eps = 2^-14 ||y||_1 of the frame); each is scored exactly, the smallest
// exact score (lowest index on ties) is taken, and the row hops if it is < 0
// (a strict ED decrease), else stops. A full list within the band means more
// candidates may exist: the row goes to the FP64 rescan instead.
// One thread per row; its reads are issued in dependency waves so a thread
// keeps several in flight: (1) trajectory id and list, (2) what they name --
// frame and ||y||_1, centre, D, state word, the first candidate's support --
// (3) the samples of that support.
__global__ void __launch_bounds__(kHopThreads) hop_kernel(const Workspace ws, const CodeDev c, int iter, int L,
                                                          const float *y) {
    const int nrows = ws.counters[1 + iter];
    const int *act_in = ws.act[0];
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int W = c.W, wq = c.wq_max, n = c.n;
    unsigned long long my_cand = 0, my_hops = 0;
    // iterate in whole warps so the aggregated appends see converged lanes
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nrows; base += stride) {
        const int r = base + lane;
        int outcome = kRowNone, t = 0;
        if (r < nrows) {
            // wave 1
            t = act_in[r];
            const float4 v = reinterpret_cast<const float4 *>(ws.topk_val)[r];
            const int4 ix = reinterpret_cast<const int4 *>(ws.topk_idx)[r];
            // wave 2
            const int slot = t / L;
            const int frame = ws.slot_frame[slot];
            const float l1 = ws.slot_l1[slot];
            uint64_t *cwp = ws.traj_cw + (int64_t)t * W;
            const uint64_t c0 = cwp[0], c1 = W > 1 ? cwp[1] : 0ull;
            const double D = ws.traj_D[t];
            const uint32_t st = ws.traj_state[t];
            uint32_t wd0[4];
            support_words(c.pat_supp + (int64_t)max(ix.x, 0) * wq, wq, 0, wd0);
            const float *yr = y + (int64_t)frame * n;
            const float thr = __fadd_ru(v.x, __fmul_ru(2.0f, kEpsScale * l1));
            if (ix.w >= 0 && v.w <= thr) {
                outcome = kRowRescan;
            } else {
                // the candidates are the leading entries (the list is ascending)
                const int ncand = (ix.x >= 0 && v.x <= thr) + (ix.y >= 0 && v.y <= thr) + (ix.z >= 0 && v.z <= thr);
                double best = CUDART_INF;
                int bp = -1;
#pragma unroll 1
                for (int q = 0; q < ncand; ++q) {
                    const int p = q == 0 ? ix.x : q == 1 ? ix.y : ix.z;
                    const uint32_t *supp = c.pat_supp + (int64_t)p * wq;
                    // wave 3 for the first candidate: its first support words are in hand
                    int sum = 0;
                    for (int q0 = 0; q0 < wq; q0 += 4) {
                        uint32_t wd[4];
                        if (q == 0 && q0 == 0) {
#pragma unroll
                            for (int u = 0; u < 4; ++u) wd[u] = wd0[u];
                        } else {
                            support_words(supp, wq, q0, wd);
                        }
                        sum += exact_round(yr, c0, c1, wd, n);
                    }
                    const double s = (double)sum * (1.0 / 524288.0);
                    if (s < best || (s == best && p < bp)) {
                        best = s;
                        bp = p;
                    }
                }
                my_cand += (unsigned long long)ncand;
                outcome = kRowStop;
                if (bp >= 0 && best < 0.0) {
                    // hop to c xor p (a strict ED decrease of 4 |S|)
                    const uint64_t *pb = c.pat_bits + (int64_t)bp * W;
                    cwp[0] = c0 ^ pb[0];
                    if (W > 1) cwp[1] = c1 ^ pb[1];
                    ws.traj_D[t] = D + 2.0 * best;
                    ws.traj_state[t] = st + 1u;  // hops counter in the low byte (<= MPWSD_MAX_T)
                    outcome = kRowHop;
                    ++my_hops;
                }
                // pool: a trajectory ends when it stops or has made its T hops
                if (ws.pool.cap > 0 && (outcome == kRowStop || (int)((st & kTrajHopsMask) + 1u) >= ws.pool.T)) {
                    pool_end_traj(ws, t, L);
                    outcome = kRowNone;
                }
            }
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
    int *act_out = ws.act[1];
    int *n_out = ws.counters + kHoppedBase + iter;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = blockIdx.x; i < nres; i += gridDim.x) {
        const int t = ws.rescan_rows[i];
        const float *yr = y + (int64_t)ws.slot_frame[t / L] * c.n;
        const uint64_t *cw = ws.traj_cw + (int64_t)t * c.W;
        double best = CUDART_INF;
        int bp = -1;
        for (int p = threadIdx.x; p < (int)c.P; p += blockDim.x) {
            const double s = exact_score(yr, cw[0], c.W > 1 ? cw[1] : 0ull, c.pat_supp + (int64_t)p * c.wq_max, c.wq_max, c.n);
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
            const bool hop = apply_decision(ws, c, t, bp, best);
            if (hop) atomicAdd(&c.stats->hops, 1ull);
            if (ws.pool.cap > 0 && (!hop || (int)(ws.traj_state[t] & kTrajHopsMask) >= ws.pool.T))
                pool_end_traj(ws, t, L);  // pool: stopped, or its T hops are done
            else if (hop)
                act_out[atomicAdd(n_out, 1)] = t;
        }
        __syncthreads();
    }
}

// A row that has just hopped is retired when a lower-numbered trajectory of
// its frame sits on the same centre and is itself live. Live means it hopped
// onto that centre in this same iteration, or it stopped there. A twin that
// hopped in the same iteration makes the same decisions from then on (a
// decision depends on the centre and y alone) with the same hop count. A twin
// that stopped proves that no improving pattern exists at that centre, so
// the row would stop next time anyway. A retired trajectory's centre is stale
// (its twin may have moved on), so it never serves as a twin. The retired row
// keeps its centre, D and hop count, and the result is unchanged. The frame's
// output is the smallest-ED trajectory (lowest anchor on ties), and a retired
// row never beats its twin: its D is at least the twin's final D, and its
// anchor is higher. The iteration count is the largest hop count plus one,
// which the twin reaches as well. Flags written by this pass may or may not be
// seen by other rows of the same pass; either way the outcome is the same,
// because a row retired now has a live lower-numbered twin on the same centre,
// and that twin serves every later row too.
__global__ void __launch_bounds__(kHopThreads) dedup_kernel(const Workspace ws, const CodeDev c, int iter, int L) {
    const int nrows = ws.counters[kHoppedBase + iter];
    int *n_out = ws.counters + 1 + iter + 1;
    const int stride = gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const int W = c.W;
    for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < nrows; base += stride) {
        const int r = base + lane;
        bool keep = false;
        int t = 0;
        if (r < nrows) {
            t = ws.act[1][r];
            const int64_t first = (int64_t)(t / L) * L;
            const uint64_t *cw = ws.traj_cw + (int64_t)t * W;
            const uint64_t c0 = cw[0], c1 = W > 1 ? cw[1] : 0ull;
            // the lower-numbered trajectories four at a time, their loads issued together
            bool dup = false;
            for (int64_t t2 = first; t2 < t; t2 += 4) {
                uint32_t st2[4];
                uint64_t a2[4], b2[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int64_t x = t2 + u;
                    const bool in = x < t;
                    st2[u] = in ? ws.traj_state[x] : 0u;
                    a2[u] = in ? ws.traj_cw[x * W] : 0ull;
                    b2[u] = (in && W > 1) ? ws.traj_cw[x * W + 1] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    dup |= (st2[u] & kTrajValid) && !(st2[u] & kTrajRetired) && a2[u] == c0 && b2[u] == c1;
            }
            keep = !dup;
            if (dup) {
                ws.traj_state[t] |= kTrajRetired;
                if (ws.pool.cap > 0) pool_end_traj(ws, t, L);
            }
        }
        const int po = append_slot(0xffffffffu, n_out, keep);
        if (po >= 0) ws.act[0][po] = t;
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

// Pool mode: the frames whose last trajectory ended in this step. Same choice
// as final_kernel (smallest ED, lowest anchor on ties); the result goes where
// the frame's submission asked, with the step number as its done entry, and
// the slot returns to the free ring.
__global__ void __launch_bounds__(kHopThreads) pool_final_kernel(const Workspace ws, const CodeDev c, int L) {
    const PoolDev &p = ws.pool;
    const int F = p.ctr[kPoolCompleted];
    const int step = p.ctr[kPoolSteps] + 1;
    const int W = c.W;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < F; i += gridDim.x * blockDim.x) {
        const int s = p.completed[i];
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
        unsigned syn = 0;
        for (int b = 0; b < c.crc_len; ++b) {
            int q = 0;
            for (int w = 0; w < W; ++w) q += __popcll(cw[w] & c.crc_masks[b * W + w]);
            syn |= (unsigned)(q & 1);
        }
        const unsigned iters = min((unsigned)p.T, maxh + 1u);
        uint16_t fl = (uint16_t)(MPWSD_FLAG_STAGE2 | (iters << MPWSD_FLAG_ITERS_SHIFT));
        if (c.crc_len > 0 && syn == 0) fl |= MPWSD_FLAG_CRC_OK;
        if (rescan) fl |= MPWSD_FLAG_RESCAN;
        if (c.stats->error) fl |= MPWSD_FLAG_ERROR;
        const unsigned long long *d = p.dst + 3 * (int64_t)s;
        uint64_t *cw_out = (uint64_t *)d[0];
        for (int w = 0; w < W; ++w) cw_out[w] = cw[w];
        *(uint16_t *)d[1] = fl;
        if (d[2]) *(int32_t *)d[2] = step;
        p.free_ring[(unsigned)atomicAdd(p.ctr + kPoolPush, 1) % (unsigned)p.cap] = s;
    }
}

// Pool mode, end of a step: the rows that go on (written by the twin
// retirement from 0) become the next step's rows, after which submissions
// append theirs; statistics of the step; the step count.
__global__ void pool_end_kernel(const Workspace ws, const CodeDev c) {
    const PoolDev &p = ws.pool;
    const int scored = ws.counters[1], done = p.ctr[kPoolCompleted];
    atomicAdd(&c.stats->pattern_evals, (unsigned long long)scored * (unsigned long long)c.P);
    atomicAdd(&c.stats->stage2_frames, (unsigned long long)done);
    ws.counters[1] = ws.counters[2];
    ws.counters[2] = 0;
    ws.counters[32] = 0;
    ws.counters[kHoppedBase] = 0;
    p.ctr[kPoolCompleted] = 0;
    p.ctr[kPoolFinished] += done;
    p.ctr[kPoolSteps] += 1;
}

}  // namespace

cudaError_t launch_pool_final(const CodeDev &c, const Workspace &ws, int L, cudaStream_t s) {
    pool_final_kernel<<<c.num_sms, kHopThreads, 0, s>>>(ws, c, L);
    return cudaGetLastError();
}

cudaError_t launch_pool_end(const CodeDev &c, const Workspace &ws, cudaStream_t s) {
    pool_end_kernel<<<1, 1, 0, s>>>(ws, c);
    return cudaGetLastError();
}

cudaError_t launch_hop(const CodeDev &c, const Workspace &ws, int iter, int L, const float *y, cudaStream_t s) {
    hop_kernel<<<c.num_sms * 8, kHopThreads, 0, s>>>(ws, c, iter, L, y);
    return cudaGetLastError();
}

cudaError_t launch_rescan(const CodeDev &c, const Workspace &ws, int iter, int L, const float *y, cudaStream_t s) {
    rescan_kernel<<<c.num_sms * 2, kHopThreads, 0, s>>>(ws, c, iter, L, y);
    return cudaGetLastError();
}

cudaError_t launch_dedup(const CodeDev &c, const Workspace &ws, int iter, int L, cudaStream_t s) {
    dedup_kernel<<<c.num_sms * 4, kHopThreads, 0, s>>>(ws, c, iter, L);
    return cudaGetLastError();
}

cudaError_t launch_final(const CodeDev &c, const Workspace &ws, int L, int T, int64_t B, uint64_t *cw_out,
                         uint16_t *flags_out, cudaStream_t s) {
    final_kernel<<<c.num_sms * 2, kHopThreads, 0, s>>>(ws, c, L, T, B, cw_out, flags_out);
    return cudaGetLastError();
}

}  // namespace mpwsd
