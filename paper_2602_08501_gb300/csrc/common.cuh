// Small device helpers shared by the stage-2 kernels of libmpwsd.
#pragma once

#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "internal.h"

namespace mpwsd {

// Integer image of a received sample on the 2^-19 grid (round to nearest
// even, clamped to 24-bit magnitudes). Every stage reads y through this, so
// the decoder is decode(quantize(y)) and exact for any input.
__device__ __forceinline__ int grid_q(float y) {
    int v = __float2int_rn(y * 524288.0f);
    return max(-kGridMax, min(kGridMax, v));
}

__device__ __forceinline__ float grid_f(float y) { return (float)grid_q(y) * (1.0f / 524288.0f); }

// Sorted (ascending) insertion into a K-entry list; s must be < v[K-1]. Equal
// values keep the earlier (lower-index) entry first.
template <int K>
__device__ __forceinline__ void topk_insert(float (&v)[K], int (&ix)[K], float s, int p) {
#pragma unroll
    for (int i = K - 1; i > 0; --i) {
        const bool before = s < v[i - 1];
        const bool here = !before && s < v[i];
        v[i] = before ? v[i - 1] : (here ? s : v[i]);
        ix[i] = before ? ix[i - 1] : (here ? p : ix[i]);
    }
    if (s < v[0]) {
        v[0] = s;
        ix[0] = p;
    }
}

// Exact score S = sum_{j in supp p} y_j x_j(c), returned in FP64. The terms
// are grid integers round(y 2^19) (|.| < 2^23) and at most 128 of them are
// added, so the sum is accumulated exactly in int32 and converted once; this is
// the same number an FP64 summation gives (exact on the grid) at a fraction of
// the FP64-pipe work. The support list of p (4 uint8 indices per word, padded
// with index n) is taken 16 indices (4 words) at a time, so their 16 loads of
// y are in flight together instead of one after another.
__device__ __forceinline__ int exact_round(const float *yr, uint64_t c0, uint64_t c1, const uint32_t (&wd)[4], int n) {
    float v[16];
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int j = (int)((wd[e >> 2] >> (8 * (e & 3))) & 255u);
        v[e] = j < n ? yr[j] : 0.0f;
    }
    int s = 0;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        const int j = (int)((wd[e >> 2] >> (8 * (e & 3))) & 255u);
        const uint64_t word = (j & 64) ? c1 : c0;
        const int g = grid_q(v[e]);  // 0 for padding
        s += ((word >> (j & 63)) & 1ull) ? -g : g;
    }
    return s;
}

// Support words q0 .. q0+3 of a pattern (index 255 past its wq words: no sample).
__device__ __forceinline__ void support_words(const uint32_t *supp, int wq, int q0, uint32_t (&wd)[4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) wd[u] = q0 + u < wq ? supp[q0 + u] : 0xffffffffu;
}

__device__ __forceinline__ double exact_score(const float *yr, uint64_t c0, uint64_t c1, const uint32_t *supp, int wq,
                                              int n) {
    int s = 0;
    for (int q0 = 0; q0 < wq; q0 += 4) {
        uint32_t wd[4];
        support_words(supp, wq, q0, wd);
        s += exact_round(yr, c0, c1, wd, n);
    }
    return (double)s * (1.0 / 524288.0);
}

// Warp-aggregated append: every lane of `mask` calls this; lanes with pred
// get consecutive slots of the list behind *counter.
__device__ __forceinline__ int append_slot(unsigned mask, int *counter, bool pred) {
    const unsigned ballot = __ballot_sync(mask, pred);
    if (!pred) return -1;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(ballot) - 1;
    int base = 0;
    if (lane == leader) base = atomicAdd(counter, __popc(ballot));
    base = __shfl_sync(ballot, base, leader);
    return base + __popc(ballot & ((1u << lane) - 1u));
}

// Decision of Algorithm 1 for trajectory t: hop to c xor p when the exact score
// S < 0 (a strict ED decrease of 4|S|), else deactivate. Returns true on a hop.
__device__ __forceinline__ bool apply_decision(const Workspace &ws, const CodeDev &c, int t, int p, double S) {
    const int W = c.W;
    if (p >= 0 && S < 0.0) {
        uint64_t *cw = ws.traj_cw + (int64_t)t * W;
        const uint64_t *pb = c.pat_bits + (int64_t)p * W;
        for (int w = 0; w < W; ++w) cw[w] ^= pb[w];
        ws.traj_D[t] += 2.0 * S;
        ws.traj_state[t] += 1u;  // hops counter in the low byte (<= MPWSD_MAX_T)
        return true;
    }
    return false;
}

enum RowOutcome { kRowNone = 0, kRowHop = 1, kRowStop = 2, kRowRescan = 3 };

// Pool mode: trajectory t (slot t / L) has ended; the last one of its slot
// puts the slot on the step's completed list.
__device__ __forceinline__ void pool_end_traj(const Workspace &ws, int t, int L) {
    const int slot = t / L;
    if (atomicSub(ws.pool.live + slot, 1) == 1) ws.pool.completed[atomicAdd(ws.pool.ctr + kPoolCompleted, 1)] = slot;
}

// Pool mode: a failing frame of a submission takes a free slot (the host keeps
// the frames in flight within the pool's capacity, so one is always free).
__device__ __forceinline__ int pool_take_slot(const Workspace &ws) {
    const int k = atomicAdd(ws.pool.ctr + kPoolPop, 1);
    return ws.pool.free_ring[(unsigned)k % (unsigned)ws.pool.cap];
}

// Active lists: iteration `iter` scores the rows of act[0] (count counters[1 +
// iter]); the rows that hop go to act[1] (count counters[kHoppedBase + iter]),
// and the duplicate retirement moves the distinct ones back into act[0] for
// the next iteration.
constexpr int kHoppedBase = 48;

// Append trajectory t to the hopped list or the rescan list, with
// warp-aggregated atomics; every lane of the warp calls this together.
__device__ __forceinline__ void route_row(const Workspace &ws, int iter, int outcome, int t) {
    const int po = append_slot(0xffffffffu, ws.counters + kHoppedBase + iter, outcome == kRowHop);
    if (po >= 0) ws.act[1][po] = t;
    const int pr = append_slot(0xffffffffu, ws.counters + 32 + iter, outcome == kRowRescan);
    if (pr >= 0) ws.rescan_rows[pr] = t;
}

}  // namespace mpwsd
