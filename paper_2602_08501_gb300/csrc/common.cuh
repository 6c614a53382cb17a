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

// Exact score S = sum_{j in supp p} y_j x_j(c) in FP64 (exact on the grid).
__device__ __forceinline__ double exact_score(const float *yr, const uint64_t *c, const uint64_t *p, int W) {
    double s = 0.0;
    for (int w = 0; w < W; ++w) {
        uint64_t m = p[w];
        const uint64_t cw = c[w];
        while (m) {
            const int b = __ffsll((long long)m) - 1;
            m &= m - 1;
            const double v = (double)grid_q(yr[w * 64 + b]) * (1.0 / 524288.0);
            s += ((cw >> b) & 1ull) ? -v : v;
        }
    }
    return s;
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

}  // namespace mpwsd
