// Tensor-core scoring (see score_tc_impl.cuh for the kernel): the launcher
// that picks the instantiated shape, the default shape of each code length,
// and the split preparation of direct scoring calls.
#include "score_tc_impl.cuh"

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

}  // namespace

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
