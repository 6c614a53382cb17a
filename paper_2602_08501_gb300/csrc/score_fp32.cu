// Scoring step of stage 2 on FP32 CUDA cores (the plain form).
//
// For every active trajectory (row) with centre c and received y, and every
// pattern p of the sphere S_r(0) \ {0}, the score is
//     S(p) = sum_{j in supp p} z_j,   z_j = y_j x_j(c),  x = 1 - 2c,
// i.e. -G(p)/2 with G the correlation gain of Eq. (5); ED(c xor p) - ED(c)
// = 4 S(p) (translation identity, Eq. (3)). The kernel keeps, per row, the K
// smallest scores that lie within 2 eps of the row's smallest (eps the re-rank
// margin) with their pattern indices and never writes S itself; the re-rank
// and the hop of a decode follow in their own kernel.
//
// Mapping: one thread per row, 128 rows per CTA. The CTA stages its rows'
// z vectors in shared memory (row stride n+1 floats: conflict-free per-thread
// gathers) and streams the pattern supports (4 uint8 indices per word,
// padded with index n, which reads a zero) through shared memory; each
// thread accumulates w additions per pattern in ascending support order.
// FP32 error per score <= w 2^-24 ||y||_1, inside the re-rank margin.
#include <algorithm>

#include "common.cuh"

namespace mpwsd {
namespace {

constexpr int kRows = 128;
constexpr int kPatTile = 256;

template <int N>
__global__ void __launch_bounds__(kRows) score_fp32_kernel(const ScoreArgs a, const CodeDev c) {
    constexpr int W = (N + 63) / 64;
    constexpr int ZS = N + 1;
    extern __shared__ float smem[];
    float *zs = smem;                                     // [kRows][N+1]
    uint32_t *ps = reinterpret_cast<uint32_t *>(zs + kRows * ZS);  // [kPatTile][wq]
    const int wq = c.wq_max;
    const int P = (int)c.P;
    const int nrows = a.n_rows_dev ? *a.n_rows_dev : (int)a.n_rows;
    const int nblk = (nrows + kRows - 1) / kRows;
    const int tid = threadIdx.x;
    float *zr = zs + tid * ZS;
    for (int rb = blockIdx.x; rb < nblk; rb += gridDim.x) {
        const int r = rb * kRows + tid;
        const bool live = r < nrows;
        __syncthreads();
        float l1 = 0.0f;
        if (live) {
            const int t = a.rows ? a.rows[r] : r;
            const int frame = a.row_frame ? a.row_frame[r] : a.slot_frame[t / a.L];
            const float *yr = a.y + (int64_t)frame * N;
            const uint64_t *cw = a.cw + (int64_t)t * W;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint64_t bits = cw[w];
#pragma unroll 8
                for (int b = 0; b < 64 && w * 64 + b < N; ++b) {
                    const float v = grid_f(yr[w * 64 + b]);
                    l1 += fabsf(v);
                    zr[w * 64 + b] = ((bits >> b) & 1ull) ? -v : v;
                }
            }
        } else {
            for (int j = 0; j < N; ++j) zr[j] = 0.0f;
        }
        zr[N] = 0.0f;
        float tv[kTopK];
        int ti[kTopK];
#pragma unroll
        for (int q = 0; q < kTopK; ++q) {
            tv[q] = CUDART_INF_F;
            ti[q] = -1;
        }
        // admission threshold: below the K-th best kept and within 2 eps of the best kept
        const float eps2 = __fmul_ru(2.0f * kEpsScale, __fmul_ru(l1, 1.0f + 1.0f / 1024.0f));
        float thr = CUDART_INF_F;
        for (int p0 = 0; p0 < P; p0 += kPatTile) {
            const int np = min(kPatTile, P - p0);
            __syncthreads();
            const uint32_t *src = c.pat_supp + (int64_t)p0 * wq;
            for (int i = tid; i < np * wq; i += kRows) ps[i] = src[i];
            __syncthreads();
            if (!live) continue;
            for (int p = 0; p < np; ++p) {
                const uint32_t *sp = ps + p * wq;
                float s = 0.0f;
#pragma unroll 4
                for (int q = 0; q < wq; ++q) {
                    const uint32_t w4 = sp[q];
                    s += zr[w4 & 255u];
                    s += zr[(w4 >> 8) & 255u];
                    s += zr[(w4 >> 16) & 255u];
                    s += zr[w4 >> 24];
                }
                if (s < thr) {
                    topk_insert<kTopK>(tv, ti, s, p0 + p);
                    thr = fminf(tv[kTopK - 1], __fadd_ru(tv[0], eps2));
                }
            }
        }
        if (live) {
            // entries admitted before the minimum was seen may lie outside its band
            const float band = __fadd_ru(tv[0], eps2);
#pragma unroll
            for (int q = 0; q < kTopK; ++q) {
                const bool keep = q == 0 || tv[q] < band;
                a.topk_val[(int64_t)r * kTopK + q] = keep ? tv[q] : CUDART_INF_F;
                a.topk_idx[(int64_t)r * kTopK + q] = keep ? ti[q] : -1;
            }
        }
    }
}

template <int N>
cudaError_t launch_n(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    const size_t smem = (size_t)kRows * (N + 1) * 4 + (size_t)kPatTile * c.wq_max * 4;
    cudaError_t e = cudaFuncSetAttribute(score_fp32_kernel<N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)c.num_sms * 4;
    if (!a.n_rows_dev) grid = std::min<int64_t>(grid, (a.n_rows + kRows - 1) / kRows);
    if (grid <= 0) return cudaSuccess;
    score_fp32_kernel<N><<<(unsigned)grid, kRows, smem, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_score_fp32(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    if (c.n == 32) return launch_n<32>(c, a, s);
    if (c.n == 64) return launch_n<64>(c, a, s);
    return launch_n<128>(c, a, s);
}

}  // namespace mpwsd
