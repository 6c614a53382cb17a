// Exact scoring of a flat pattern set (MPWSD_SCORE_FLATS): the intra-path
// structure of Sec. III-C used to cut the work of Eq. (5).
//
// The minimum-weight codewords of RM(r, m) are the cosets a + V of the linear
// subspaces V of dimension m - r of F_2^m (position j read as the m-bit vector
// of its binary digits). With z_x = y_x x_x(c) and the Walsh-Hadamard transform
// Z(w) = sum_x z_x (-1)^{w.x}, the indicator of a coset of V is an average of
// characters over V's orthogonal complement D = span(w1, w2) (dimension kd), so
//     2^kd S(a + V) = Z(0) + (-1)^{c1} Z(w1) + (-1)^{c2} Z(w2) + (-1)^{c1 ^ c2} Z(w1 ^ w2),
// with c_i = w_i . a (for kd = 1 only the first two terms). One n-point
// transform (n log2 n additions) and 2^kd kd additions per complement give the
// exact score of every pattern: for RM(2,6) 384 + 651 x 8 additions per row
// against 2604 x 16 for the pattern sums of Eq. (5) taken one by one. All sums
// are of grid integers round(y 2^19) and are exact in int32: a result is a sum
// of at most 32 terms below 2^23, and intermediate wrap-around cancels in
// two's-complement arithmetic.
//
// Mapping: one thread per row, FT threads per CTA. The row's z goes through
// the transform in registers; the coefficients are stored to shared memory
// with the thread index innermost (conflict-free), and the loop over the
// complements reads them at byte offsets that each CTA first derives from the
// code's table (w1, w2, w1 ^ w2 of each complement) into shared memory, one
// 32-bit offset per coefficient (16 bytes an entry, so the loop spends no
// instruction on unpacking; every lane reads the same entry, a broadcast). Z(0) is common to the 2^kd sums of a complement and the smallest of
// them is Z(0) + min(Z(w1) - |Z(w2) + Z(w1^w2)|, -Z(w1) - |Z(w2) - Z(w1^w2)|)
// (Z(0) - |Z(w1)| for kd = 1), so pass 1 takes that minimum relative to Z(0),
// keeping the smallest value, the first complement that reaches it and
// whether a later one ties it; the pattern index is then resolved
// exactly (lowest pattern index among equal scores, as Algorithm 1 breaks
// ties), with a second pass only when two complements tie. The output is the
// row's list with that single exact candidate, so the re-rank downstream scores
// one pattern.
#include "common.cuh"

#include <climits>

namespace mpwsd {
namespace {

// threads per CTA for n = 32, 64, 128 (256 for n = 64 measured the same as 128)
constexpr int kFlatsThreads32 = 128, kFlatsThreads64 = 128, kFlatsThreads128 = 128;

template <int KD>
__device__ __forceinline__ void coset_sums(int z0, int z1, int z2, int z3, int &s0, int &s1, int &s2, int &s3) {
    if constexpr (KD == 2) {
        const int t0 = z0 + z1, t1 = z0 - z1, t2 = z2 + z3, t3 = z2 - z3;
        s0 = t0 + t2;  // c = (0, 0)
        s1 = t1 + t3;  // c = (1, 0)
        s2 = t0 - t2;  // c = (0, 1)
        s3 = t1 - t3;  // c = (1, 1)
    } else {
        s0 = z0 + z1;  // c = 0
        s1 = z0 - z1;  // c = 1
        s2 = s3 = INT_MAX;
    }
}

template <int N, int KD, int kFT>
__global__ void __launch_bounds__(kFT) score_flats_kernel(const ScoreArgs a, const CodeDev c) {
    constexpr int W = (N + 63) / 64;
    extern __shared__ int zs[];  // Z(w) of thread t at zs[w * kFT + t]
    const int nrows = a.n_rows_dev ? *a.n_rows_dev : (int)a.n_rows;
    const int tid = threadIdx.x;
    const char *zb = reinterpret_cast<const char *>(zs + tid);
    const int ne = c.n_flat;
    uint4 *tab = reinterpret_cast<uint4 *>(zs + N * kFT);  // the complement table, after the coefficients
    constexpr unsigned stride = (unsigned)kFT * 4u;  // bytes between Z(w) and Z(w + 1) of one thread
    for (int e = tid; e < ne; e += kFT) {
        const uint32_t q = c.flat_w[e];
        tab[e] = make_uint4((q & 0xffu) * stride, ((q >> 8) & 0xffu) * stride, ((q >> 16) & 0xffu) * stride, 0u);
    }
    __syncthreads();
    for (int r = blockIdx.x * kFT + tid; r < nrows; r += gridDim.x * kFT) {
        const int t = a.rows ? a.rows[r] : r;
        const int fr = a.row_frame ? a.row_frame[r] : a.slot_frame[t / a.L];
        const float *yr = a.y + (int64_t)fr * N;
        uint64_t cb[W];
#pragma unroll
        for (int w = 0; w < W; ++w) cb[w] = a.cw[(int64_t)t * W + w];
        int z[N];
#pragma unroll
        for (int j = 0; j < N; j += 4) {
            const float4 v = *reinterpret_cast<const float4 *>(yr + j);
            z[j] = grid_q(v.x);
            z[j + 1] = grid_q(v.y);
            z[j + 2] = grid_q(v.z);
            z[j + 3] = grid_q(v.w);
        }
#pragma unroll
        for (int j = 0; j < N; ++j) z[j] = ((cb[j >> 6] >> (j & 63)) & 1ull) ? -z[j] : z[j];
        // Walsh-Hadamard transform in place: Z(w) = sum_x z_x (-1)^{w.x}
#pragma unroll
        for (int h = 1; h < N; h <<= 1)
#pragma unroll
            for (int i = 0; i < N; ++i)
                if (!(i & h)) {
                    const int u = z[i], v = z[i + h];
                    z[i] = u + v;
                    z[i + h] = u - v;
                }
#pragma unroll
        for (int w = 0; w < N; ++w) zs[w * kFT + tid] = z[w];
        const int z0 = z[0];
        // pass 1: the smallest coset sum (relative to Z(0)), the first complement
        // reaching it, and whether a later complement ties it
        int best = INT_MAX, be = 0;
        bool tie = false;
        for (int e = 0; e < ne; ++e) {
            const uint4 o = tab[e];
            const int z1 = *reinterpret_cast<const int *>(zb + o.x);
            int m;
            if constexpr (KD == 2) {
                const int z2 = *reinterpret_cast<const int *>(zb + o.y);
                const int z3 = *reinterpret_cast<const int *>(zb + o.z);
                m = min(z1 - abs(z2 + z3), -z1 - abs(z2 - z3));
            } else {
                m = -abs(z1);
            }
            tie = m < best ? false : (tie || m == best);
            be = m < best ? e : be;
            best = min(best, m);
        }
        best += z0;
        // the pattern: lowest index among the cosets whose sum is the minimum
        int bi = INT_MAX;
        const int e0 = tie ? 0 : be, e1 = tie ? ne : be + 1;
        for (int e = e0; e < e1; ++e) {
            const uint4 o = tab[e];
            const int z1 = *reinterpret_cast<const int *>(zb + o.x);
            const int z2 = KD == 2 ? *reinterpret_cast<const int *>(zb + o.y) : 0;
            const int z3 = KD == 2 ? *reinterpret_cast<const int *>(zb + o.z) : 0;
            int s[4];
            coset_sums<KD>(z0, z1, z2, z3, s[0], s[1], s[2], s[3]);
            const int4 ix = __ldg(reinterpret_cast<const int4 *>(c.flat_idx) + e);
            bi = s[0] == best ? min(bi, ix.x) : bi;
            bi = s[1] == best ? min(bi, ix.y) : bi;
            if (KD == 2) {
                bi = s[2] == best ? min(bi, ix.z) : bi;
                bi = s[3] == best ? min(bi, ix.w) : bi;
            }
        }
        // score of the pattern: best / 2^kd on the 2^-19 grid (the value only sets
        // the re-rank band; the re-rank recomputes it exactly)
        const float v = (float)best * (1.0f / (float)(1 << KD)) * (1.0f / 524288.0f);
        float4 *tv = reinterpret_cast<float4 *>(a.topk_val + (int64_t)r * kTopK);
        int4 *ti = reinterpret_cast<int4 *>(a.topk_idx + (int64_t)r * kTopK);
        *tv = make_float4(v, CUDART_INF_F, CUDART_INF_F, CUDART_INF_F);
        *ti = make_int4(bi, -1, -1, -1);
    }
}

template <int N, int KD, int kFT>
cudaError_t launch_nk(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    const int smem = N * kFT * 4 + c.n_flat * 16;
    cudaError_t e = cudaFuncSetAttribute(score_flats_kernel<N, KD, kFT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;  // CTAs that fit on an SM beside each other (registers, shared memory)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, score_flats_kernel<N, KD, kFT>, kFT, smem);
    if (e != cudaSuccess) return e;
    int64_t grid = (int64_t)c.num_sms * std::max(per_sm, 1);
    if (!a.n_rows_dev) grid = std::min<int64_t>(grid, (a.n_rows + kFT - 1) / kFT);
    if (grid <= 0) return cudaSuccess;
    score_flats_kernel<N, KD, kFT><<<(unsigned)grid, kFT, smem, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_score_flats(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    static_assert(kTopK == 4, "one float4 / int4 list per row");
    if (c.n_flat == 0) return cudaErrorInvalidValue;
    const bool k2 = c.flat_kd == 2;
    // threads per CTA: shared memory holds n coefficients per thread plus the table
    if (c.n == 32) return k2 ? launch_nk<32, 2, kFlatsThreads32>(c, a, s) : launch_nk<32, 1, kFlatsThreads32>(c, a, s);
    if (c.n == 64) return k2 ? launch_nk<64, 2, kFlatsThreads64>(c, a, s) : launch_nk<64, 1, kFlatsThreads64>(c, a, s);
    if (c.n == 128)
        return k2 ? launch_nk<128, 2, kFlatsThreads128>(c, a, s) : launch_nk<128, 1, kFlatsThreads128>(c, a, s);
    return cudaErrorNotSupported;
}

}  // namespace mpwsd
