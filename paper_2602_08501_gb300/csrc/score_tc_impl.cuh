// Scoring step of stage 2 on tcgen05 tensor cores (BF16 hi+lo split).
//
// Score of pattern p for a trajectory with centre c (Eq. (5), translation
// identity of Eq. (3)):   S(p) = sum_{j in supp p} z_j,  z_j = y_j x_j(c).
// With the 0/1 pattern matrix P (|P| x n) and Z the rows' z vectors this is
// S = Z P^T, a dense contraction. z is split as z = hi + lo with hi, lo
// bf16 (|z - hi - lo| <= 2^-16 |z|), so S ~= [Z_hi | Z_lo] [P | P]^T is two
// bf16 MMAs per K step into one FP32 accumulator; P is exact in bf16. The
// epilogue keeps each row's candidate groups for the exact argmin (at most
// four groups of 8 consecutive patterns, those whose smallest approximate
// score is within the re-rank margin of the row's minimum), so the score
// matrix never reaches HBM. Locating the column inside a group would cost the
// epilogue, which paces this kernel for n = 64, more than the MMAs; instead
// resolve_groups_kernel scores the patterns of the kept groups exactly (integer
// sums on the 2^-19 grid) and leaves the single exact argmin, and the hop
// follows in its own kernel, where a grid of short rows hides memory latency.
//
// Kernel shape (sm_103a): persistent, one CTA per SM, units of 256 rows (two
// 128-row blocks that share every pattern tile, halving the L2 traffic of the
// pattern stream per flop):
//   warp 0      bulk-copy producer: pattern tiles of P (256 patterns for
//               n = 64, 128 for n = 128), stored in HBM as the exact
//               shared-memory image of a K-major 128B-swizzled UMMA operand,
//               streamed through a two-stage smem ring;
//   warp 1      TMEM allocator and single-thread MMA issuer
//               (tcgen05.mma.cta_group::1.kind::f16, M = 128, K = 16);
//   A builders  warps 2-3 (and 12-13 in the four-builder shapes): gather frame and centre of
//               their rows, then y rows 16 at a time, form z, split to bf16
//               hi / lo, write the swizzled A tiles;
//   warps 4-11  epilogue: warp 4 + 4h + q reads TMEM lane quadrant q (one row
//               per thread) and column half h of every accumulator with
//               tcgen05.ld (x64 chunks for n = 64; for n = 128 x32 slices,
//               the next one's load in flight while one is scanned, and the
//               accumulator released once its last columns are in
//               registers); takes minima of 8-column groups with
//               three-input mins, and only groups that beat the row's
//               admission threshold enter its running top-K (as group
//               indices); at the end of a unit the two halves of each row's
//               list meet in shared memory.
// MMAs into one accumulator serialise (one chain of 128 x 128 x 16 MMAs runs
// at about 60 % of the tensor rate, 128 x 256 x 16 at the full rate), so the
// issue order is chosen per n. n = 64: per tile, row block 0 then row block 1,
// each one chain of 128 x 256 x 16 MMAs into its own 256-column accumulator;
// the epilogue of one row block overlaps the other's MMAs. n = 128: per K
// step one 128 x 128 x 16 MMA per row block (two chains), and two tile-sized
// accumulators (2 x 256 columns) let the epilogue of tile j overlap the MMAs
// of tile j+1. Every mbarrier wait is bounded in time; on expiry the kernel
// records an error word, drains its own copies, frees TMEM and exits.
#pragma once
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"

namespace mpwsd {
namespace {

static_assert(kTopK == 4, "the split merge loads one float4 / int4 per chunk list");
constexpr int BM = 128;                 // rows per MMA (TMEM lanes)
constexpr int RB = 2;                   // row blocks per unit, sharing every pattern tile
constexpr int UM = BM * RB;             // rows per unit
constexpr int kEpiWarps = 8;                 // warps 4-11
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr unsigned long long kErrTcTimeout = 0x7C01;
constexpr uint32_t kWaitHintNs = 100000;  // longest sleep of one try_wait (the bounded waits re-check)

// Shape of the kernel: code length N, pattern tile BN_ (the MMA N), A-builder
// warps BLD and stages BST of the pattern-tile ring (MPWSD_TUNE_TC_SHAPE picks
// one of the instantiated shapes at run time).
template <int N, int BN_, int BLD, int BST>
struct TcCfg {
    static constexpr int KC = N / 64;                    // 64-element (128 B) K chunks
    static constexpr int BN = BN_;                       // patterns per tile (MMA N)
    // SEQ: the row blocks take turns on the tensor core, one unbroken chain of
    // MMAs per (tile, row block) into that row block's own accumulator, so the
    // epilogue of one row block overlaps the other's MMAs (RB x BN = all 512
    // TMEM columns). Otherwise the row blocks' MMAs interleave per K step and
    // two tile-sized accumulators alternate.
    static constexpr bool SEQ = (RB * BN == 512);
    static_assert(SEQ || 2 * RB * BN <= 512, "accumulators exceed TMEM");
    static constexpr int A_BUFS = (N == 64) ? 2 : 1;
    static constexpr int B_STAGES = BST;
    // A builders: one or two per row block (warps 2-3, then 12-13), each
    // filling BM / (BUILDERS / RB) rows of its row block per unit
    static constexpr int BUILDERS = BLD;
    static constexpr int QN = BM / 32 / (BUILDERS / RB);   // 32-row slices per builder
    static constexpr int THREADS = (4 + kEpiWarps + BUILDERS - 2) * 32;
    static constexpr int A_PART_BYTES = BM * N * 2;      // one row block, hi or lo
    static constexpr int A_BUF_BYTES = RB * 2 * A_PART_BYTES;
    static constexpr int B_STAGE_BYTES = BN * N * 2;
    static constexpr int TILE_BYTES = A_BUFS * A_BUF_BYTES + B_STAGES * B_STAGE_BYTES;
    static constexpr int BAR_BYTES = 256;
    static_assert((2 * B_STAGES + 3 * A_BUFS + 7) * 8 + 12 <= BAR_BYTES, "mbarriers and flags fit their region");
    static constexpr int XCHG_BYTES = RB * BM * kTopK * 8;  // exchanged (value, index) lists
    static constexpr int L1_BYTES = A_BUFS * UM * 4;  // ||y||_1 of each row of the A buffers
    static constexpr int BEST_BYTES = RB * BM * 2 * 8;  // shared running minima of the row halves
    static constexpr int SMEM_BYTES = TILE_BYTES + 1024 + BAR_BYTES + XCHG_BYTES + L1_BYTES + BEST_BYTES;
    static constexpr int G = 8;                          // rows whose y loads are in flight together
};

// ---- PTX wrappers -------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t tx) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(tx) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// try_wait with a suspend-time hint: a waiting thread sleeps until the phase
// completes (or the hint runs out) instead of spinning, which leaves the issue
// slots of its SM sub-partition to the warps that have work
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kWaitHintNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Bounded wait for the phase of parity `parity`; false on abort or timeout.
// The first try is inline (usually the phase is complete, and a call would
// cost the epilogue register moves around it); the sleeping loop is a call.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, const volatile int *abort_flag,
                                            uint64_t limit_ns) {
    const uint64_t t0 = global_ns();
    for (uint32_t i = 1; i < (1u << 30); ++i) {
        if (mbar_try_sleep(bar, parity)) return true;
        if (*abort_flag) return false;
        if (global_ns() - t0 > limit_ns) return false;
    }
    return false;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int *abort_flag,
                                          uint64_t limit_ns) {
    return mbar_try(bar, parity) || mbar_wait_slow(bar, parity, abort_flag, limit_ns);
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// Shared-memory matrix descriptor of a K-major, 128-byte-swizzled operand:
// start address >> 4 (bits 0-13), leading offset (ignored for this layout),
// stride 1024 B between 8-row groups (bits 32-45), descriptor version 1
// (bits 46-47), swizzle mode 128B (bits 61-63).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) |
           ((uint64_t)1u << 46) | ((uint64_t)2u << 61);
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bits 17-22, M >> 4 at bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accum) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accum)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}


#define MPWSD_R8(i) "=r"(v[i + 0]), "=r"(v[i + 1]), "=r"(v[i + 2]), "=r"(v[i + 3]), "=r"(v[i + 4]), "=r"(v[i + 5]), \
                    "=r"(v[i + 6]), "=r"(v[i + 7])
// 64 consecutive FP32 columns of this thread's TMEM lane (load and wait)
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&v)[64]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
        "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
        "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
        : MPWSD_R8(0), MPWSD_R8(8), MPWSD_R8(16), MPWSD_R8(24), MPWSD_R8(32), MPWSD_R8(40), MPWSD_R8(48),
          MPWSD_R8(56)
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// issue a load of 32 consecutive FP32 columns of this thread's TMEM lane (no wait)
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : MPWSD_R8(0), MPWSD_R8(8), MPWSD_R8(16), MPWSD_R8(24)
        : "r"(taddr));
}
#undef MPWSD_R8
#define MPWSD_R8(i) "+r"(v[i + 0]), "+r"(v[i + 1]), "+r"(v[i + 2]), "+r"(v[i + 3]), "+r"(v[i + 4]), "+r"(v[i + 5]), \
                    "+r"(v[i + 6]), "+r"(v[i + 7])
// wait for this thread's outstanding TMEM loads; v (the last one's registers) is
// passed through so that nothing reads it before the wait
__device__ __forceinline__ void tmem_wait(uint32_t (&v)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : MPWSD_R8(0), MPWSD_R8(8), MPWSD_R8(16), MPWSD_R8(24)::"memory");
}
#undef MPWSD_R8

__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// minimum of the 8 values v[8g .. 8g+7]
template <int G8, int CW>
__device__ __forceinline__ float min8(const uint32_t (&v)[CW]) {
    return fmin3(fmin3(__uint_as_float(v[8 * G8]), __uint_as_float(v[8 * G8 + 1]), __uint_as_float(v[8 * G8 + 2])),
                 fmin3(__uint_as_float(v[8 * G8 + 3]), __uint_as_float(v[8 * G8 + 4]), __uint_as_float(v[8 * G8 + 5])),
                 fminf(__uint_as_float(v[8 * G8 + 6]), __uint_as_float(v[8 * G8 + 7])));
}

// Current admission threshold of a row: a value enters the running list only
// if it beats the K-th best kept so far and lies within 2 eps of the best kept
// so far (anything above that band can never be a candidate of the re-rank).
__device__ __forceinline__ float admit_thr(const float (&tv)[kTopK], float eps2) {
    return fminf(tv[kTopK - 1], __fadd_ru(tv[0], eps2));
}

// Admission of one CW-column chunk whose minimum m beats the row's threshold.
// Once m is in the list nothing at or above t1 = min(thr, m + 2 eps) can
// enter, so the chunk matters only through its 8-column groups whose minimum
// is below t1; each enters as (group minimum, group index). Usually that is
// the one group holding m, inserted without a search; two or more (a near tie
// across groups of the chunk) are inserted one by one in group order.
template <int CW>
__device__ __forceinline__ void admit_chunk(const float (&gm)[CW / 8], float m, float (&tv)[kTopK], int (&ti)[kTopK],
                                            float &thr, float eps2, int gbase) {
    static_assert(CW == 32 || CW == 64, "chunks of 32 or 64 columns");
    const float t1 = fminf(thr, __fadd_ru(m, eps2));
    unsigned below = 0u;
#pragma unroll
    for (int g = 0; g < CW / 8; ++g) below |= gm[g] < t1 ? (1u << g) : 0u;
    if (__popc(below) == 1) {
        topk_insert<kTopK>(tv, ti, m, gbase + __ffs(below) - 1);
        thr = admit_thr(tv, eps2);
    } else {
#pragma unroll
        for (int g = 0; g < CW / 8; ++g) {
            if (gm[g] < thr) {
                topk_insert<kTopK>(tv, ti, gm[g], gbase + g);
                thr = admit_thr(tv, eps2);
            }
        }
    }
}

template <int G8, int CW>
__device__ __forceinline__ void group_mins(const uint32_t (&v)[CW], float (&gm)[CW / 8]) {
    if constexpr (G8 < CW / 8) {
        gm[G8] = min8<G8, CW>(v);
        group_mins<G8 + 1, CW>(v, gm);
    }
}

// One CW-column chunk of a row's scores into its running list: group minima,
// the chunk minimum, and an admission when it beats the row's threshold.
// Columns at or past P (the last tile's padding) count as +inf. cbase is the
// chunk's first column, a multiple of 8 (list entries are group indices).
template <int CW>
__device__ __forceinline__ void epi_chunk(uint32_t (&v)[CW], int cbase, int P, bool full, float (&tv)[kTopK],
                                          int (&ti)[kTopK], float &thr, float eps2) {
    if (!full) {
#pragma unroll
        for (int e = 0; e < CW; ++e)
            if (cbase + e >= P) v[e] = __float_as_uint(CUDART_INF_F);
    }
    float gm[CW / 8];
    group_mins<0, CW>(v, gm);
    float m;
    if constexpr (CW == 64)
        m = fmin3(fmin3(gm[0], gm[1], gm[2]), fmin3(gm[3], gm[4], gm[5]), fminf(gm[6], gm[7]));
    else
        m = fminf(fmin3(gm[0], gm[1], gm[2]), gm[3]);
    if (m < thr) admit_chunk<CW>(gm, m, tv, ti, thr, eps2, cbase / kGroupCols);
}

__device__ __forceinline__ uint32_t bf16_bits(__nv_bfloat16 h) { return (uint32_t)__bfloat16_as_ushort(h); }

// hi / lo bf16 parts of z (both round to nearest even; z - hi is exact in FP32)
__device__ __forceinline__ void split_bf16(float z, uint32_t &hi, uint32_t &lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(z);
    const __nv_bfloat16 l = __float2bfloat16_rn(z - __bfloat162float(h));
    hi = bf16_bits(h);
    lo = bf16_bits(l);
}

struct TcShared {
    uint64_t *b_full, *b_empty, *a_full, *a_empty, *acc_full, *acc_empty;
    uint32_t *tmem_slot;
    int *abort_flag;
    int *last_flag;
    uint64_t *epi_pub, *epi_last;  // split: chunk lists published / last-chunk flag ready
    uint64_t *xchg;                // epilogue halves: lists written / read (two phases per unit)
    uint64_t *l1_free;             // per A buffer: every epilogue thread has read its rows' norms
    float *xv;                     // exchanged lists, RB x BM x kTopK
    int *xi;
    float *l1;                     // ||y||_1 of the rows of each A buffer, A_BUFS x UM
    unsigned long long *best;      // (work item, best value so far) of each row half, RB x BM x 2
};

__device__ __forceinline__ void record_abort(const TcShared &sh, const CodeDev &c) {
    *(volatile int *)sh.abort_flag = 1;
    atomicExch(&c.stats->error, kErrTcTimeout);
}

template <int N, int BN_, int BLD, int BST>
__global__ void __launch_bounds__(TcCfg<N, BN_, BLD, BST>::THREADS, 1) score_tc_kernel(const ScoreArgs a,
                                                                                        const CodeDev c) {
    using C = TcCfg<N, BN_, BLD, BST>;
    constexpr int W = (N + 63) / 64;
    constexpr int EPL = N / 32;  // elements of a row per lane in the A builder
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t *Abase = smem;
    uint8_t *Bbase = smem + C::A_BUFS * C::A_BUF_BYTES;
    uint64_t *bars = (uint64_t *)(Bbase + C::B_STAGES * C::B_STAGE_BYTES);
    TcShared sh;
    sh.b_full = bars;
    sh.b_empty = bars + C::B_STAGES;
    sh.a_full = bars + 2 * C::B_STAGES;
    sh.a_empty = sh.a_full + C::A_BUFS;
    sh.acc_full = sh.a_empty + C::A_BUFS;
    sh.acc_empty = sh.acc_full + 2;
    sh.epi_pub = sh.acc_empty + 2;
    sh.epi_last = sh.epi_pub + 1;
    sh.xchg = sh.epi_last + 1;
    sh.l1_free = sh.xchg + 1;
    sh.tmem_slot = (uint32_t *)(sh.l1_free + C::A_BUFS);
    sh.abort_flag = (int *)(sh.tmem_slot + 1);
    sh.last_flag = sh.abort_flag + 1;
    sh.xv = (float *)((uint8_t *)bars + C::BAR_BYTES);
    sh.xi = (int *)(sh.xv + RB * BM * kTopK);
    sh.l1 = (float *)(sh.xi + RB * BM * kTopK);
    sh.best = (unsigned long long *)(sh.l1 + C::A_BUFS * UM);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nrows = a.n_rows_dev ? *a.n_rows_dev : (int)a.n_rows;
    const int nunits = (nrows + UM - 1) / UM;
    const int P = (int)c.P;
    const int nt = (P + C::BN - 1) / C::BN;
    // Work items: (unit, chunk of pattern tiles). When there are fewer units than
    // the split target, each unit's tiles are split into nch chunks scanned by
    // different CTAs; the last CTA to finish a unit merges the chunks' lists.
    int nch = 1;
    if (a.split_val && nunits < a.split_items) nch = min(nt, (a.split_items + nunits - 1) / nunits);
    const int nitems = nunits * nch;
    const int my_units =
        nitems > (int)blockIdx.x ? (nitems - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    if (my_units == 0) return;

    for (int e = threadIdx.x; e < RB * BM * 2; e += blockDim.x) sh.best[e] = ~0ull;  // no work item
    if (threadIdx.x == 0) {
        for (int s = 0; s < C::B_STAGES; ++s) {
            mbar_init(smem_u32(&sh.b_full[s]), 1);
            mbar_init(smem_u32(&sh.b_empty[s]), 1);
        }
        for (int s = 0; s < C::A_BUFS; ++s) {
            mbar_init(smem_u32(&sh.a_full[s]), 32 * C::BUILDERS);
            mbar_init(smem_u32(&sh.a_empty[s]), 1);
            mbar_init(smem_u32(&sh.l1_free[s]), kEpiThreads);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(smem_u32(&sh.acc_full[s]), 1);
            mbar_init(smem_u32(&sh.acc_empty[s]), kEpiThreads);
        }
        mbar_init(smem_u32(sh.epi_pub), kEpiThreads);
        mbar_init(smem_u32(sh.epi_last), 1);
        mbar_init(smem_u32(sh.xchg), kEpiThreads);
        *sh.abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(sh.tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *sh.tmem_slot;
    const volatile int *abort_flag = sh.abort_flag;

    if (warp == 0) {
        // ---- producer: pattern tiles into the B ring ----
        if (lane == 0 && !c.test_stall) {
            int g = 0;
            bool ok = true;
            for (int i = 0; i < my_units && ok; ++i) {
                const int item = (int)blockIdx.x + i * (int)gridDim.x, ch = item % nch;
                for (int j = ch * nt / nch; j < (ch + 1) * nt / nch; ++j, ++g) {
                    const int s = g % C::B_STAGES;
                    const uint32_t ph = (uint32_t)(g / C::B_STAGES) & 1u;
                    if (!mbar_wait(smem_u32(&sh.b_empty[s]), ph ^ 1u, abort_flag, c.wait_limit_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t full = smem_u32(&sh.b_full[s]);
                    mbar_arrive_tx(full, C::B_STAGE_BYTES);
                    const uint8_t *src = (const uint8_t *)c.pat_tiles + (size_t)j * C::B_STAGE_BYTES;
                    const uint32_t dst = smem_u32(Bbase + s * C::B_STAGE_BYTES);
                    for (int part = 0; part < C::B_STAGE_BYTES; part += 16384)
                        bulk_g2s(dst + part, src + part, 16384, full);
                }
            }
            if (!ok) {
                record_abort(sh, c);
                // drain: wait (bounded) for the copies this thread issued
                const int zero = 0;
                for (int d = (g > C::B_STAGES ? g - C::B_STAGES : 0); d < g; ++d)
                    mbar_wait(smem_u32(&sh.b_full[d % C::B_STAGES]), (uint32_t)(d / C::B_STAGES) & 1u,
                              (const volatile int *)&zero, 10000000ull);
            }
        }
    } else if (warp == 1) {
        // ---- MMA issuer (issue order per n: see the file comment) ----
        if (lane == 0) {
            constexpr uint32_t idesc_full = idesc_bf16(BM, C::BN);
            // the last tile holds P - (nt - 1) BN patterns: its MMAs are only as wide
            // as those, rounded up to the MMA's N granularity of 16 (M = 128)
            const uint32_t idesc_last = idesc_bf16(BM, min(C::BN, ((P - (nt - 1) * C::BN) + 15) & ~15));
            int gb = 0, gacc = 0;
            bool ok = true;
            uint32_t last_bar = 0, last_par = 0;
            for (int i = 0; i < my_units && ok; ++i) {
                const int ab = i % C::A_BUFS;
                if (!mbar_wait(smem_u32(&sh.a_full[ab]), (uint32_t)(i / C::A_BUFS) & 1u, abort_flag, c.wait_limit_ns)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t abuf = smem_u32(Abase + ab * C::A_BUF_BYTES);
                const int item = (int)blockIdx.x + i * (int)gridDim.x, ch = item % nch;
                for (int j = ch * nt / nch; j < (ch + 1) * nt / nch; ++j, ++gb, ++gacc) {
                    const int s = gb % C::B_STAGES;
                    if (!mbar_wait(smem_u32(&sh.b_full[s]), (uint32_t)(gb / C::B_STAGES) & 1u, abort_flag,
                                   c.wait_limit_ns)) {
                        ok = false;
                        break;
                    }
                    const uint32_t bsm = smem_u32(Bbase + s * C::B_STAGE_BYTES);
                    const uint32_t idesc = j == nt - 1 ? idesc_last : idesc_full;
                    if constexpr (C::SEQ) {
                        for (int rb = 0; rb < RB; ++rb) {
                            if (!mbar_wait(smem_u32(&sh.acc_empty[rb]), ((uint32_t)gacc & 1u) ^ 1u, abort_flag,
                                           c.wait_limit_ns)) {
                                ok = false;
                                break;
                            }
                            tc_fence_after();
#pragma unroll
                            for (int split = 0; split < 2; ++split) {
                                const uint32_t apart = abuf + (uint32_t)((rb * 2 + split) * C::A_PART_BYTES);
#pragma unroll
                                for (int kc = 0; kc < C::KC; ++kc) {
#pragma unroll
                                    for (int kk = 0; kk < 4; ++kk) {
                                        const uint64_t bd = sw128_desc(bsm + kc * (C::BN * 128) + kk * 32);
                                        const uint64_t ad = sw128_desc(apart + kc * (BM * 128) + kk * 32);
                                        mma_bf16(tmem + (uint32_t)(rb * C::BN), ad, bd, idesc,
                                                 (split | kc | kk) ? 1u : 0u);
                                    }
                                }
                            }
                            mma_commit(smem_u32(&sh.acc_full[rb]));
                            last_bar = smem_u32(&sh.acc_full[rb]);
                            last_par = (uint32_t)gacc & 1u;
                        }
                        if (!ok) break;
                        mma_commit(smem_u32(&sh.b_empty[s]));
                    } else {
                        const int acc = gacc & 1;
                        if (!mbar_wait(smem_u32(&sh.acc_empty[acc]), ((uint32_t)(gacc >> 1) & 1u) ^ 1u, abort_flag,
                                       c.wait_limit_ns)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
#pragma unroll
                        for (int split = 0; split < 2; ++split) {
#pragma unroll
                            for (int kc = 0; kc < C::KC; ++kc) {
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk) {
                                    const uint64_t bd = sw128_desc(bsm + kc * (C::BN * 128) + kk * 32);
                                    const uint32_t accum = (split | kc | kk) ? 1u : 0u;
#pragma unroll
                                    for (int rb = 0; rb < RB; ++rb) {
                                        const uint32_t apart = abuf + (uint32_t)((rb * 2 + split) * C::A_PART_BYTES);
                                        const uint64_t ad = sw128_desc(apart + kc * (BM * 128) + kk * 32);
                                        mma_bf16(tmem + (uint32_t)(acc * RB * C::BN + rb * C::BN), ad, bd, idesc,
                                                 accum);
                                    }
                                }
                            }
                        }
                        mma_commit(smem_u32(&sh.b_empty[s]));
                        mma_commit(smem_u32(&sh.acc_full[acc]));
                        last_bar = smem_u32(&sh.acc_full[acc]);
                        last_par = (uint32_t)(gacc >> 1) & 1u;
                    }
                }
                if (!ok) break;
                mma_commit(smem_u32(&sh.a_empty[ab]));
            }
            if (!ok) {
                record_abort(sh, c);
                // drain: the last committed MMAs must finish before TMEM is freed
                if (last_bar) {
                    const int zero = 0;
                    mbar_wait(last_bar, last_par, (const volatile int *)&zero, 10000000ull);
                }
            }
        }
    } else if (warp < 4 || warp >= 4 + kEpiWarps) {
        // ---- A builders: builder b (warps 2, 3, 12, 13) fills row block b % RB,
        // 32-row slices (b / RB) * QN .. + QN - 1 of it, for each unit ----
        const int b = warp < 4 ? warp - 2 : warp - 4 - kEpiWarps + 2;
        const int rb = b % RB, s0 = (b / RB) * C::QN;
        // slot, ||y||_1 and centre of this lane's QN rows of a unit; gathered for
        // the next unit as soon as one is built, so the loads overlap the wait
        int sl[C::QN];
        float l1r[C::QN];
        uint64_t cwl[C::QN][W];
        auto gather = [&](int ii) {
            const int row0 = (((int)blockIdx.x + ii * (int)gridDim.x) / nch) * UM + rb * BM;
#pragma unroll
            for (int q = 0; q < C::QN; ++q) {
                const int row = row0 + (s0 + q) * 32 + lane;
                sl[q] = -1;
                l1r[q] = 0.0f;
#pragma unroll
                for (int w = 0; w < W; ++w) cwl[q][w] = 0;
                if (row < nrows) {
                    const int t = a.rows ? a.rows[row] : row;
                    sl[q] = a.row_frame ? a.row_frame[row] : t / a.L;
                    l1r[q] = a.l1[sl[q]];
                    const uint64_t *cw = a.cw + (int64_t)t * W;
#pragma unroll
                    for (int w = 0; w < W; ++w) cwl[q][w] = cw[w];
                }
            }
        };
        const int j0 = lane * EPL;  // this lane's elements of every row
        const int kcl = j0 / 64, e64 = j0 % 64;
        const int unit16 = e64 / 8, within = (e64 % 8) * 2;
        constexpr int WPL = EPL / 2;            // hi (and lo) words of a row per lane
        constexpr int GPS = 32 / C::G;          // groups of G rows per 32-row slice
        constexpr int NGRP = C::QN * GPS;       // groups per unit
        // split y of group gi (rows (s0 + gi / GPS) * 32 + (gi % GPS) * G + u):
        // their slots sit in lanes (gi % GPS) * G + u of slot gi / GPS
        auto load_group = [&](int gi, uint32_t (&dh)[C::G][WPL], uint32_t (&dl)[C::G][WPL]) {
            const int qq = gi / GPS, g0 = (gi % GPS) * C::G;
            int slq = sl[0];
#pragma unroll
            for (int u = 1; u < C::QN; ++u) slq = qq == u ? sl[u] : slq;
#pragma unroll
            for (int u = 0; u < C::G; ++u) {
                const int slot = __shfl_sync(0xffffffffu, slq, g0 + u);
                if (slot >= 0) {
                    const uint32_t *src = a.yhl + (int64_t)slot * N;
                    if constexpr (WPL == 1) {
                        dh[u][0] = src[lane];
                        dl[u][0] = src[N / 2 + lane];
                    } else {
                        const uint2 h2 = reinterpret_cast<const uint2 *>(src)[lane];
                        const uint2 l2 = reinterpret_cast<const uint2 *>(src + N / 2)[lane];
                        dh[u][0] = h2.x;
                        dh[u][1] = h2.y;
                        dl[u][0] = l2.x;
                        dl[u][1] = l2.y;
                    }
                } else {
#pragma unroll
                    for (int w = 0; w < WPL; ++w) dh[u][w] = dl[u][w] = 0u;
                }
            }
        };
        if (my_units > 0) gather(0);
        for (int i = 0; i < my_units; ++i) {
            const int ab = i % C::A_BUFS;
            // the buffer is free once its MMAs are done and the epilogue has read its norms
            bool ok = mbar_wait(smem_u32(&sh.a_empty[ab]), ((uint32_t)(i / C::A_BUFS) & 1u) ^ 1u, abort_flag,
                                c.wait_limit_ns) &&
                      mbar_wait(smem_u32(&sh.l1_free[ab]), ((uint32_t)(i / C::A_BUFS) & 1u) ^ 1u, abort_flag,
                                c.wait_limit_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) {
                if (lane == 0) record_abort(sh, c);
                break;
            }
            // ||y||_1 of this lane's rows, for the epilogue's re-rank margin
#pragma unroll
            for (int q = 0; q < C::QN; ++q) sh.l1[ab * UM + rb * BM + (s0 + q) * 32 + lane] = l1r[q];
            uint8_t *Ahi = Abase + ab * C::A_BUF_BYTES + (rb * 2 + 0) * C::A_PART_BYTES;
            uint8_t *Alo = Abase + ab * C::A_BUF_BYTES + (rb * 2 + 1) * C::A_PART_BYTES;
            // z = y x(c) in split form is the split of y with the sign bits of the
            // elements where c_j = 1 flipped (bf16 rounding is symmetric);
            // groups of G rows, the loads of group gi+1 in flight while gi is stored
            uint32_t ch[C::G][WPL], cl[C::G][WPL], nh[C::G][WPL], nl[C::G][WPL];
            load_group(0, ch, cl);
#pragma unroll 1
            for (int gi = 0; gi < NGRP; ++gi) {
                if (gi + 1 < NGRP) load_group(gi + 1, nh, nl);
                const int qq = gi / GPS, g0 = (gi % GPS) * C::G;
                uint64_t cq0 = cwl[0][0], cq1 = cwl[0][W - 1];
#pragma unroll
                for (int u = 1; u < C::QN; ++u) {
                    cq0 = qq == u ? cwl[u][0] : cq0;
                    cq1 = qq == u ? cwl[u][W - 1] : cq1;
                }
#pragma unroll
                for (int u = 0; u < C::G; ++u) {
                    const int r = (s0 + qq) * 32 + g0 + u;
                    // both words come from the row's owner lane; this lane keeps its chunk's word
                    uint64_t bits = __shfl_sync(0xffffffffu, cq0, g0 + u);
                    if constexpr (W > 1) {
                        const uint64_t hi_word = __shfl_sync(0xffffffffu, cq1, g0 + u);
                        bits = kcl ? hi_word : bits;
                    }
                    const uint32_t cb = (uint32_t)(bits >> (j0 & 63));  // c of this lane's elements, bit e
                    uint32_t hw[WPL], lw[WPL];
#pragma unroll
                    for (int w = 0; w < WPL; ++w) {
                        const uint32_t flip = ((cb >> (2 * w)) & 1u) << 15 | ((cb >> (2 * w + 1)) & 1u) << 31;
                        hw[w] = ch[u][w] ^ flip;
                        lw[w] = cl[u][w] ^ flip;
                    }
                    // element j of row r: chunk j/64, 16-B unit (j%64)/8 stored at unit ^ (r%8)
                    const int off =
                        kcl * (BM * 128) + (r / 8) * 1024 + (r % 8) * 128 + ((unit16 ^ (r % 8)) * 16) + within;
                    if constexpr (WPL == 1) {
                        *(uint32_t *)(Ahi + off) = hw[0];
                        *(uint32_t *)(Alo + off) = lw[0];
                    } else {
                        *(uint2 *)(Ahi + off) = make_uint2(hw[0], hw[1]);
                        *(uint2 *)(Alo + off) = make_uint2(lw[0], lw[1]);
                    }
                }
                (void)cq1;
#pragma unroll
                for (int u = 0; u < C::G; ++u)
#pragma unroll
                    for (int w = 0; w < WPL; ++w) {
                        ch[u][w] = nh[u][w];
                        cl[u][w] = nl[u][w];
                    }
            }
            if (i + 1 < my_units) gather(i + 1);
            fence_proxy_async();
            mbar_arrive(smem_u32(&sh.a_full[ab]));
        }
    } else {
        // ---- epilogue: TMEM -> registers -> running top-K lists ----
        // Warp 4 + 4h + q reads TMEM lane quadrant q, column half h of every
        // accumulator, so all eight warps work on each accumulator. A thread
        // keeps partial lists for row q*32+lane of both row blocks; at the end
        // of a unit it hands the one of row block 1-h to its partner (warp
        // 4 + 4(1-h) + q, same lane) through shared memory and finishes row
        // block h.
        const int q = warp & 3;
        const int h = (warp - 4) >> 2;
        const int r = q * 32 + lane;
        constexpr int HALF = C::BN / 2;  // columns per warp per accumulator
        int gacc = 0;
        bool ok = true;
        int nsplit = 0;  // split items finished by this CTA (phase of epi_pub / epi_last)
        auto row_of = [&](int ii, int rbx) {
            return (((int)blockIdx.x + ii * (int)gridDim.x) / nch) * UM + rbx * BM + r;
        };
        for (int i = 0; i < my_units && ok; ++i) {
            const int item = (int)blockIdx.x + i * (int)gridDim.x;
            const int unit = item / nch, ch = item % nch;
            // the builders leave ||y||_1 of this unit's rows beside its A tiles
            const int ab = i % C::A_BUFS;
            {
                bool w = mbar_wait(smem_u32(&sh.a_full[ab]), (uint32_t)(i / C::A_BUFS) & 1u, abort_flag, c.wait_limit_ns);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
            }
            float tv[RB][kTopK], thr[RB], eps2[RB];
            int ti[RB][kTopK];
#pragma unroll
            for (int rbx = 0; rbx < RB; ++rbx) {
#pragma unroll
                for (int k = 0; k < kTopK; ++k) {
                    tv[rbx][k] = CUDART_INF_F;
                    ti[rbx][k] = -1;
                }
                thr[rbx] = CUDART_INF_F;
                // 2 eps of this row (the re-rank margin), from ||y||_1 of its frame, and at
                // least the smallest normal float: with y = 0 every score ties at 0, and a
                // zero margin would admit only the first of them where the band holds all
                eps2[rbx] = fmaxf(__fmul_ru(2.0f * kEpsScale, __fmul_ru(sh.l1[ab * UM + rbx * BM + r], 1.0f + 1.0f / 1024.0f)),
                                  1.17549435e-38f);
            }
            mbar_arrive(smem_u32(&sh.l1_free[ab]));
            for (int j = ch * nt / nch; j < (ch + 1) * nt / nch && ok; ++j, ++gacc) {
                const bool full = (j + 1) * C::BN <= P;
                if constexpr (!C::SEQ) {
                    bool w = mbar_wait(smem_u32(&sh.acc_full[gacc & 1]), (uint32_t)(gacc >> 1) & 1u, abort_flag,
                                       c.wait_limit_ns);
                    if (!__all_sync(0xffffffffu, w)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                }
                // both row blocks' code unrolled, each on its own list registers (one
                // copy with the lists swapped after each row block measured 4-6 % slower:
                // the swaps cost more moves than the second copy costs fetch)
#pragma unroll
                for (int rbx = 0; rbx < RB; ++rbx) {
                    if constexpr (C::SEQ) {
                        bool w = mbar_wait(smem_u32(&sh.acc_full[rbx]), (uint32_t)gacc & 1u, abort_flag, c.wait_limit_ns);
                        if (!__all_sync(0xffffffffu, w)) {
                            ok = false;
                            break;
                        }
                        tc_fence_after();
                    }
                    const uint32_t col = (C::SEQ ? (uint32_t)(rbx * C::BN) : (uint32_t)((gacc & 1) * RB * C::BN + rbx * C::BN)) +
                                         (uint32_t)(h * HALF);
                    // the other half's best so far is an upper bound on the row's
                    // minimum: nothing at or above it + 2 eps can be a candidate
                    volatile unsigned long long *best = sh.best + (rbx * BM + r) * 2;
                    {
                        const unsigned long long pb = best[1 - h];
                        if ((int)(pb >> 32) == item)
                            thr[rbx] = fminf(thr[rbx], __fadd_ru(__uint_as_float((uint32_t)pb), eps2[rbx]));
                    }
                    const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + col;
                    const int cb0 = j * C::BN + h * HALF;
                    if constexpr (C::SEQ) {
                        // 64-column chunks in one register buffer (two buffers would not
                        // fit; 32-column slices in two buffers measured slower here)
#pragma unroll 1
                        for (int cc = 0; cc < HALF / 64; ++cc) {
                            // columns past P hold nothing (the last tile's MMAs are narrower)
                            if (cb0 + cc * 64 >= P) break;
                            uint32_t v[64];
                            __syncwarp();
                            tmem_ld64(tbase + (uint32_t)(cc * 64), v);
                            epi_chunk<64>(v, cb0 + cc * 64, P, full, tv[rbx], ti[rbx], thr[rbx], eps2[rbx]);
                        }
                        tc_fence_before();
                        mbar_arrive(smem_u32(&sh.acc_empty[rbx]));
                    } else {
                        // 32-column slices in two register buffers: the next slice's TMEM
                        // load is in flight while the current one is scanned, and the
                        // accumulator is released once the last slice is in registers
                        constexpr int NS = HALF / 32;
                        static_assert(NS % 2 == 0, "slices come in pairs");
                        uint32_t va[32], vb[32];
                        __syncwarp();
                        tmem_ld32(tbase, va);
                        tmem_wait(va);
#pragma unroll 1
                        for (int sl = 0; sl < NS; sl += 2) {
                            __syncwarp();
                            tmem_ld32(tbase + (uint32_t)((sl + 1) * 32), vb);
                            epi_chunk<32>(va, cb0 + sl * 32, P, full, tv[rbx], ti[rbx], thr[rbx], eps2[rbx]);
                            __syncwarp();
                            tmem_wait(vb);
                            if (sl + 2 < NS) {
                                tmem_ld32(tbase + (uint32_t)((sl + 2) * 32), va);
                            } else if (rbx == RB - 1) {
                                // every column of the accumulator has been read
                                tc_fence_before();
                                mbar_arrive(smem_u32(&sh.acc_empty[gacc & 1]));
                            }
                            epi_chunk<32>(vb, cb0 + (sl + 1) * 32, P, full, tv[rbx], ti[rbx], thr[rbx], eps2[rbx]);
                            if (sl + 2 < NS) {
                                __syncwarp();
                                tmem_wait(va);
                            }
                        }
                    }
                    best[h] = ((unsigned long long)(uint32_t)item << 32) | __float_as_uint(tv[rbx][0]);
                }

            }
            if (!ok) break;
            // exchange halves: publish the list of row block 1-h (after the partner
            // has read the previous unit's), then merge the partner's of row block h
            if (i > 0) {
                bool w = mbar_wait(smem_u32(sh.xchg), 1u, abort_flag, c.wait_limit_ns);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
            }
#pragma unroll
            for (int k = 0; k < kTopK; ++k) {
                sh.xv[((1 - h) * BM + r) * kTopK + k] = h ? tv[0][k] : tv[1][k];
                sh.xi[((1 - h) * BM + r) * kTopK + k] = h ? ti[0][k] : ti[1][k];
            }
            mbar_arrive(smem_u32(sh.xchg));
            {
                bool w = mbar_wait(smem_u32(sh.xchg), 0u, abort_flag, c.wait_limit_ns);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
            }
            const int row = row_of(i, h);
            float fv[kTopK];
            int fi[kTopK];
            const float feps2 = h ? eps2[1] : eps2[0];
            float fthr = h ? thr[1] : thr[0];
#pragma unroll
            for (int k = 0; k < kTopK; ++k) {
                fv[k] = h ? tv[1][k] : tv[0][k];
                fi[k] = h ? ti[1][k] : ti[0][k];
            }
#pragma unroll
            for (int k = 0; k < kTopK; ++k) {
                const float pv = sh.xv[(h * BM + r) * kTopK + k];
                const int pi = sh.xi[(h * BM + r) * kTopK + k];
                if (pi >= 0 && pv < fthr) {
                    topk_insert<kTopK>(fv, fi, pv, pi);
                    fthr = admit_thr(fv, feps2);
                }
            }
            mbar_arrive(smem_u32(sh.xchg));
            if (nch > 1) {
                // publish this chunk's list; the last chunk of the unit merges them all
                const size_t slot = ((size_t)item * UM + h * BM + r) * kTopK;
#pragma unroll
                for (int k = 0; k < kTopK; ++k) {
                    a.split_val[slot + k] = fv[k];
                    a.split_idx[slot + k] = fi[k];
                }
                __threadfence();
                // all epilogue threads published -> one thread counts the chunk -> all read
                // whether it was the unit's last (bounded waits, so an abort cannot wedge them)
                const uint32_t par = (uint32_t)(nsplit & 1);
                ++nsplit;
                mbar_arrive(smem_u32(sh.epi_pub));
                if (threadIdx.x == 4 * 32) {
                    if (mbar_wait(smem_u32(sh.epi_pub), par, abort_flag, c.wait_limit_ns)) {
                        *(volatile int *)sh.last_flag = (atomicAdd(&a.unit_done[unit], 1) == nch - 1);
                        __threadfence();
                    }
                    mbar_arrive(smem_u32(sh.epi_last));
                }
                bool w2 = mbar_wait(smem_u32(sh.epi_last), par, abort_flag, c.wait_limit_ns);
                w2 = __all_sync(0xffffffffu, w2);
                if (!w2) {
                    ok = false;
                    break;
                }
                const bool last = *(volatile int *)sh.last_flag != 0;
                if (!last) continue;
                __threadfence();
#pragma unroll
                for (int k = 0; k < kTopK; ++k) {
                    fv[k] = CUDART_INF_F;
                    fi[k] = -1;
                }
                fthr = CUDART_INF_F;
                // chunks in pattern order (ties keep the lower index), four chunks' loads in flight
                for (int c0 = 0; c0 < nch; c0 += 4) {
                    float pv[4][kTopK];
                    int pi[4][kTopK];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const size_t src = ((size_t)(unit * nch + min(c0 + u, nch - 1)) * UM + h * BM + r) * kTopK;
                        const float4 v4 = __ldcg(reinterpret_cast<const float4 *>(a.split_val + src));
                        const int4 i4 = __ldcg(reinterpret_cast<const int4 *>(a.split_idx + src));
                        pv[u][0] = v4.x; pv[u][1] = v4.y; pv[u][2] = v4.z; pv[u][3] = v4.w;
                        pi[u][0] = i4.x; pi[u][1] = i4.y; pi[u][2] = i4.z; pi[u][3] = i4.w;
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        if (c0 + u >= nch) break;
#pragma unroll
                        for (int k = 0; k < kTopK; ++k) {
                            if (pi[u][k] >= 0 && pv[u][k] < fthr) {
                                topk_insert<kTopK>(fv, fi, pv[u][k], pi[u][k]);
                                fthr = admit_thr(fv, feps2);
                            }
                        }
                    }
                }
                if (threadIdx.x == 4 * 32) a.unit_done[unit] = 0;  // ready for the next launch
            }
            if (row < nrows) {
                // entries admitted before the minimum was seen may lie outside its band
                const float band = __fadd_ru(fv[0], feps2);
#pragma unroll
                for (int k = 0; k < kTopK; ++k) {
                    const bool keep = k == 0 || fv[k] < band;
                    a.topk_val[(int64_t)row * kTopK + k] = keep ? fv[k] : CUDART_INF_F;
                    a.topk_idx[(int64_t)row * kTopK + k] = keep ? fi[k] : -1;
                }
            }
        }
        if (!ok && lane == 0) record_abort(sh, c);
    }

    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

template <int N, int BN_, int BLD, int BST>
cudaError_t launch_shape(const CodeDev &c, const ScoreArgs &a, cudaStream_t s) {
    using C = TcCfg<N, BN_, BLD, BST>;
    static_assert(C::SMEM_BYTES <= 227 * 1024, "shared memory of one CTA");
    // the pattern tiles are stored for tc_patterns_per_tile(N); a narrower tile
    // must be a prefix of each stored tile's image (one 128-byte K chunk)
    static_assert(BN_ == tc_patterns_per_tile(N) || (C::KC == 1 && tc_patterns_per_tile(N) % BN_ == 0),
                  "pattern tile images");
    constexpr int smem = C::SMEM_BYTES;
    cudaError_t e = cudaFuncSetAttribute(score_tc_kernel<N, BN_, BLD, BST>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         smem);
    if (e != cudaSuccess) return e;
    int64_t grid = c.num_sms;
    if (!a.n_rows_dev) grid = std::min<int64_t>(grid, (a.n_rows + UM - 1) / UM);
    if (grid <= 0) return cudaSuccess;
    score_tc_kernel<N, BN_, BLD, BST><<<(unsigned)grid, C::THREADS, smem, s>>>(a, c);
    return cudaGetLastError();
}

}  // namespace
}  // namespace mpwsd
