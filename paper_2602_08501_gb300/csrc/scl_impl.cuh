#pragma once
// Stage-1 kernel templates (included by the scl_*.cu instantiation units).
//
// Stage 1 of the two-stage decoder (Sec. III-A): batched min-sum SC-list
// decoding on the Arikan transform, CRC check of the most reliable candidate
// with early termination, and compaction of the failing frames into stage-2
// trajectories (one per list entry = anchor, Algorithm 1 init).
//
// GPU mapping: one thread per list path, LW = next power of two >= L lanes per
// frame, 32 / LW frames per warp. The SC schedule (which f / g updates run
// before each leaf) does not depend on the data, so it is unrolled at compile
// time and every LLR lives in a register. At an information leaf the 2|list|
// children are ordered by the key (metric, parent position, bit) with bitonic
// networks across the frame's lanes; each surviving child takes a lane and
// copies from its parent lane only the state still needed later (LLR arrays
// of ancestors whose right subtree is pending, left-subtree codewords of
// ancestors whose right subtree is running). Integer LLRs: inputs on the 2^-19 grid are exact int32, path
// metrics int64, so the list equals the FP64 formulation bit for bit.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math_constants.h>
#include <stdint.h>

#include "common.cuh"

namespace mpwsd {
namespace scl_detail {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;

template <int X>
struct Log2 {
    static constexpr int v = 1 + Log2<X / 2>::v;
};
template <>
struct Log2<1> {
    static constexpr int v = 0;
};

constexpr int cpop(uint32_t x) { return x == 0 ? 0 : (int)(x & 1u) + cpop(x >> 1); }

// Frozen mask of RM(r, m) in the Arikan form: row i is frozen iff its weight
// 2^popcount(i) is below the minimum distance 2^(m-r).
constexpr uint64_t rm_mask(int m, int r, int word) {
    uint64_t v = 0;
    for (int b = 0; b < 64; ++b) {
        int i = word * 64 + b;
        if (i < (1 << m) && cpop((uint32_t)i) < m - r) v |= 1ull << b;
    }
    return v;
}

struct FrozenRT {
    static constexpr bool kConst = false;
    uint64_t lo, hi;
    template <int I>
    __device__ __forceinline__ bool frozen() const {
        if constexpr (I < 64)
            return (lo >> I) & 1ull;
        else
            return (hi >> (I - 64)) & 1ull;
    }
};

template <uint64_t LO, uint64_t HI>
struct FrozenCT {
    static constexpr bool kConst = true;
    uint64_t lo, hi;  // unused, keeps the launch signature uniform
    template <int I>
    __device__ __forceinline__ static constexpr bool frozen() {
        if constexpr (I < 64)
            return (LO >> I) & 1ull;
        else
            return (HI >> (I - 64)) & 1ull;
    }
};

template <int N>
struct PathState {
    int llr[N];                    // node of size S < N keeps its LLRs at [S, 2S)
    uint64_t beta[Log2<N>::v];     // beta[log2 H]: codeword of the finished left child of size H
    // Lazy cloning: a path that takes over another path's history at an
    // information leaf does not copy the pending arrays; it records the lane
    // that holds them. src[log2 S]: lane holding this path's inputs of the
    // running node of size S; bsrc[log2 H]: lane holding its beta[log2 H].
    // Every path runs the same schedule, so no lane overwrites a pending
    // array before the step that reads it fetches it.
    int src[Log2<N>::v];
    int bsrc[Log2<N>::v];
    long long pm;                  // path metric, units of 2^-19
};

template <class FZ>
struct SclCtx {
    const int *ych;                // channel LLRs of this frame (shared memory)
    int lane;                      // lane within the frame's segment
    uint32_t dirs;                 // directions of this lane's sorting-network stages
    int count;                     // current list size (uniform over the warp)
    long long pref;                // lower bound on every path metric of the frame
    int L;
    uint64_t root_cw[2];           // root codeword when n = 128
    FZ fz;
};

// sign(a) sign(b) min(|a|,|b|) with sign(0) = +1, as max(min(a,b), -max(a,b)):
// both >= 0 gives min(a,b); both <= 0 gives -max(a,b) = min(|a|,|b|); mixed
// signs give the larger of two non-positive values, -min(|a|,|b|)
__device__ __forceinline__ int minsum_f(int a, int b) {
    return max(min(a, b), -max(a, b));
}

template <int N, int S>
__device__ __forceinline__ int parent_llr(const int *ych, const PathState<N> &st, int k) {
    if constexpr (S == N)
        return ych[k];
    else
        return st.llr[S + k];
}

// A path continuing the history of lane par: for every node that is still
// running (leaf I in its left half: inputs pending; in its right half: left
// child's codeword pending) take over par's source lane.
template <int N, int LW, int I, int S>
__device__ __forceinline__ void clone_src(PathState<N> &st, int par) {
    if constexpr (S <= N / 2) {
        if constexpr ((I & (S / 2)) == 0) st.src[Log2<S>::v] = __shfl_sync(kFull, st.src[Log2<S>::v], par, LW);
        clone_src<N, LW, I, S * 2>(st, par);
    }
}

template <int N, int LW, int I, int H>
__device__ __forceinline__ void clone_bsrc(PathState<N> &st, int par) {
    if constexpr (H <= N / 2) {
        if constexpr ((I & H) != 0) st.bsrc[Log2<H>::v] = __shfl_sync(kFull, st.bsrc[Log2<H>::v], par, LW);
        clone_bsrc<N, LW, I, H * 2>(st, par);
    }
}

// Whether leaves [OFF, OFF + LEN) hold an information leaf (always assumed for
// a frozen set known only at run time).
template <class FZ, int OFF, int LEN>
__device__ __forceinline__ constexpr bool has_info() {
    if constexpr (!FZ::kConst) {
        return true;
    } else if constexpr (LEN == 1) {
        return !FZ::template frozen<OFF>();
    } else {
        return has_info<FZ, OFF, LEN / 2>() || has_info<FZ, OFF + LEN / 2, LEN / 2>();
    }
}

// Outcome of the list step at an information leaf, for one lane.
struct LeafStep {
    long long pm;   // new path metric (kept lanes)
    long long pref; // smallest metric of the new list (a lower bound on every later one)
    int par;        // lane whose history this lane continues
    int count;      // new list size
    unsigned bit;   // decided u of this lane's path
};

// Which stages of the bitonic sort below keep the smaller key at this lane:
// bit s for stage s (stages in network order). It depends only on the lane,
// so each thread computes it once instead of at every stage of every list step.
template <int LW>
__device__ __forceinline__ uint32_t sort_dirs(int lane) {
    uint32_t d = 0;
    int s = 0;
    for (int k = 2; k <= LW; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1, ++s)
            if (((lane & k) == 0) == ((lane & j) == 0)) d |= 1u << s;
    return d;
}

// Bitonic sort of one key per lane over the LW lanes of a frame (ascending in
// lane order): each stage compares with the lane j apart and keeps the smaller
// or the larger key by the lane's place in the network (dirs = sort_dirs).
template <int LW, class K>
__device__ __forceinline__ K seg_sort(K x, uint32_t dirs) {
    int s = 0;
#pragma unroll
    for (int k = 2; k <= LW; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1, ++s) {
            const K o = __shfl_xor_sync(kFull, x, j, LW);
            x = (dirs & (1u << s)) ? min(x, o) : max(x, o);
        }
    }
    return x;
}

// The LW smallest of two ascending sequences a (in lane order) and b: against
// b reversed, the lane-wise minima are those LW keys as a bitonic sequence,
// which the merge half of the network puts in ascending lane order.
template <int LW, class K>
__device__ __forceinline__ K seg_merge_low(K a, K b, int lane) {
    K x = min(a, __shfl_sync(kFull, b, LW - 1 - lane, LW));
#pragma unroll
    for (int j = LW / 2; j > 0; j >>= 1) {
        const K o = __shfl_xor_sync(kFull, x, j, LW);
        x = (lane & j) ? max(x, o) : min(x, o);
    }
    return x;
}

// The list step at an information leaf (it does not depend on which leaf, so
// one copy of its code serves all of them): each of the |list| paths spawns
// the children (u = HD, metric pm) and (u = 1 - HD, metric pm + |lam|); the
// 2 |list| children are ordered by the key (metric, parent position, bit) and
// the first min(2 |list|, L) are kept, child r going to lane r. The keys are
// distinct (parent position and bit are in them), so sorting them gives that
// order exactly: the two children sets are sorted apart (bitonic networks
// across the frame's lanes) and merged keeping the smallest LW, so lane r ends
// with the r-th child. Metrics are taken relative to the smallest metric the
// list had after the previous list step (metrics only grow, so none is
// below it); when every relative metric of the segment fits 25 bits the keys
// fit 32 bits (the usual case), otherwise the same network runs on 64-bit keys.
template <int LW>
__device__ __noinline__ LeafStep list_step(int lam, long long pm, int lane, uint32_t dirs, int count, int L, long long pref) {
    const unsigned hd = lam < 0 ? 1u : 0u;
    const long long a = lam < 0 ? -(long long)lam : (long long)lam;
    const bool valid = lane < count;
    // metrics only grow, so the smallest metric after the last list step bounds every
    // metric now from below: keys relative to it are non-negative
    const long long d0 = pm - pref;
    const bool small = !valid || d0 + a < (1LL << 25);
    const int nc = min(2 * count, L);
    const bool keep = lane < nc;
    LeafStep out;
    out.count = nc;
    if (__all_sync(kFull, small)) {
        const uint32_t base32 = (uint32_t)lane << 1;
        const uint32_t q0 = valid ? (((uint32_t)d0 << 6) | base32 | hd) : 0xffffffffu;
        const uint32_t q1 = valid ? (((uint32_t)(d0 + a) << 6) | base32 | (hd ^ 1u)) : 0xffffffffu;
        const uint32_t kk = seg_merge_low<LW>(seg_sort<LW>(q0, dirs), seg_sort<LW>(q1, dirs), lane);
        out.par = keep ? (int)((kk >> 1) & 31u) : lane;
        out.pm = keep ? pref + (long long)(kk >> 6) : pm;
        out.bit = keep ? (kk & 1u) : 0u;
        out.pref = pref + (long long)(__shfl_sync(kFull, kk, 0, LW) >> 6);
    } else {
        const unsigned long long base = ((unsigned long long)lane << 1);
        const unsigned long long k0 = valid ? (((unsigned long long)pm << 6) | base | hd) : ~0ull;
        const unsigned long long k1 = valid ? (((unsigned long long)(pm + a) << 6) | base | (hd ^ 1u)) : ~0ull;
        const unsigned long long kk = seg_merge_low<LW>(seg_sort<LW>(k0, dirs), seg_sort<LW>(k1, dirs), lane);
        out.par = keep ? (int)((kk >> 1) & 31ull) : lane;
        out.pm = keep ? (long long)(kk >> 6) : pm;
        out.bit = keep ? (unsigned)(kk & 1ull) : 0u;
        out.pref = (long long)(__shfl_sync(kFull, kk, 0, LW) >> 6);
    }
    return out;
}

template <int N, int LW, class FZ, int I>
__device__ __forceinline__ uint64_t info_leaf(SclCtx<FZ> &cx, PathState<N> &st) {
    const int lam = st.llr[1];
    if constexpr (LW == 1) {
        // one path: the child with the smaller key is always the hard decision
        return lam < 0 ? 1u : 0u;
    } else {
        const LeafStep o = list_step<LW>(lam, st.pm, cx.lane, cx.dirs, cx.count, cx.L, cx.pref);
        cx.pref = o.pref;
        clone_src<N, LW, I, 2>(st, o.par);
        clone_bsrc<N, LW, I, 1>(st, o.par);
        st.pm = o.pm;
        cx.count = o.count;
        return o.bit;
    }
}
template <int N, int LW, class FZ, int I>
__device__ __forceinline__ uint64_t leaf(SclCtx<FZ> &cx, PathState<N> &st) {
    bool frz;
    if constexpr (FZ::kConst)
        frz = FZ::template frozen<I>();
    else
        frz = cx.fz.template frozen<I>();
    if (frz) {
        const int lam = st.llr[1];
        st.pm += max(-lam, 0);  // decided bit 0 disagrees with HD = 1 when lam < 0
        return 0;
    }
    return info_leaf<N, LW, FZ, I>(cx, st);
}

// Node of size S whose first leaf is OFF: returns the node's codeword (S <= 64)
template <int N, int LW, class FZ, int S, int OFF>
__device__ __forceinline__ uint64_t node(SclCtx<FZ> &cx, PathState<N> &st) {
    if constexpr (S == 1) {
        return leaf<N, LW, FZ, OFF>(cx, st);
    } else if constexpr (S < N && !has_info<FZ, OFF, S>()) {
        // all-frozen node: every leaf decides 0. With P(x) = max(0, -x) the
        // min-sum updates satisfy P(f(a, b)) + P(a + b) = P(a) + P(b), so the
        // leaves' metric increments add up to sum_k P(input_k) of this node
        // (integers: exactly the leaf-by-leaf sum), and its codeword is 0
        int add = 0;  // at most 2^23 N <= 2^30: every input of a node of size S is at most 2^23 N / S
#pragma unroll
        for (int k = 0; k < S; ++k) add += max(-st.llr[S + k], 0);
        st.pm += add;
        return 0;
    } else {
        constexpr int H = S / 2;
        constexpr int LG = Log2<H>::v;
        // a xor b on the left half: f (this node's inputs are still this lane's own)
#pragma unroll
        for (int k = 0; k < H; ++k)
            st.llr[H + k] = minsum_f(parent_llr<N, S>(cx.ych, st, k), parent_llr<N, S>(cx.ych, st, k + H));
        if constexpr (H > 1) st.src[Log2<H>::v] = cx.lane;
        st.beta[LG] = node<N, LW, FZ, H, OFF>(cx, st);
        if constexpr (LW > 1) st.bsrc[LG] = cx.lane;
        // b on the right half: g with the re-encoded left decisions; if the left
        // half branched, this path's inputs now live in lane src
        constexpr bool moved = LW > 1 && S < N && has_info<FZ, OFF, H>();
#pragma unroll
        for (int k = 0; k < H; ++k) {
            int a, b;
            if constexpr (moved) {
                a = __shfl_sync(kFull, st.llr[S + k], st.src[Log2<S>::v], LW);
                b = __shfl_sync(kFull, st.llr[S + k + H], st.src[Log2<S>::v], LW);
            } else {
                a = parent_llr<N, S>(cx.ych, st, k);
                b = parent_llr<N, S>(cx.ych, st, k + H);
            }
            st.llr[H + k] = ((st.beta[LG] >> k) & 1ull) ? b - a : b + a;
        }
        if constexpr (H > 1) st.src[Log2<H>::v] = cx.lane;
        const uint64_t gr = node<N, LW, FZ, H, OFF + H>(cx, st);
        uint64_t be = st.beta[LG];
        if constexpr (LW > 1 && has_info<FZ, OFF + H, H>()) be = __shfl_sync(kFull, be, st.bsrc[LG], LW);
        if constexpr (S <= 64) {
            return (be ^ gr) | (gr << (H & 63));
        } else {
            cx.root_cw[0] = be ^ gr;
            cx.root_cw[1] = gr;
            return 0;
        }
    }
}

__device__ __forceinline__ int quantize(float y) {
    int v = __float2int_rn(y * 524288.0f);  // y * 2^19, round to nearest even
    return max(-kGridMax, min(kGridMax, v));
}

template <int N, int LW>
struct SclShape {
    static constexpr int kFPW = 32 / LW;  // frames per warp
    static constexpr int kBytesPerWarp = kFPW * N * 4;
    static constexpr int kWarps = kBytesPerWarp * kWarpsPerBlock <= 32768 ? kWarpsPerBlock
                                  : (kBytesPerWarp * 2 <= 32768 ? 2 : 1);
    // n = 64 with 2 to 16 lanes per frame: 7 blocks of 4 warps per SM (at most 72
    // registers a thread, 28 warps instead of the 24 that 80 registers allow)
    static constexpr bool kOcc = N == 64 && LW > 1 && LW < 32 && kWarps == 4;
    static constexpr int kMinBlocks = 7;
};

template <int N, int LW, class FZ>
__device__ __forceinline__ void scl_body(const SclArgs &a, const CodeDev &c, const FZ &fz) {
    constexpr int FPW = SclShape<N, LW>::kFPW;
    constexpr int WPB = SclShape<N, LW>::kWarps;
    constexpr int W = (N + 63) / 64;
    __shared__ int s_y[WPB][FPW][N];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int seg = lane / LW, sl = lane % LW;
    const int64_t fbase = ((int64_t)blockIdx.x * WPB + warp) * FPW;
    if (a.ws.pool.cap > 0 && blockIdx.x == 0 && threadIdx.x == 0 && a.mode == 0)
        atomicAdd(&c.stats->frames, (unsigned long long)a.B);  // pool: counted per submission
    if (fbase >= a.B) return;  // whole warp leaves together
    for (int idx = lane; idx < FPW * N; idx += 32) {
        const int64_t f = fbase + idx / N;
        s_y[warp][idx / N][idx % N] = f < a.B ? quantize(a.y[f * N + (idx % N)]) : 0;
    }
    __syncwarp();

    SclCtx<FZ> cx;
    cx.ych = s_y[warp][seg];
    cx.lane = sl;
    cx.dirs = sort_dirs<LW>(sl);
    cx.count = 1;
    cx.pref = 0;
    cx.L = a.L;
    cx.fz = fz;
    PathState<N> st;
    st.pm = 0;
    uint64_t cw[2];
    {
        const uint64_t r = node<N, LW, FZ, N, 0>(cx, st);
        if constexpr (N <= 64) {
            cw[0] = r;
            cw[1] = 0;
        } else {
            cw[0] = cx.root_cw[0];
            cw[1] = cx.root_cw[1];
        }
    }
    const int count = cx.count;
    const bool valid = sl < count;
    int pos = sl;
    if (c.trailing_frozen) {  // frozen leaves after the last branching: stable re-sort by metric
        int rank = 0;
#pragma unroll
        for (int s = 0; s < LW; ++s) {
            const long long pm_s = __shfl_sync(kFull, st.pm, s, LW);
            rank += (s < count) && (pm_s < st.pm || (pm_s == st.pm && s < sl));
        }
        pos = valid ? rank : sl;
    }
    const int64_t frame = fbase + seg;
    const unsigned segmask = (LW == 32) ? kFull : (((1u << LW) - 1u) << (seg * LW));
    if (frame >= a.B) return;  // whole segment leaves together

    if (a.mode == 1) {
        if (valid) {
            uint64_t *dst = a.list_cw + (frame * a.L + pos) * W;
            dst[0] = cw[0];
            if (W > 1) dst[1] = cw[1];
            a.list_pm[frame * a.L + pos] = st.pm;
        }
        return;
    }

    // CRC in the codeword domain: syndrome bit b = parity(c & mask_b)
    bool ok = false;
    if (a.use_crc && valid) {
        unsigned syn = 0;
        for (int b = 0; b < c.crc_len; ++b) {
            const uint64_t *mk = c.crc_masks + (size_t)b * W;
            int p = __popcll(cw[0] & mk[0]);
            if (W > 1) p += __popcll(cw[1] & mk[1]);
            syn |= (unsigned)(p & 1);
        }
        ok = syn == 0;
    }
    int key = (ok && (a.rule == MPWSD_RULE_ANY || pos == 0)) ? pos : 0x7fff;
#pragma unroll
    for (int o = LW / 2; o >= 1; o >>= 1) key = min(key, __shfl_xor_sync(segmask, key, o, LW));
    const bool pool = a.ws.pool.cap > 0;
    if (key != 0x7fff) {
        if (pos == key) {
            uint64_t *dst = a.cw_out + frame * W;
            dst[0] = cw[0];
            if (W > 1) dst[1] = cw[1];
            a.flags_out[frame] = (uint16_t)MPWSD_FLAG_CRC_OK;
            if (a.done_out) a.done_out[frame] = -(a.submit_id + 1);
        }
        return;
    }
    // stage 2: this frame becomes a slot with one trajectory per list entry
    int slot = 0, base = 0;
    if (sl == 0) {
        slot = pool ? pool_take_slot(a.ws) : atomicAdd(&a.ws.counters[0], 1);
        base = atomicAdd(&a.ws.counters[1], count);
    }
    slot = __shfl_sync(segmask, slot, 0, LW);
    base = __shfl_sync(segmask, base, 0, LW);
    // ||y||_1 on the grid, summed across the segment's lanes (exact: < 2^30)
    int l1 = 0;
    for (int j = sl; j < N; j += LW) l1 += abs(cx.ych[j]);
#pragma unroll
    for (int o = LW / 2; o >= 1; o >>= 1) l1 += __shfl_xor_sync(segmask, l1, o, LW);
    if (sl == 0) {
        // a pool slot keeps its own copy of y, so y is read at the slot itself
        a.ws.slot_frame[slot] = pool ? slot : (int)(a.f0 + frame);
        a.ws.slot_l1[slot] = (float)l1 * (1.0f / 524288.0f);
        if (pool) {
            a.ws.pool.live[slot] = count;
            unsigned long long *d = a.ws.pool.dst + 3 * (int64_t)slot;
            d[0] = (unsigned long long)(a.cw_out + frame * W);
            d[1] = (unsigned long long)(a.flags_out + frame);
            d[2] = a.done_out ? (unsigned long long)(a.done_out + frame) : 0ull;
        }
    }
    if (pool)
        for (int j = sl; j < N; j += LW) a.ws.pool.slot_y[(int64_t)slot * N + j] = (float)cx.ych[j] * (1.0f / 524288.0f);
    if (a.write_yhl) {
        // y in the split form the tensor-core scoring consumes: word w holds
        // elements 2w (low half) and 2w+1 of hi = bf16(y) and of lo = bf16(y - hi)
        uint32_t *dst = a.ws.slot_yhl + (int64_t)slot * N;
        for (int w = sl; w < N / 2; w += LW) {
            uint32_t h2 = 0, l2 = 0;
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const float v = (float)cx.ych[2 * w + e] * (1.0f / 524288.0f);
                const __nv_bfloat16 h = __float2bfloat16_rn(v);
                const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
                h2 |= (uint32_t)__bfloat16_as_ushort(h) << (16 * e);
                l2 |= (uint32_t)__bfloat16_as_ushort(l) << (16 * e);
            }
            dst[w] = h2;
            dst[N / 2 + w] = l2;
        }
    }
    if (sl < a.L) {
        const int64_t t = (int64_t)slot * a.L + pos;
        uint64_t *dst = a.ws.traj_cw + t * W;
        if (valid) {
            int corr = 0;  // sum_j yhat_j x_j, exact (|.| < 2^30)
#pragma unroll 8
            for (int j = 0; j < N; ++j) {
                const int v = cx.ych[j];
                corr += ((cw[j >> 6] >> (j & 63)) & 1ull) ? -v : v;
            }
            dst[0] = cw[0];
            if (W > 1) dst[1] = cw[1];
            a.ws.traj_D[t] = -(double)corr * (1.0 / 524288.0);
            a.ws.traj_state[t] = kTrajValid;
            a.ws.act[0][base + pos] = (int)t;
        } else {
            dst[0] = 0;
            if (W > 1) dst[1] = 0;
            a.ws.traj_D[t] = CUDART_INF;
            a.ws.traj_state[t] = 0;
        }
    }
}

template <int N, int LW, class FZ>
__global__ void __launch_bounds__(SclShape<N, LW>::kWarps * 32) scl_kernel(const SclArgs a, const CodeDev c, const FZ fz) {
    scl_body<N, LW, FZ>(a, c, fz);
}

// the same kernel with the register bound of SclShape::kMinBlocks resident blocks
template <int N, int LW, class FZ>
__global__ void __launch_bounds__(SclShape<N, LW>::kWarps * 32, SclShape<N, LW>::kMinBlocks)
    scl_kernel_occ(const SclArgs a, const CodeDev c, const FZ fz) {
    scl_body<N, LW, FZ>(a, c, fz);
}

template <int N, int LW, class FZ>
cudaError_t launch_one(const CodeDev &c, const SclArgs &a, const FZ &fz, cudaStream_t s) {
    constexpr int WPB = SclShape<N, LW>::kWarps;
    constexpr int FPB = WPB * (32 / LW);
    const int64_t blocks = (a.B + FPB - 1) / FPB;
    if (blocks == 0) return cudaSuccess;
    if constexpr (SclShape<N, LW>::kOcc)
        scl_kernel_occ<N, LW, FZ><<<(unsigned)blocks, WPB * 32, 0, s>>>(a, c, fz);
    else
        scl_kernel<N, LW, FZ><<<(unsigned)blocks, WPB * 32, 0, s>>>(a, c, fz);
    return cudaGetLastError();
}

template <int N, class FZ>
cudaError_t launch_lw(const CodeDev &c, const SclArgs &a, const FZ &fz, cudaStream_t s) {
    if (a.L <= 1) return launch_one<N, 1>(c, a, fz, s);
    if (a.L <= 2) return launch_one<N, 2>(c, a, fz, s);
    if (a.L <= 4) return launch_one<N, 4>(c, a, fz, s);
    if (a.L <= 8) return launch_one<N, 8>(c, a, fz, s);
    if (a.L <= 16) return launch_one<N, 16>(c, a, fz, s);
    return launch_one<N, 32>(c, a, fz, s);
}

}  // namespace scl_detail

// Reed-Muller frozen masks, also used by the host to pick a specialisation.
using scl_detail::rm_mask;

}  // namespace mpwsd
