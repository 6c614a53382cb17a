// Internal declarations shared by the translation units of libmpwsd.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mpwsd.h"

namespace mpwsd {

constexpr int kTopK = MPWSD_TOPK;
// Pattern tile of the tensor-core scoring kernel (the MMA N): 256 patterns
// for n = 64 (one 128 x 256 x 16 MMA chain per row block), 128 for n = 128
// (shared memory holds fewer, twice-as-deep tiles).
__host__ __device__ constexpr int tc_patterns_per_tile(int n) { return n == 64 ? 256 : 128; }
// The tensor-core epilogue keeps candidate groups of kGroupCols consecutive
// patterns (group g: patterns 8g .. 8g + 7); resolve_groups_kernel scores their
// patterns exactly and leaves the argmin pattern.
constexpr int kGroupCols = 8;
constexpr int kGridShift = 19;            // y is read on the 2^-19 grid
constexpr int kGridMax = (1 << 23) - 1;   // |round(y 2^19)| <= 2^23 - 1
// Margin of the near-tie re-rank: every approximate score is within
// kEpsScale * ||y||_1 of the exact one (bf16 hi+lo split: 2^-16 ||y||_1;
// FP32 accumulation: < 2^-18 ||y||_1 for the kernels here), so any pattern
// whose approximate score is within 2 eps of the approximate minimum may be
// the exact minimum and is re-scored exactly.
constexpr float kEpsScale = 1.0f / 16384.0f;  // 2^-14

// Trajectory state bits
constexpr uint32_t kTrajHopsMask = 0xffu;
constexpr uint32_t kTrajRescan = 1u << 8;
constexpr uint32_t kTrajValid = 1u << 9;
constexpr uint32_t kTrajRetired = 1u << 10;  // dropped as the twin of a lower-numbered trajectory

// Device-side counters (accumulated by the kernels; read by mpwsd_stats_get).
struct DevStats {
    unsigned long long frames;
    unsigned long long stage2_frames;
    unsigned long long trajectories;
    unsigned long long pattern_evals;
    unsigned long long rerank_candidates;
    unsigned long long rescans;
    unsigned long long hops;
    unsigned long long error;  // nonzero after a bounded device wait gave up
};

// Continuous stage-2 batching: a pool of frame slots that many submissions
// share. A failing frame of a submission takes a free slot; its L trajectories
// join the rows every pool step scores, whichever submission they came from
// and however many iterations they have done. A trajectory ends when it stops,
// reaches T hops or is retired as a twin; when the last one of a slot ends, the
// step's final pass writes the frame's result where the submission asked and
// frees the slot. All pointers are null in a one-batch decode.
struct PoolDev {
    int cap = 0;                   // slots
    int T = 0;                     // iterations (hops) per trajectory at most
    int *ctr = nullptr;            // kPool* counters below
    int *free_ring = nullptr;      // cap: free slot ids, popped at ctr[kPoolPop], pushed at ctr[kPoolPush]
    int *live = nullptr;           // cap: trajectories of the slot still running
    int *completed = nullptr;      // cap: slots whose last trajectory ended in this step
    unsigned long long *dst = nullptr;  // cap x 3: addresses of the frame's codeword, flags and done entry
    float *slot_y = nullptr;       // cap x n: the frame's y (read by the exact re-rank and the rescan)
};
constexpr int kPoolPop = 0, kPoolPush = 1, kPoolSteps = 2, kPoolCompleted = 3, kPoolFinished = 4;

// Per-decode device scratch. All arrays are sized for (max_B, max_L).
struct Workspace {
    int64_t max_B = 0;
    int max_L = 0;
    int device = -1;
    void *base = nullptr;       // one cudaMalloc holding everything below
    size_t bytes = 0;
    int *counters = nullptr;    // [0] = failing frames F, [1 + i] = active rows before iteration i (i <= T), [32 + i] = rescan rows in iteration i
    int *slot_frame = nullptr;  // F: frame index of each failing-frame slot
    float *slot_l1 = nullptr;   // F: ||y||_1 of the frame
    uint32_t *slot_yhl = nullptr;  // F x n: y of the frame as bf16 hi / lo parts (n/2 words each, two per word)
    uint64_t *traj_cw = nullptr;  // F*L x W: trajectory centres
    double *traj_D = nullptr;     // F*L: -sum_j y_j x_j (ED = ||y||^2 + n + 2 D)
    uint32_t *traj_state = nullptr;  // F*L: hops | rescan | valid
    int *act[2] = {nullptr, nullptr};  // active trajectory lists (ping-pong)
    int *rescan_rows = nullptr;   // rows whose top-K overflowed the margin
    float *topk_val = nullptr;    // F*L x K
    int *topk_idx = nullptr;      // F*L x K
    // pattern-split of the tensor-core scoring kernel (absent: no split)
    float *split_val = nullptr;   // kSplitItemsPerSm * num_sms items x 256 rows x K partial lists
    int *split_idx = nullptr;
    int *unit_done = nullptr;     // per 256-row unit: chunks finished in the current launch
    PoolDev pool;                 // continuous batching (null: one-batch decode)
};

// Work items of the split: at most this many per SM (units x chunks < 4 x SMs).
constexpr int kSplitItemsPerSm = 4;

// Everything the kernels need to know about a loaded code.
struct CodeDev {
    int n = 0, W = 0, m = 0, k = 0, k_info = 0, crc_len = 0;
    uint32_t crc_poly = 0;
    int64_t P = 0;
    uint64_t frozen_lo = 0, frozen_hi = 0;
    int rm_spec = 0;              // 0 = generic frozen set, else a compiled Reed-Muller specialisation id
    bool trailing_frozen = false; // a frozen leaf follows the last information leaf
    int w_max = 0;                // largest pattern weight
    int wq_max = 0;               // support words per pattern (4 indices per word)
    bool supp_dense = false;      // every pattern has weight 4 wq_max: no padding entries
    // device arrays
    uint64_t *pat_bits = nullptr;   // P x W
    uint32_t *pat_supp = nullptr;   // P x wq_max, 4 uint8 indices per word, padded with index n
    uint16_t *pat_tiles = nullptr;  // tiles of tc_patterns_per_tile(n) x n bf16, smem image (128B swizzle, K-major)
    int64_t n_tiles = 0;
    uint64_t *crc_masks = nullptr;  // crc_len x W, codeword domain: syndrome bit b = parity(c & mask_b)
    uint64_t *gen_rows = nullptr;   // k x W: generator rows (Arikan rows at the non-frozen indices, ascending)
    // OSD row sets of at most kOsdMaxOrder rows in candidate-number order (by size, then
    // lexicographic): rows at 5 bits each from bit 0, the size in bits 20..22; k <= 32 only
    uint32_t *osd_sets = nullptr;
    // Flat structure of the pattern set (MPWSD_SCORE_FLATS; n_flat = 0: none).
    // Every pattern is a coset a + V of a linear subspace V of F_2^m (a position
    // j read as the m-bit vector of its binary digits) whose orthogonal
    // complement has dimension flat_kd (1 or 2); one entry per complement D:
    // flat_w[e] = w1 | w2 << 8 | (w1 ^ w2) << 16 for a basis w1, w2 of D (w2 = 0
    // when kd = 1); flat_idx[4 e + c1 + 2 c2] = the pattern that is the coset
    // with w1.a = c1, w2.a = c2 (every coset of every entry is present).
    uint32_t *flat_w = nullptr;
    int32_t *flat_idx = nullptr;
    int n_flat = 0;
    int flat_kd = 0;
    DevStats *stats = nullptr;
    int num_sms = 0;
    // Bounded device waits: a wait that exceeds this records an error and the
    // kernel exits cleanly. test_stall (set from MPWSD_TEST_TC_STALL when the
    // code is loaded, tests only) makes the tensor-core kernel's producer issue
    // no copies, so its consumers' waits run out on purpose.
    unsigned long long wait_limit_ns = 2000000000ull;
    int test_stall = 0;
    int split_items = 0;  // MPWSD_TUNE_SPLIT_ITEMS (0: no pattern split)
    int tc_shape = 0;     // MPWSD_TUNE_TC_SHAPE: instantiated shape of the tensor-core scoring kernel
};

struct SclArgs {
    const float *y;      // frame f of this launch at y + f n; cw_out, flags_out indexed the same way
    int64_t B;
    int64_t f0;          // decode: index of this launch's frame 0 in the whole batch (slot_frame)
    int L;
    int write_yhl;       // decode: also store each failing frame's y as bf16 hi / lo (tensor-core scoring)
    int mode;            // 0 = decode (CRC + compaction), 1 = list output
    int rule;            // MPWSD_RULE_*
    int use_crc;         // stage-1 early exit enabled
    // decode mode
    uint64_t *cw_out;
    uint16_t *flags_out;
    int32_t *done_out;   // pool mode: done entry of frame f (nullable)
    int submit_id;       // pool mode: frames that pass stage 1 get done = -(submit_id + 1)
    Workspace ws;
    // list mode
    uint64_t *list_cw;
    int64_t *list_pm;
};

struct OsdArgs {
    const float *y;      // as in SclArgs
    int64_t B;
    int64_t f0;
    int L;
    int order;
    int ncand;           // osd_candidates(k, order)
    int mode;            // 0 = decode (CRC + compaction), 1 = list output
    int rule;            // MPWSD_RULE_*
    int use_crc;
    int write_yhl;
    uint64_t *cw_out;
    uint16_t *flags_out;
    int32_t *done_out;   // as in SclArgs
    int submit_id;
    Workspace ws;
    uint64_t *list_cw;
    int64_t *list_d;
};

struct ScoreArgs {
    const float *y;
    const int *rows;          // active list: trajectory ids (decode) or row ids (direct)
    const int *n_rows_dev;    // device count of rows (nullptr: use n_rows)
    int64_t n_rows;
    const uint64_t *cw;       // centre of trajectory id t at cw + t*W
    const int *slot_frame;    // frame of trajectory id t = slot_frame[t / L] (decode) ...
    const int32_t *row_frame; // ... or frame of row r = row_frame[r] (direct)
    int L;
    // tensor-core scoring: y of each slot (decode: trajectory t is in slot t / L;
    // direct: row r reads slot row_frame[r]) as bf16 hi / lo words, and ||y||_1
    const uint32_t *yhl;
    const float *l1;
    float *topk_val;          // row-indexed: the kept (value, index) list of each row
    int *topk_idx;
    unsigned long long *evals; // stats counter (may be null)
    // split buffers (both modes; nullptr: every CTA scans whole units)
    float *split_val;
    int *split_idx;
    int *unit_done;
    int split_items;  // target work items of the split (<= kSplitItemsPerSm / 2 x SMs)
};

// Launchers (return cudaError_t of the launch).
cudaError_t launch_scl(const CodeDev &c, const SclArgs &a, cudaStream_t s);
constexpr int kOsdMaxOrder = 4;
// number of OSD(order) candidates: sum_{w <= order} C(k, w)
inline int osd_candidates(int k, int order) {
    long long tot = 0, cw = 1;
    for (int w = 0; w <= order && w <= k; ++w) {
        tot += cw;
        cw = cw * (k - w) / (w + 1);
    }
    return (int)tot;
}
cudaError_t launch_osd(const CodeDev &c, const OsdArgs &a, cudaStream_t s);
cudaError_t launch_score_fp32(const CodeDev &c, const ScoreArgs &a, cudaStream_t s);
// Exact scoring of a flat pattern set by Walsh-Hadamard coefficients (score_flats.cu)
cudaError_t launch_score_flats(const CodeDev &c, const ScoreArgs &a, cudaStream_t s);
cudaError_t launch_score_tc(const CodeDev &c, const ScoreArgs &a, cudaStream_t s);
// exact argmin pattern of each row from the candidate groups launch_score_tc keeps;
// with a workspace (a decode's iteration `iter`), the hop decision of each row
// as well (in place of launch_hop), the lists left unwritten
cudaError_t launch_resolve_groups(const CodeDev &c, const ScoreArgs &a, const Workspace *ws, int iter,
                                  cudaStream_t s);
// y (B x n) -> bf16 hi / lo words and ||y||_1 per frame, for direct-mode tensor-core scoring
cudaError_t launch_split_prep(const CodeDev &c, const float *y, int64_t B, uint32_t *yhl, float *l1, cudaStream_t s);
bool score_tc_supported(const CodeDev &c);
// Shapes of the tensor-core scoring kernel (MPWSD_TUNE_TC_SHAPE): 0 is the
// default of each code length, the others are compiled in score_tc_alt.cu.
constexpr int kTcShapes = 4;
bool tc_shape_valid(int n, int shape);
cudaError_t launch_score_tc_alt(const CodeDev &c, const ScoreArgs &a, cudaStream_t s);
int rm_specialisation(int n, uint64_t lo, uint64_t hi);
cudaError_t launch_hop(const CodeDev &c, const Workspace &ws, int iter, int L, const float *y, cudaStream_t s);
cudaError_t launch_rescan(const CodeDev &c, const Workspace &ws, int iter, int L, const float *y, cudaStream_t s);
cudaError_t launch_dedup(const CodeDev &c, const Workspace &ws, int iter, int L, cudaStream_t s);
cudaError_t launch_final(const CodeDev &c, const Workspace &ws, int L, int T, int64_t B, uint64_t *cw_out, uint16_t *flags_out,
                         cudaStream_t s);
// pool mode: final select of the slots completed in this step, their release,
// and the step's bookkeeping (rows of the next step, counters, statistics)
cudaError_t launch_pool_final(const CodeDev &c, const Workspace &ws, int L, cudaStream_t s);
cudaError_t launch_pool_end(const CodeDev &c, const Workspace &ws, cudaStream_t s);

}  // namespace mpwsd
