/*
 * mpwsd.h -- C ABI of libmpwsd, a GB300 (sm_103a) implementation of two-stage
 * near-ML decoding with multipoint code-weight sphere decoding (MP-WSD),
 * arXiv 2602.08501.
 *
 * The decoder has two stages (Sec. III):
 *   stage 1  CRC-aided SC-list decoding of every frame; the most reliable
 *            candidate is checked by the CRC and, if it passes, is the output
 *            (Sec. III-A);
 *   stage 2  for the frames that fail, every list entry is an anchor; each
 *            (frame, anchor) trajectory repeatedly moves to the best codeword
 *            of its code-weight sphere S_r(c) = c xor S_r(0) (Eqs. (2)-(4)),
 *            found by scoring every precomputed low-weight pattern p with the
 *            correlation gain of Eq. (5), and stops when nothing strictly
 *            improves or after T iterations; the frame's output is the
 *            trajectory end point of smallest Euclidean distance
 *            (Algorithm 1).
 *
 * Conventions used by every entry point:
 *   - n = 2^m with n in {32, 64, 128}; W = (n + 63) / 64 words per bit vector.
 *   - Bit vectors (codewords, patterns) are packed little-endian: bit j of
 *     word j / 64 is position j.
 *   - The code is the Arikan form c = u [[1,0],[1,1]]^{(x)m} restricted to
 *     the non-frozen rows (Reed-Muller codes are the frozen sets that keep
 *     rows of weight >= 2^(m-r)).
 *   - Received samples y are FP32. Stage 1 and every exact comparison work on
 *     the integer image round(y * 2^19) clamped to +-(2^23 - 1); inputs that
 *     are already multiples of 2^-19 with |y| < 16 are used exactly.
 *   - "device" pointers are CUDA device memory of the device that was current
 *     when the code handle was created; "host" pointers are ordinary memory.
 *     The caller owns every buffer it passes; the library never keeps a
 *     caller pointer after the call returns (asynchronous work on a stream
 *     reads/writes the caller's device buffers until the stream reaches it).
 *   - Every function returns an int status (0 = MPWSD_OK, < 0 = error) and
 *     never aborts or exits. mpwsd_last_error() gives a message for the
 *     calling thread's most recent failure.
 */
#ifndef MPWSD_H
#define MPWSD_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define MPWSD_API __attribute__((visibility("default")))
#else
#define MPWSD_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define MPWSD_OK 0
#define MPWSD_EINVAL (-1)       /* an argument is out of range or inconsistent */
#define MPWSD_ENOMEM (-2)       /* a device or host allocation failed; handles stay usable */
#define MPWSD_ECUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define MPWSD_ETIMEOUT (-4)     /* a bounded device-side wait gave up (see mpwsd_sync) */
#define MPWSD_EUNSUPPORTED (-5) /* valid request this build does not implement */

/* ---- limits ------------------------------------------------------------- */
#define MPWSD_MAX_L 32          /* list size / anchors per frame */
#define MPWSD_MAX_T 15          /* stage-2 iterations (J of Algorithm 1) */
#define MPWSD_TOPK 4            /* candidates kept per trajectory by the scoring kernels */

/* ---- options ------------------------------------------------------------ */
#define MPWSD_SCORE_BF16X2 0    /* tcgen05 tensor cores, y split into bf16 hi + lo, FP32 accumulate; the
                                   kernel keeps candidate groups of 8 consecutive patterns, and a second
                                   kernel scores their patterns exactly (integers on the 2^-19 grid) */
#define MPWSD_SCORE_FP32 1      /* FP32 CUDA cores, sparse gather-add over each pattern's support */
#define MPWSD_SCORE_FLATS 2     /* exact integer scores from Walsh-Hadamard coefficients, for pattern sets made
                                   of all cosets of subspaces whose complements have dimension 1 or 2 (the
                                   minimum-weight codewords of RM(1, m) and RM(2, m)); MPWSD_EUNSUPPORTED
                                   for other pattern sets */

#define MPWSD_RULE_TOP1 0       /* stage 1 succeeds iff the best-metric list entry passes the CRC (Sec. III-A) */
#define MPWSD_RULE_ANY 1        /* stage 1 succeeds with the best-metric entry that passes the CRC */

#define MPWSD_STAGE1_SCL 0      /* stage 1 = min-sum SC-list decoding (Sec. III-A) */
#define MPWSD_STAGE1_OSD 1      /* stage 1 = ordered-statistics decoding OSD(osd_order), the anchors of the RM
                                   experiment (Sec. IV-A); needs k <= 32 */
#define MPWSD_MAX_OSD_ORDER 4

/* Output flag bits (one uint16 per frame). */
#define MPWSD_FLAG_STAGE2 0x0001u   /* stage 2 ran for this frame */
#define MPWSD_FLAG_CRC_OK 0x0002u   /* the output codeword passes the CRC */
#define MPWSD_FLAG_RESCAN 0x0004u   /* some trajectory needed a full FP64 rescan (near-tie overflow) */
#define MPWSD_FLAG_ITERS_SHIFT 4    /* bits 4..7: stage-2 iterations used (0 if stage 2 did not run) */
#define MPWSD_FLAG_ERROR 0x0100u    /* a device-side wait timed out; the frame's output is not valid */

typedef struct mpwsd_opts {
    int score_mode;  /* MPWSD_SCORE_BF16X2 (default), MPWSD_SCORE_FP32 or MPWSD_SCORE_FLATS */
    int stage1_rule; /* MPWSD_RULE_TOP1 (default) or MPWSD_RULE_ANY */
    int always_on;   /* nonzero: run stage 2 on every frame, CRC or not (always-on mode, Sec. III-C) */
    int use_graph;   /* nonzero: replay the decode's launch sequence as a CUDA graph. The first call with a
                        given (workspace, buffers, B, L, T, options) captures it (on a private stream,
                        without running it) and later identical calls replay it; the handle keeps up to
                        256 graphs. Same results as without. */
    int stage1;      /* MPWSD_STAGE1_SCL (default) or MPWSD_STAGE1_OSD */
    int osd_order;   /* OSD reprocessing order, 0..MPWSD_MAX_OSD_ORDER (MPWSD_STAGE1_OSD only) */
    int reserved[2]; /* must be zero */
} mpwsd_opts;

/* Counters accumulated on the device by every decode of a code handle since
 * the last mpwsd_stats_reset. */
typedef struct mpwsd_stats {
    int64_t frames;            /* frames decoded */
    int64_t stage2_frames;     /* frames that ran stage 2 (P_act = stage2_frames / frames, Eq. (7)) */
    int64_t trajectories;      /* (frame, anchor) trajectories started */
    int64_t pattern_evals;     /* (active trajectory, pattern) pairs scored, over all iterations; a
                                  trajectory that hops onto the centre of a live lower-numbered one of
                                  its frame is retired (same outputs) and no longer scored */
    int64_t rerank_candidates; /* candidates re-scored exactly in FP64 */
    int64_t rescans;           /* trajectories that needed a full FP64 rescan */
    int64_t hops;              /* strict-improvement moves taken */
    int64_t kernel_launches;   /* kernels launched by the library (host-side count) */
} mpwsd_stats;

typedef struct mpwsd_code mpwsd_code;           /* opaque, owned by the library */
typedef struct mpwsd_workspace mpwsd_workspace; /* opaque, owned by the library */
typedef struct mpwsd_pool mpwsd_pool;           /* opaque, owned by the library */

/* Human-readable name of a status code (static storage). */
MPWSD_API const char *mpwsd_strerror(int status);

/* Message describing the calling thread's most recent failed call ("" if none). */
MPWSD_API const char *mpwsd_last_error(void);

/*
 * mpwsd_load_code -- validate a code and its move-pattern set and upload them.
 * Code model: Sec. II-B (c = mG, CRC precoding v = [m, crc(m)]); pattern set:
 * the code-weight sphere S_r(0) without 0, Sec. II-C Eqs. (1)-(3).
 *
 *   n           code length, 32, 64 or 128.
 *   G           host, k x n bytes (0/1), or NULL. If given it must equal the
 *               rows of [[1,0],[1,1]]^{(x)m} at the non-frozen indices in
 *               ascending order; the library uses only the frozen set.
 *   frozen      host, n bytes, 1 = frozen (u_i = 0), 0 = information.
 *   k_info      message bits; k = #non-frozen = k_info + crc_len.
 *   crc_poly    CRC generator without its leading term: g(x) = x^crc_len +
 *               sum_b bit_b(crc_poly) x^b (x^6 + x^5 + 1 -> 0x21). The CRC is
 *               the remainder of m(x) x^crc_len mod g(x), message bit 0 the
 *               highest power, zero initial value, no reflection, no final XOR;
 *               v = [m_0..m_{k_info-1}, r_0..r_{crc_len-1}] fills the
 *               information indices in ascending order.
 *   crc_len     0..32; 0 = no CRC (stage 2 then runs on every frame).
 *   patterns    host, n_patterns x W words: nonzero, distinct codewords. Their
 *               order is the tie-break order of stage 2 (lower index wins).
 *   n_patterns  1 .. 2^31 - 1.
 *   out         receives the handle.
 *
 * Returns MPWSD_EINVAL if G does not match the frozen set, if a pattern is 0,
 * not a codeword, or repeated, or if k_info + crc_len != k; MPWSD_ENOMEM if
 * device memory runs out; MPWSD_ECUDA on a CUDA failure. The inputs are
 * copied; the caller may free them when the call returns. Synchronous.
 */
MPWSD_API int mpwsd_load_code(int n, const uint8_t *G, const uint8_t *frozen, int k_info, uint32_t crc_poly, int crc_len,
                    const uint64_t *patterns, int64_t n_patterns, mpwsd_code **out);

/* Release a code handle and everything it owns (waits for the device). NULL is a no-op. */
MPWSD_API void mpwsd_free_code(mpwsd_code *code);

/* Code parameters as loaded: any pointer may be NULL. */
MPWSD_API int mpwsd_code_info(const mpwsd_code *code, int *n, int *k, int64_t *n_patterns, int *max_pattern_weight);

/*
 * mpwsd_decode -- two-stage decode of B frames (Sec. III, Algorithm 1).
 *
 *   y_dev     device, B x n FP32, row-major (frame f at y_dev + f*n).
 *   B         frames, >= 0 (0 launches nothing).
 *   L         list size of stage 1 = anchors of stage 2, 1..MPWSD_MAX_L.
 *   T         stage-2 iterations J, 1..MPWSD_MAX_T.
 *   opts      NULL for defaults (BF16X2 scoring, TOP1 rule, CRC gating).
 *   cw_dev    device, B x W uint64: decoded codewords (written asynchronously).
 *   flags_dev device, B uint16: MPWSD_FLAG_* bits per frame.
 *   stream    cudaStream_t (NULL = legacy default stream); all work is
 *             enqueued on it and the call returns without waiting.
 *
 * Arguments are checked before anything is enqueued (MPWSD_EINVAL). Uses the
 * handle's internal workspace, grown on demand with cudaMalloc (a growth
 * waits for the device); concurrent calls on one handle must be serialised
 * by the caller -- use mpwsd_decode_ws with one workspace per caller instead.
 * A device-side timeout is reported by MPWSD_FLAG_ERROR on the affected
 * frames and by the next mpwsd_sync.
 */
MPWSD_API int mpwsd_decode(mpwsd_code *code, const float *y_dev, int64_t B, int L, int T, const mpwsd_opts *opts,
                 uint64_t *cw_dev, uint16_t *flags_dev, void *stream);

/*
 * mpwsd_decode_host -- mpwsd_decode on HOST buffers: the copies to and from the
 * device are part of the call and overlap the decode. The paper has no
 * counterpart: this is an interface of the library.
 *
 *   y_host     host, B x n FP32, row-major; page-locked (cudaHostAlloc /
 *              cudaHostRegister) for the copies to overlap, and required to be
 *              page-locked when opts->use_graph is set.
 *   cw_host    host, B x W uint64: decoded codewords.
 *   flags_host host, B uint16: MPWSD_FLAG_* bits per frame.
 *   B, L, T, opts, stream as in mpwsd_decode.
 *
 * The batch is cut into up to 8 chunks of at least 65,536 frames. Chunk i is
 * copied to the device on a second stream of the handle while stage 1 runs on
 * chunk i - 1 (stage 1 of a chunk waits for its copy); stage 2 then runs on
 * the whole batch, and the results are copied back on `stream`. Everything is
 * enqueued and the call returns without waiting: the host buffers must stay
 * valid, and the results are there once `stream` has been synchronised. Uses
 * the handle's internal workspace and device staging buffers for y (two,
 * used by turns: without use_graph the input copies of a call run while the
 * stage 2 of the call before it, on the other buffer, still runs), cw and
 * flags (grown on demand with cudaMalloc; a growth waits for the device);
 * concurrent calls on one handle must be serialised by the caller. Errors as
 * in mpwsd_decode.
 */
MPWSD_API int mpwsd_decode_host(mpwsd_code *code, const float *y_host, int64_t B, int L, int T,
                                const mpwsd_opts *opts, uint64_t *cw_host, uint16_t *flags_host, void *stream);

/*
 * mpwsd_workspace_create -- device scratch for decodes of up to max_B frames
 * with lists of up to max_L. One workspace may be used by one stream at a
 * time; several workspaces let several streams decode concurrently with one
 * code handle (continuous batching). MPWSD_ENOMEM when device memory is
 * short (the admission-refusal signal of a serving loop).
 */
MPWSD_API int mpwsd_workspace_create(const mpwsd_code *code, int64_t max_B, int max_L, mpwsd_workspace **out);

/* Release a workspace (waits for the device). NULL is a no-op. */
MPWSD_API void mpwsd_workspace_free(mpwsd_workspace *ws);

/* Bytes of device memory a workspace for (max_B, max_L) takes (no allocation). */
MPWSD_API int mpwsd_workspace_bytes(const mpwsd_code *code, int64_t max_B, int max_L, size_t *bytes);

/* mpwsd_decode with a caller-provided workspace (B <= its max_B, L <= its max_L). */
MPWSD_API int mpwsd_decode_ws(mpwsd_code *code, mpwsd_workspace *ws, const float *y_dev, int64_t B, int L, int T,
                    const mpwsd_opts *opts, uint64_t *cw_dev, uint16_t *flags_dev, void *stream);

/*
 * Continuous stage-2 batching (pools). Algorithm 1 (Sec. III-B) treats each
 * trajectory on its own, and each iteration of its loop depends only on the
 * trajectory's current centre, so trajectories of frames that arrived at
 * different times can share one scoring pass. A pool holds the stage-2 state
 * of one code between calls: mpwsd_pool_submit runs stage 1 (Sec. III-A) on a
 * batch, writes the frames that pass the CRC at once, and adds the L
 * trajectories of every failing frame to the pool's rows; mpwsd_pool_step runs
 * one iteration of Algorithm 1 on all rows of the pool (score every pattern,
 * exact re-rank, strict-improvement hop, twin retirement), then, for each frame
 * whose trajectories have all ended (stopped, made T hops, or retired), the
 * final choice of Algorithm 1 (smallest ED, lowest anchor on ties) into that
 * frame's output entries, and frees its slot. Every result equals what
 * mpwsd_decode returns for the frame, whatever it was batched with.
 * The paper has no counterpart for the pool itself: it is an interface of the
 * library for serving.
 *
 * Calls on one pool must be ordered on the device (one stream, or events);
 * the pool's device state is read and written by every call. Several pools
 * (one per code, or several per code) can run on different streams at once.
 */

/*
 * mpwsd_pool_create -- a pool of max_frames frame slots for lists of L anchors
 * and at most T iterations. opts as in mpwsd_decode (scoring form, stage-1
 * rule and kind, always-on; use_graph records the step's launches into a CUDA
 * graph on the first step and replays it). One cudaMalloc holds everything;
 * MPWSD_ENOMEM when device memory is short.
 */
MPWSD_API int mpwsd_pool_create(mpwsd_code *code, int64_t max_frames, int L, int T, const mpwsd_opts *opts,
                                mpwsd_pool **out);

/* Release a pool (waits for the device). NULL is a no-op. */
MPWSD_API void mpwsd_pool_free(mpwsd_pool *pool);

/* Bytes of device memory a pool of (max_frames, L) takes (no allocation). */
MPWSD_API int mpwsd_pool_bytes(const mpwsd_code *code, int64_t max_frames, int L, size_t *bytes);

/*
 * mpwsd_pool_free_frames -- how many frames the next submission may carry. A
 * submission's frames have all finished T steps after it, so the pool counts
 * every frame of the submissions of the last T steps as in flight (whether or
 * not it passed stage 1); no device read-back is involved.
 */
MPWSD_API int mpwsd_pool_free_frames(const mpwsd_pool *pool, int64_t *frames);

/*
 * mpwsd_pool_submit -- stage 1 on B frames; their trajectories join the pool.
 *
 *   y_dev      device, B x n FP32 (read by this call's stage-1 kernel only: it
 *              may be overwritten once the stream has passed this call).
 *   cw_dev     device, B x W uint64; flags_dev device, B uint16: each frame's
 *              result, written by this call (stage-1 frames) or by the step in
 *              which the frame finishes. They must stay valid until then.
 *   done_dev   device, B int32, or NULL: for each frame, when it finished --
 *              -(s + 1) for a frame that passed stage 1 in submission s (the
 *              pool's submissions numbered from 0), or k >= 1 for a frame that
 *              finished in the pool's k-th step.
 * MPWSD_ENOMEM (nothing launched) when B exceeds mpwsd_pool_free_frames.
 * Asynchronous on `stream`.
 */
MPWSD_API int mpwsd_pool_submit(mpwsd_pool *pool, const float *y_dev, int64_t B, uint64_t *cw_dev, uint16_t *flags_dev,
                                int32_t *done_dev, void *stream);

/*
 * mpwsd_pool_step -- one iteration of Algorithm 1 on every row of the pool,
 * then the final choice for the frames that finished in it (see above). A
 * step with no rows launches the same kernels, which find nothing to do.
 * Asynchronous on `stream`.
 */
MPWSD_API int mpwsd_pool_step(mpwsd_pool *pool, void *stream);

/*
 * mpwsd_decode_noalloc -- mpwsd_decode for callers that cannot allocate device
 * memory when they decode. The paper has no counterpart: this is an interface
 * of the library. Such callers include serving threads that must not call an
 * allocator once warmed up (an allocation can block or fail at an arbitrary
 * moment), and hosts whose device memory belongs to an allocator that the
 * library must not bypass (a framework's pool that owns the GPU's memory).
 *
 * Same arguments and results as mpwsd_decode; the caller still provides y_dev,
 * cw_dev and flags_dev. The scratch is one fixed 4 MiB array in device memory
 * that every GPU loading the library keeps until the process exits; this
 * entry point never calls cudaMalloc, cudaFree or any allocating routine.
 *  - Capacity: a call needs 4n + 8 bytes per frame and 8W + 56 bytes per
 *    trajectory (W = n/64 words per codeword), each array rounded up to 256
 *    bytes, plus 256 bytes of counters. So 4 MiB holds about
 *    4 MiB / (4n + 8 + L (8W + 56)) frames: about 5,400 frames (43,000
 *    trajectories B*L) for n = 64, L = 8; about 2,500 frames (40,000
 *    trajectories) for n = 128, L = 16. Larger requests return MPWSD_EINVAL
 *    with the sizes in mpwsd_last_error().
 *  - Speed: the scratch holds no room for the pattern split of the
 *    tensor-core scoring kernel (MPWSD_TUNE_SPLIT_ITEMS), so small batches
 *    score without it and can run slower than through mpwsd_decode; the
 *    results are identical.
 *  - Set-up: the first call on each device (with that device current) looks
 *    up the array's device address (cudaGetSymbolAddress, not an allocation)
 *    and keeps it for later calls.
 *  - Sharing: every call on a device uses the same array and finds the
 *    previous call's contents in it (the counters it needs zeroed are cleared
 *    on the stream). Calls whose work overlaps on the GPU, on any stream or
 *    code handle, race on the array: serialise them.
 *  - MPWSD_EINVAL while mpwsd_profile_begin is active on the handle (kernel
 *    timing creates CUDA events).
 */
MPWSD_API int mpwsd_decode_noalloc(mpwsd_code *code, const float *y_dev, int64_t B, int L, int T,
                                   const mpwsd_opts *opts, uint64_t *cw_dev, uint16_t *flags_dev, void *stream);

/*
 * mpwsd_stage1_list -- stage 1 alone (Sec. III-A): min-sum SC-list decoding
 * of B frames, returning the whole final list in order (best metric first).
 *
 *   list_cw_dev  device, B x L x W uint64: candidate codewords.
 *   list_pm_dev  device, B x L int64: path metrics in units of 2^-19.
 * Entries past the list size min(L, 2^k) are not written. Asynchronous.
 */
MPWSD_API int mpwsd_stage1_list(mpwsd_code *code, const float *y_dev, int64_t B, int L, uint64_t *list_cw_dev,
                      int64_t *list_pm_dev, void *stream);

/*
 * mpwsd_osd_list -- the OSD(order) stage 1 alone: the list of the min(L, #candidates)
 * candidates of smallest discrepancy D(c) = sum_j |y_j| [c_j != hd_j] (ED order;
 * ties in the enumeration order), for B frames. Construction: hard decisions
 * hd_j = [y_j < 0]; the most reliable basis (positions by decreasing |y|, ties
 * to the lower index, kept when independent of those before); the codeword
 * that agrees with hd on it, and every codeword that differs from it on at most
 * `order` of the basis positions, enumerated by the number of flips, then
 * lexicographically by basis rank.
 *
 *   list_cw_dev  device, B x L x W uint64 codewords.
 *   list_d_dev   device, B x L int64: D in units of 2^-19.
 * Entries past the list size are not written. Needs k <= 32, 0 <= order <=
 * MPWSD_MAX_OSD_ORDER, 1 <= L <= MPWSD_MAX_L. Asynchronous.
 */
MPWSD_API int mpwsd_osd_list(mpwsd_code *code, const float *y_dev, int64_t B, int order, int L, uint64_t *list_cw_dev,
                             int64_t *list_d_dev, void *stream);

/*
 * mpwsd_score_topk -- the scoring step of stage 2 alone: for each row r,
 * the trajectory centre c_r (frame frame_dev[r] of y_dev) gets the scores
 * S(r, p) = sum_{j in supp p} y_j x_j(c_r) for every pattern p (-G/2 of
 * Eq. (5); ED(c xor p) - ED(c) = 4 S). Scores are the kernel's
 * approximations S~ (mode BF16X2 or FP32), each within eps = 2^-14 ||y||_1 of
 * the exact one. Returned, in ascending order: the MPWSD_TOPK smallest S~ among
 * the patterns with S~ <= min S~ + 2 eps, i.e. every pattern that can be the
 * exact minimum unless MPWSD_TOPK of them fill the list (then the list's last
 * value is within 2 eps of its first, which the caller reads as "rescan").
 * BF16X2 and FLATS go further and return the exact argmin: one entry, the
 * pattern of smallest exact S (lowest index among equal ones) with that S.
 * BF16X2 keeps groups of 8 consecutive patterns and scores the patterns of the
 * groups within 2 eps exactly; when four groups lie within 2 eps (a full list,
 * "rescan"), each entry is a group's smallest S~ with the group's pattern of
 * smallest exact S.
 *
 *   y_dev       device, B x n FP32.       frame_dev  device, M int32 in [0, B).
 *   cw_dev      device, M x W uint64.     M          rows, >= 0.
 *   topk_val_dev device, M x MPWSD_TOPK FP32; topk_idx_dev device, M x
 *   MPWSD_TOPK int32 (-1 in the unused tail slots).
 * Asynchronous. BF16X2 takes B*(4n + 4) bytes of stream-ordered scratch
 * (cudaMallocAsync / cudaFreeAsync on the stream) for y in split form.
 */
MPWSD_API int mpwsd_score_topk(mpwsd_code *code, int score_mode, const float *y_dev, int64_t B, const int32_t *frame_dev,
                     const uint64_t *cw_dev, int64_t M, float *topk_val_dev, int32_t *topk_idx_dev, void *stream);

/* Wait for `stream`, then report (and clear) a device-side timeout recorded
 * by earlier work of this handle: MPWSD_OK or MPWSD_ETIMEOUT. */
MPWSD_API int mpwsd_sync(mpwsd_code *code, void *stream);

/* Kernel classes for mpwsd_profile_end. */
#define MPWSD_KERNEL_SCL 0        /* stage 1: SC-list + CRC + compaction */
#define MPWSD_KERNEL_SCORE_TC 1   /* scoring, tcgen05 BF16 hi+lo */
#define MPWSD_KERNEL_SCORE_FP32 2 /* scoring, FP32 CUDA cores */
#define MPWSD_KERNEL_HOP 3        /* FP64 near-tie re-rank + hop + compaction (FP32 and FLATS scoring), and twin
                                     retirement */
#define MPWSD_KERNEL_RESCAN 4     /* full FP64 rescan of overflowing rows */
#define MPWSD_KERNEL_FINAL 5      /* per-frame argmin ED + flags */
#define MPWSD_KERNEL_OSD 6        /* stage 1 by OSD(order) + CRC + compaction */
#define MPWSD_KERNEL_SCORE_FLATS 7 /* scoring, exact Walsh-Hadamard coset sums (MPWSD_SCORE_FLATS) */
#define MPWSD_KERNEL_RESOLVE 8    /* exact argmin inside the candidate groups of the tcgen05 scoring; in a
                                     decode also the re-rank decision, hop and compaction of each row */
#define MPWSD_KERNEL_KINDS 9

typedef struct mpwsd_kernel_time {
    int64_t launches; /* kernels of this class launched while profiling */
    double ms;        /* summed device time between CUDA events recorded around each launch */
} mpwsd_kernel_time;

/* mpwsd_profile_begin: from now on, record a CUDA event pair on the launch
 * stream around every kernel this handle launches (a few microseconds of
 * overhead per launch). mpwsd_profile_end: wait for those events, write the
 * per-class launch counts and summed durations to out[MPWSD_KERNEL_KINDS],
 * and stop recording. */
MPWSD_API int mpwsd_profile_begin(mpwsd_code *code);
MPWSD_API int mpwsd_profile_end(mpwsd_code *code, mpwsd_kernel_time *out);

/* Tunable launch parameters of a code handle (set by the autotuner in
 * paper_2602_08501_gb300/autotune.py or by hand; they change speed only, never
 * results). */
#define MPWSD_TUNE_SPLIT_ITEMS 0 /* tensor-core scoring: when a launch has fewer 256-row units than this, each
                                    unit's pattern tiles are split into chunks scanned by different CTAs so the
                                    launch has about this many work items; 0 = never split. Default: SMs / 2 */
#define MPWSD_TUNE_TC_SHAPE 1    /* tensor-core scoring kernel shape: 0 (default) n = 64: 256-pattern tiles, two
                                    A-builder warps, two-stage tile ring; n = 128: 128-pattern tiles, two builders,
                                    two stages. 1: as 0 with four A-builder warps. n = 64 only: 2: 128-pattern
                                    tiles (two accumulators per row block alternate), two stages; 3: as 2 with a
                                    four-stage ring */
#define MPWSD_TUNE_KNOBS 2

/* Set / get a tunable (MPWSD_EINVAL for an unknown knob or a value outside its range). */
MPWSD_API int mpwsd_tune_set(mpwsd_code *code, int knob, int value);
MPWSD_API int mpwsd_tune_get(const mpwsd_code *code, int knob, int *value);

/* Read (synchronising the device) / reset the handle's counters. */
MPWSD_API int mpwsd_stats_get(mpwsd_code *code, mpwsd_stats *out);
MPWSD_API int mpwsd_stats_reset(mpwsd_code *code);

/*
 * mpwsd_enumerate_codewords -- host helper that builds pattern sets: every
 * codeword of the code defined by `frozen` whose Hamming weight is in
 * weights[0..n_weights), in the order (weight ascending as listed in
 * `weights`, which must be ascending; then message integer ascending, where
 * the message integer reads the information bits with the lowest index as the
 * most significant bit). Brute force over all 2^k messages (k <= 40).
 * If out is NULL only *count is set; otherwise at most max_out codewords are
 * written (MPWSD_EINVAL if more exist). Host memory only; synchronous.
 */
MPWSD_API int mpwsd_enumerate_codewords(int n, const uint8_t *frozen, const int *weights, int n_weights, uint64_t *out,
                              int64_t max_out, int64_t *count);

#ifdef __cplusplus
}
#endif

#endif /* MPWSD_H */
