/*
 * polar.h -- C ABI of the GB300 (sm_103a) list-CRC polar decoder.
 *
 * Method: "Fast List Decoders for Polar Codes" (Sarkis, Giard, Vardy,
 * Thibeault, Gross). A polar code of length N = 2^n with K information
 * positions (CRC included) is decoded by successive-cancellation list
 * decoding with list size L over the Fast-SSC decoding tree: inner nodes
 * apply F (Eq. (1), min-sum), G (Eq. (2)) and Combine (Eq. (3)) to every path;
 * Rate-0, Rate-1, repetition and single-parity-check nodes are decoded
 * directly and fork paths with the metric of Eq. (9) (Sec. III); the L best
 * candidates survive each forking node (Algorithm 1); the output is the best
 * path that passes the CRC (Sec. II-B).
 *
 * Conventions shared by every entry point:
 *  - Bit order is natural: codeword x = u * G_N, G_N = F^{(x)n},
 *    F = [[1,0],[1,1]] (Fig. 1). No bit-reversal permutation.
 *  - BPSK maps bit 0 to a positive LLR: an LLR a decides 0 iff a >= 0 (Eq. (4)).
 *  - The path metric returned is the penalty P = -PM >= 0 of Sec. III-A
 *    (smaller is better); winners are chosen by argmin.
 *  - K counts the CRC bits. The payload is the first k = K - crc_len
 *    information positions in ascending index; the CRC fills the last
 *    crc_len. CRC: MSB-first division by crc_poly (normal form, e.g.
 *    0x04C11DB7 for CRC-32, 0x07 for CRC-8), register starts at 0, no
 *    reflection, no final xor (the paper does not fix these, Sec. II-B).
 *  - Payload bits are returned packed LSB-first: payload bit b is bit (b % 8)
 *    of byte b / 8 of the frame's ceil(k/8)-byte row.
 *  - float32 LLRs are used as given. int8 LLRs are saturated values in
 *    [-127, 127] (-128 is read as -127); G saturates to [-127, 127] and all
 *    penalties are exact integers.
 *  - Device pointers are CUDA device (or managed) memory of the calling
 *    process's current device; the caller owns every I/O buffer. Work is
 *    enqueued on `stream` (a cudaStream_t; NULL = legacy default stream) and
 *    runs asynchronously; an entry point returns after launching.
 *  - Every entry point returns POLAR_OK (0) or a negative status; nothing is
 *    thrown across the ABI. polar_strerror names a status.
 */
#ifndef POLAR_GB300_H
#define POLAR_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(POLAR_BUILD)
#define POLAR_API __attribute__((visibility("default")))
#else
#define POLAR_API
#endif

/* A cudaStream_t, declared without the CUDA headers. */
typedef struct CUstream_st *polar_stream_t;

/* Opaque code object: the decoding schedule and device tables of one code. */
typedef struct polar_code polar_code_t;

enum polar_status {
    POLAR_OK = 0,
    POLAR_EINVAL = -1,        /* an argument is out of range or NULL */
    POLAR_ENOMEM = -2,        /* host or device allocation failed */
    POLAR_ECUDA = -3,         /* a CUDA call failed (no device, launch error, ...) */
    POLAR_EUNSUPPORTED = -4,  /* a valid request the library does not support */
    POLAR_ETIMEDOUT = -5,     /* a bounded device or host wait ran out */
    POLAR_EBUSY = -6          /* no room right now (serving admission) */
};

enum polar_llr_dtype { POLAR_LLR_F32 = 0, POLAR_LLR_I8 = 1 };

/* polar_code_create flags. The low byte selects the node set. */
enum polar_flags {
    POLAR_SPC_MAX_4 = 0,            /* Rate-0, Rate-1, repetition, SPC of length <= 4
                                       ("Dec-SPC-4", Sec. VI) -- the default */
    POLAR_SPC_ANY = 1,              /* SPC nodes of any length, four least reliable
                                       bits ("Dec-SPC-4+", Sec. III-D, VI) */
    POLAR_NO_SPECIAL_NODES = 2,     /* length-one leaves only: unrolled SC-list
                                       (Table I, "Unrolled SC-list") */
    POLAR_HOST_ONLY = 0x100,        /* build the schedule and tables on the host
                                       only: no CUDA call, cannot decode (for
                                       inspecting schedules without a GPU) */
    POLAR_SYSTEMATIC = 0x200        /* systematic code (the encoder cited in
                                       Sec. I): payload and CRC are read from the
                                       decoded codeword x at the information
                                       positions instead of from u = x G_N */
};

/* Create a code object.
 *   N            code length, a power of two, 8 <= N <= 4096.
 *   K            information positions including the CRC, crc_len < K <= N.
 *   frozen_mask  host array of N bytes, nonzero = frozen; exactly N-K nonzero.
 *                Read during the call only.
 *   crc_len      0 (no CRC: the best path wins) or 1..32.
 *   crc_poly     generator polynomial without the x^crc_len term.
 *   L            list size, a power of two, 1 <= L <= 128 (L = 1 is Fast-SSC
 *                decoding, Sec. V, with kernels of its own: one lane per
 *                frame, or one warp per frame for batches no larger than
 *                the SM count). 2 <= L <= 32 runs the warp-per-frame kernels;
 *                L = 64 and 128 (the paper's Fig. 3 uses L = 128) run one CTA
 *                of L threads per frame over the fully unrolled schedule, with
 *                its stages in global scratch (polar_code_set_smem_budget can
 *                move the smallest on chip). Wide codes decode through
 *                polar_list_decode, polar_list_decode_host and
 *                polar_adaptive_decode; set_launch, the allocation-free entry,
 *                batch plans and servers return POLAR_EUNSUPPORTED for them.
 *   flags        one node-set value, optionally | POLAR_HOST_ONLY and/or
 *                POLAR_SYSTEMATIC.
 * Builds the decoding tree (Sec. II-D: the largest Rate-0 / Rate-1 /
 * repetition / SPC sub-tree from the root down), the unrolled operation list
 * (Listing 2) and the CRC tables, and copies them to the current device.
 * Errors: POLAR_EINVAL (bad N, K, mask, crc_len, flags, NULL out),
 * POLAR_EUNSUPPORTED (L not a power of two in 1..128), POLAR_ENOMEM,
 * POLAR_ECUDA. On error *out is set to NULL. */
POLAR_API int polar_code_create(polar_code_t **out, uint32_t N, uint32_t K, const uint8_t *frozen_mask,
                      uint32_t crc_len, uint64_t crc_poly, uint32_t L, uint32_t flags);

/* Free a code object and its device tables. The caller must make sure no
 * decode that uses it is still running (synchronise its streams first).
 * NULL is accepted. */
POLAR_API int polar_code_destroy(polar_code_t *code);

/* List-decode n_frames frames of one code (the plain, one-code-per-launch form).
 *   llr_dev          device, [n_frames][N] float32 (POLAR_LLR_F32) or int8
 *                    (POLAR_LLR_I8), row-major, read only.
 *   info_bits_dev    device, [n_frames][ceil(k/8)] bytes, written (payload of
 *                    the winning path, LSB-first).
 *   path_metric_dev  device, [n_frames] float, written (winning penalty).
 *   crc_ok_dev       device, [n_frames] bytes, 1 if the winner passed the CRC
 *                    (always 1 when crc_len = 0); may be NULL.
 *   winner_slot_dev  device, [n_frames] int32, list slot of the winner (slots
 *                    are numbered in (source slot, candidate) order after each
 *                    selection); may be NULL.
 * Re-entrant: concurrent calls on distinct streams are safe (each call takes
 * its own scratch from the stream-ordered allocator when the code needs any).
 * A call with no more frames than the device has SMs runs them with a
 * latency shape (four warps and a CTA's shared memory per frame; at L = 1 one
 * warp over the node elements) unless polar_code_set_launch fixed the shape;
 * results do not depend on the shape.
 * The call is asynchronous: it reports launch errors; an error raised while
 * its kernels run shows up in polar_sync (or the next CUDA call).
 * Errors: POLAR_EINVAL (NULL code/required pointer, bad dtype, host-only
 * code), POLAR_ENOMEM (scratch), POLAR_ECUDA (launch failure). n_frames = 0
 * is a no-op. */
POLAR_API int polar_list_decode(const polar_code_t *code, const void *llr_dev, int llr_dtype,
                      uint32_t n_frames, uint8_t *info_bits_dev, float *path_metric_dev,
                      uint8_t *crc_ok_dev, int32_t *winner_slot_dev, polar_stream_t stream);

/* A short English name for a status code (never NULL). */
POLAR_API const char *polar_strerror(int status);

/* Wait until everything enqueued on `stream` (NULL: the legacy default stream)
 * has finished, and report the errors of asynchronous work: POLAR_OK, or
 * POLAR_ECUDA when the stream or an earlier kernel on the current device
 * failed. Blocks the calling host thread. */
POLAR_API int polar_sync(polar_stream_t stream);

/* Facts about a code object (sizes, tree statistics, launch shape). */
typedef struct {
    uint32_t N, K, k, L, crc_len;
    uint32_t n_ops;          /* entries of the unrolled operation list */
    uint32_t n_leaves;       /* leaves of the decoding tree */
    uint32_t n_rate0, n_rate1, n_rep, n_spc;
    uint32_t warps_per_frame[2];     /* per dtype (index = polar_llr_dtype) */
    uint32_t frames_per_cta[2];
    uint32_t smem_per_frame[2];      /* bytes of shared memory per frame in flight */
    uint64_t scratch_per_frame[2];   /* bytes of global scratch per frame in flight */
    uint32_t spill_mask[2];          /* alpha stages kept in global scratch */
    uint32_t recomputed_stages[2];   /* alpha stages not stored: evaluated from the channel */
    uint32_t max_recompute_depth;    /* how many top stages may be (see polar_code_set_recompute) */
    uint32_t packed[2];              /* 1: the shape packs register subtrees (polar_code_set_packing) */
} polar_code_info_t;

/* Fill *info (host memory, caller-owned). Errors: POLAR_EINVAL (NULL). */
POLAR_API int polar_code_get_info(const polar_code_t *code, polar_code_info_t *info);

/* The unrolled operation list (Listing 2) as triples (kind, N_v, first u
 * index): kind 0 = F, 1 = G, 2 = Combine, 11 = Rate-0 leaf, 12 = Rate-1 leaf,
 * 13 = repetition leaf, 14 = SPC leaf. ops_out holds 3*cap int32. *n_ops gets
 * the full count; POLAR_EINVAL if cap is too small. */
POLAR_API int polar_code_schedule(const polar_code_t *code, int32_t *ops_out, uint32_t cap, uint32_t *n_ops);

/* Algorithmic operation count of one frame (the roofline numerator): one
 * operation is one element-wise min / add / compare / select / xor on one
 * LLR, bit word or key, counted along the schedule with the number of live
 * paths a noiseless frame has at each node (the list fills up to L at the
 * first forks and stays full). Pure host arithmetic. */
POLAR_API int polar_code_op_count(const polar_code_t *code, uint64_t *ops_per_frame);

/* Override the launch shape chosen at create time for one dtype (for the
 * autotuner and tests). warps_per_frame in {1,2,4}; smem_budget caps the
 * shared memory of one frame (0 = default), larger alpha stages move to
 * global scratch to meet it; cta_threads (a multiple of 32 * warps_per_frame,
 * at most 512; 0 = 128) sets how many frame groups share a CTA and run the
 * schedule in lockstep. Later decodes of that dtype keep this shape even for
 * small batches. A code with L = 1 normally runs a kernel of its own
 * (Fast-SSC decoding, one lane per frame, see polar_code_set_smem_budget);
 * after set_launch it runs the list kernels with this shape instead, until
 * polar_code_autotune or polar_code_set_smem_budget hands it back. Errors: POLAR_EINVAL (bad
 * arguments, or the shape cannot hold the code), POLAR_EUNSUPPORTED (a wide
 * code, L > 32), POLAR_ENOMEM / POLAR_ECUDA (uploading the flagged schedule). */
POLAR_API int polar_code_set_launch(polar_code_t *code, int llr_dtype, uint32_t warps_per_frame,
                                    uint32_t smem_budget, uint32_t cta_threads);

/* Shared memory for the codes whose kernels place their buffers by a budget
 * (0 = the default; results do not depend on it):
 *   - L = 1 (the Fast-SSC kernel: one lane per frame, 32 frames per warp,
 *     alpha stages interleaved over the lanes): bytes per warp (default 0:
 *     everything in global scratch, where the accesses are coalesced, the L1
 *     cache holds the hot low stages, and more warps fit per SM). The beta
 *     rows, if they fit, and then the lowest alpha stages that fit go to
 *     shared memory, the rest to global scratch. Also hands an L = 1 code
 *     back from the list kernels (after polar_code_set_launch).
 *   - wide codes (L = 64, 128: one CTA per frame): bytes per CTA beyond its
 *     tables (default 0: every buffer in global scratch, so that more CTAs
 *     fit per SM), filled with the smallest buffers (low alpha stages, left
 *     betas, the channel row); the others go to global scratch.
 * More on chip fits fewer warps or CTAs per SM; polar_code_autotune times the
 * budgets. Errors: POLAR_EINVAL (bad arguments), POLAR_EUNSUPPORTED (2 <= L
 * <= 32: those codes take polar_code_set_launch). */
POLAR_API int polar_code_set_smem_budget(polar_code_t *code, int llr_dtype, uint32_t bytes);

/* List sizes L <= 16 with one warp per frame: in rounds where every frame
 * group of a CTA holds a frame, run the register subtrees (Sec. III leaves of
 * up to 32 bits and their selection, Algorithm 1) of 32 / L frames in one
 * warp, L lanes each, while the other warps of those frames wait, and sort
 * and scan each frame's selection inside its own L lanes (on != 0); or run
 * each frame in its own warp with lane-per-path selection over the whole warp
 * (on = 0). Default: on for L <= 4, off for L = 8 and 16 (measured faster
 * each way). The choice is kept per LLR type: later shapes from
 * polar_code_set_launch use it where they allow it (one warp per frame), and
 * the batched and serving forms follow the code's choice for its frames.
 * Turning it on needs a shape with one warp per frame; frames are packed
 * only in CTAs of at least 32 / L frame groups, elsewhere the segments alone
 * apply. The rest of the current shape is kept. polar_code_autotune
 * and polar_batch_autotune (all classes on or off) try both settings. Results
 * do not depend on it. Errors: POLAR_EINVAL (bad arguments or shape),
 * POLAR_EUNSUPPORTED (a wide code), POLAR_ENOMEM / POLAR_ECUDA (uploading the
 * schedule). */
POLAR_API int polar_code_set_packing(polar_code_t *code, int llr_dtype, int on);

/* Stage memory against recomputation (Sec. IV-E counts one alpha row per
 * path and stage). The top `depth` alpha stages (at most
 * max_recompute_depth, at most 3) are not stored: an F or G that reads one
 * evaluates it from the channel row and the paths' left-sibling betas by
 * Eqs. (1)-(2), 2^depth channel values per element. That removes
 * L (2^(n-1) + ... + 2^(n-depth)) values per frame in flight from the
 * scratch working set (at (2048,1723) L = 32 f32, depth 2: 192 KB of 260 KB).
 * Only stages every node of which is an inner node qualify. Results do not
 * depend on the depth. The default is 0 (every stage stored); keeps the
 * current warps, budget and CTA size. polar_code_autotune times depths
 * 1 .. max_recompute_depth on the best fully stored shape and keeps a depth
 * only if it is faster. Errors: POLAR_EINVAL (bad
 * arguments, depth too large), POLAR_EUNSUPPORTED (a wide code),
 * POLAR_ENOMEM / POLAR_ECUDA (uploading the schedule). */
POLAR_API int polar_code_set_recompute(polar_code_t *code, int llr_dtype, uint32_t depth);

/* polar_list_decode on HOST buffers (same layouts, host pointers): the frames
 * go through the device in chunks, the copy in of one chunk and the copy out
 * of another overlapping the decode of a third (two device staging buffers,
 * two internal streams; the decodes run on `stream`). Pinned host memory
 * (cudaHostAlloc / cudaHostRegister) is needed for the copies to overlap;
 * pageable memory works but serialises them. Blocks until every output is in
 * host memory. Allocates its staging buffers with cudaMalloc and frees them
 * before returning. Errors as polar_list_decode; POLAR_EINVAL also when the
 * current device is not the code's. */
POLAR_API int polar_list_decode_host(const polar_code_t *code, const void *llr_host, int llr_dtype, uint32_t n_frames,
                                     uint8_t *info_bits_host, float *path_metric_host, uint8_t *crc_ok_host,
                                     int32_t *winner_slot_host, polar_stream_t stream);

/* Adaptive decoding (Sec. V): every frame is first decoded with `fast`
 * (normally the same code with L = 1, i.e. Fast-SSC decoding); the frames
 * whose CRC fails are then decoded again with `list` (the target L_max) and
 * their outputs replaced. Both codes must be the same code (N, K, frozen set,
 * CRC) created on the current device, and the code must have a CRC. Outputs
 * as polar_list_decode; crc_ok_dev is required (it drives the switch).
 * n_relisted_dev (device, one uint32, may be NULL) receives the number of
 * frames handed to the list decoder. Everything is enqueued on `stream`;
 * the second decode reads the failure count from device memory, so no host
 * synchronisation happens. Errors: POLAR_EINVAL (different codes, no CRC,
 * NULL pointers), POLAR_ENOMEM, POLAR_ECUDA. */
POLAR_API int polar_adaptive_decode(const polar_code_t *fast, const polar_code_t *list, const void *llr_dev,
                                    int llr_dtype, uint32_t n_frames, uint8_t *info_bits_dev, float *path_metric_dev,
                                    uint8_t *crc_ok_dev, int32_t *winner_slot_dev, uint32_t *n_relisted_dev,
                                    polar_stream_t stream);

/* Autotune the launch shape of one dtype on real frames: times every
 * distinct (warps per frame, CTA size, shared-memory budget) shape on n_frames
 * frames of llr_dev (device, [n_frames][N]) on `stream`, installs the fastest
 * and reports it (any out pointer may be NULL; *budget_out = 0 means no cap).
 * Blocks until the timing runs finish. Results of later decodes do not depend
 * on the shape (only speed does). A code with L = 1 gets its own kernel back
 * and its shared-memory budget per warp timed when the sample fills every SM
 * (otherwise the default is kept; see polar_code_set_smem_budget;
 * *warps_out = 1, *budget_out = that budget, *cta_out = the CTA's threads);
 * a wide code gets its shared-memory budget per CTA timed (*warps_out = L/32,
 * *budget_out = that budget, *cta_out = L). Errors: POLAR_EINVAL, POLAR_ENOMEM,
 * POLAR_ECUDA. */
POLAR_API int polar_code_autotune(polar_code_t *code, int llr_dtype, const void *llr_dev, uint32_t n_frames,
                                  polar_stream_t stream, uint32_t *warps_out, uint32_t *budget_out,
                                  uint32_t *cta_threads_out);

/* ---- Test hooks: host-side fault injection ----------------------------------
 * For tests of error paths and of reads of unwritten memory; they inject on
 * the host and never make the GPU fault. Process-wide settings, not meant to
 * change while decodes run on other threads.
 *   POLAR_INJECT_ALLOC_FAIL  the next `value` device allocations made by
 *                            decode calls (scratch, staging buffers) succeed
 *                            and every later one fails, so the call returns
 *                            POLAR_ENOMEM; value < 0 switches it off.
 *   POLAR_INJECT_POISON      value != 0: before every decode the global
 *                            scratch of the launch is filled with bytes no
 *                            decode writes (0xFF = float NaN, 0x80 = int8
 *                            -128), so a read of scratch that was never
 *                            written shows up as a parity failure.
 * Errors: POLAR_EINVAL for an unknown hook. */
enum polar_inject { POLAR_INJECT_ALLOC_FAIL = 1, POLAR_INJECT_POISON = 2 };
POLAR_API int polar_debug_inject(int what, int64_t value);

/* ---- Batched form --------------------------------------------------------
 * Frames of several codes (mixed N, rate and L) decoded by one persistent
 * launch. Frame f uses codes[frame_code[f]]; its LLRs start at byte
 * llr_offset[f] of one packed device buffer (rows of N_f elements in frame
 * order) and its payload at byte bits_offset[f] of one packed output buffer
 * (rows of ceil(k_f/8) bytes); polar_batch_layout reports both. Work items are
 * ordered by decreasing decode cost and taken from a device counter by the
 * frame groups of the persistent kernel, so large and small codes share the
 * GPU without one launch per code. All codes must be created on the current
 * device; the plan keeps pointers to them (destroy the plan first). The plan
 * owns its device tables and global scratch (allocated at plan / shape time,
 * so runs and graph replays allocate nothing). Results are identical to
 * polar_list_decode of each frame with its code. */
typedef struct polar_batch polar_batch_t;

typedef struct {
    uint32_t n_frames, n_codes;
    uint32_t warps_per_frame, frames_per_cta;
    uint32_t smem_per_frame;       /* bytes per frame group (largest class) */
    uint32_t grid;                 /* CTAs of the persistent launch */
    uint64_t scratch_bytes;        /* global scratch owned by the plan */
    uint64_t llr_bytes, bits_bytes;/* sizes of the packed input / output buffers */
} polar_batch_info_t;

/* frame_code: host [n_frames], values < n_codes; flags must be 0. Errors:
 * POLAR_EINVAL (bad handle, index, dtype, code on another device),
 * POLAR_ENOMEM, POLAR_ECUDA. */
POLAR_API int polar_batch_plan(polar_batch_t **out, polar_code_t *const *codes, uint32_t n_codes,
                               const uint32_t *frame_code, uint32_t n_frames, int llr_dtype, uint32_t flags);
POLAR_API int polar_batch_destroy(polar_batch_t *batch);
/* Sizes of the packed buffers and (optionally, host arrays of n_frames) the
 * per-frame byte offsets. */
POLAR_API int polar_batch_layout(const polar_batch_t *batch, uint64_t *llr_bytes, uint64_t *bits_bytes,
                                 uint64_t *llr_offsets, uint64_t *bits_offsets);
/* Enqueue the batched decode on `stream`: llr_dev (packed input), bits_dev
 * (packed payload output), pm_dev [n_frames] penalties, ok_dev / slot_dev
 * [n_frames] (may be NULL). Runs of one plan must not overlap on the GPU
 * (they share the plan's work counter and scratch). */
POLAR_API int polar_batch_run(polar_batch_t *batch, const void *llr_dev, uint8_t *bits_dev, float *pm_dev,
                              uint8_t *ok_dev, int32_t *slot_dev, polar_stream_t stream);
/* Choose warps per frame, the shared-memory budget per frame (larger alpha
 * stages go to the plan's global scratch) and the CTA size (a multiple of
 * 32 * warps_per_frame, at most 512; 0 = 128). A CTA takes one frame per group
 * at a time; groups holding frames of the same code run in lockstep. */
POLAR_API int polar_batch_set_launch(polar_batch_t *batch, uint32_t warps_per_frame, uint32_t smem_budget,
                                     uint32_t cta_threads);
/* Autotuner: times (warps per frame in {1,2}, CTA size, budget) shapes on the
 * plan's own frames (llr_dev as for polar_batch_run; bits_dev / pm_dev are
 * scratch outputs), keeps the fastest, reports it (out pointers may be NULL).
 * Blocks until done. */
POLAR_API int polar_batch_autotune(polar_batch_t *batch, const void *llr_dev, uint8_t *bits_dev, float *pm_dev,
                                   polar_stream_t stream, uint32_t *warps_out, uint32_t *budget_out,
                                   uint32_t *cta_threads_out);
/* Capture one run (counter reset + persistent launch) into a CUDA graph owned
 * by the plan, for the given buffers; `stream` must not be the legacy default
 * stream. polar_batch_replay launches that graph on any stream. A later
 * set_launch / autotune / capture drops the graph. */
POLAR_API int polar_batch_capture(polar_batch_t *batch, const void *llr_dev, uint8_t *bits_dev, float *pm_dev,
                                  uint8_t *ok_dev, int32_t *slot_dev, polar_stream_t stream);
POLAR_API int polar_batch_replay(polar_batch_t *batch, polar_stream_t stream);
POLAR_API int polar_batch_get_info(const polar_batch_t *batch, polar_batch_info_t *info);

/* ---- Serving form (continuous batching) ------------------------------------
 * A request is n_frames frames of one code, submitted from the host at any
 * time. A library-owned engine thread admits pending requests, in arrival
 * order, as device memory (an arena of device_mem_budget bytes allocated at
 * create) and frame slots (max_frames_in_flight) free up; copies their LLRs
 * to the device; and launches everything admitted as one batched launch on
 * one of three streams, while earlier batches are still running on the
 * others -- so requests that arrive while others are on the GPU join the
 * next batch and their work overlaps on the device. Results are copied back
 * and kept until polled. Results equal polar_list_decode of the same frames
 * (only timing depends on the mix). Latency = submit to results on the host. */
typedef struct polar_server polar_server_t;

typedef struct {
    uint64_t completed, frames, info_bits;        /* since the last reset */
    uint64_t pending, admitted, batches_in_flight;
    uint64_t batches, max_batches_in_flight;     /* launches so far, most launches on the GPU at once */
    double p50_us, p99_us, max_us, mean_us;       /* request latency (submit -> results on host) */
    double span_us;                               /* first submit -> last completion */
} polar_server_stats_t;

enum { POLAR_SERVER_PAUSED = 1 };   /* create with admission paused (tests) */

/* warps_per_frame 0 = 1; smem_budget 0 = default per-frame shared-memory budget
 * (7000 bytes with one warp per frame: larger stages go to scratch). */
POLAR_API int polar_server_create(polar_server_t **out, size_t device_mem_budget, uint32_t max_frames_in_flight,
                                  uint32_t warps_per_frame, uint32_t smem_budget, uint32_t flags);
/* Stops the engine after the batches in flight and frees everything; results
 * not yet polled are dropped. */
POLAR_API int polar_server_destroy(polar_server_t *server);
/* Copies the host LLRs ([n_frames][N] of llr_dtype) and queues the request.
 * POLAR_EINVAL if the request can never fit the arena / frame slots,
 * POLAR_EBUSY if the pending queue is full (retry later). */
POLAR_API int polar_server_submit(polar_server_t *server, const polar_code_t *code, const void *llr_host,
                                  int llr_dtype, uint32_t n_frames, uint64_t *ticket);
/* Non-blocking. *done = 1 and host outputs written (packed payload rows
 * [n][ceil(k/8)], penalties, CRC flags; any may be NULL) when finished; the
 * ticket is then released. */
POLAR_API int polar_server_poll(polar_server_t *server, uint64_t ticket, uint8_t *bits_host, float *pm_host,
                                uint8_t *ok_host, int *done);
/* Bounded wait for one request: POLAR_OK when done, POLAR_ETIMEDOUT after
 * timeout_ms, POLAR_ECUDA if the engine stopped on an error. */
POLAR_API int polar_server_wait(polar_server_t *server, uint64_t ticket, uint32_t timeout_ms);
/* Pause / resume admission (requests stay queued while paused). */
POLAR_API int polar_server_pause(polar_server_t *server, int paused);
/* Counters and latency percentiles; reset != 0 clears them afterwards. */
POLAR_API int polar_server_stats(polar_server_t *server, polar_server_stats_t *stats, int reset);
/* Latency percentiles (submit -> results on host, microseconds) over the
 * requests completed since the last reset whose size is min_frames ..
 * max_frames frames; 0 when there are none. Any output may be NULL. Errors:
 * POLAR_EINVAL (NULL server, min_frames > max_frames). */
POLAR_API int polar_server_latency(polar_server_t *server, uint32_t min_frames, uint32_t max_frames,
                                   double *p50_us, double *p99_us, uint64_t *count);

/* Allocation-free variant of polar_list_decode. The paper has no
 * counterpart: this entry point exists for callers that cannot allocate
 * device memory while decoding -- real-time paths that may not take
 * allocator locks or fail for lack of memory once they are running, and
 * hosts that give the decoder a fixed memory budget and own every other
 * allocation themselves.
 *
 * Same arguments, outputs and results as polar_list_decode, for codes with
 * L <= 32; a wide code (L = 64 or 128) is refused with POLAR_EUNSUPPORTED,
 * because its kernel keeps every stage in scratch sized per frame. Instead of
 * taking scratch from the stream-ordered allocator, the alpha stages that do
 * not fit in shared memory go to one fixed device array built into the
 * library, of polar_noalloc_scratch_bytes() bytes (64 MiB); every GPU that
 * loads the library holds it until the process exits. The call performs no
 * allocation of any kind.
 *   - The first call on a device looks up that array's device address (with
 *     the device current) and caches it; make that first call before any
 *     stream capture.
 *   - The kernel is persistent: when the full grid would need more scratch
 *     than the array holds, fewer CTAs are launched (slower, same results).
 *     A launch shape whose single CTA needs more than the array is refused
 *     with POLAR_EUNSUPPORTED (choose a smaller list size or a shape with a
 *     larger shared-memory budget).
 *   - Every call uses the same array and leaves its last contents there.
 *     Nothing in it needs to start at zero (each frame writes every stage row
 *     before reading it), but calls whose kernels overlap on the GPU -- on
 *     different streams, or from different threads -- race on the array and
 *     must not be issued.
 * Errors: as polar_list_decode, plus POLAR_EINVAL when the current device is
 * not the device the code was created on. */
POLAR_API int polar_list_decode_noalloc(const polar_code_t *code, const void *llr_dev, int llr_dtype,
                                        uint32_t n_frames, uint8_t *info_bits_dev, float *path_metric_dev,
                                        uint8_t *crc_ok_dev, int32_t *winner_slot_dev, polar_stream_t stream);

/* Size in bytes of the fixed scratch array used by polar_list_decode_noalloc. */
POLAR_API size_t polar_noalloc_scratch_bytes(void);

#ifdef __cplusplus
}
#endif

#endif /* POLAR_GB300_H */
