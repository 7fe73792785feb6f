/*
 * bpstereo.h -- C ABI of the GB300 (sm_103a) stereo hot path of arXiv 1709.06509:
 * a dense NCC matching-cost volume, 4-scale coarse-to-fine min-sum loopy belief
 * propagation with a truncated-linear smoothness term and the fast-converging skip of
 * converged pixels, and a winner-take-all disparity read-out.
 *
 * Conventions shared by every entry point
 *   - Every function returns an int status: BPS_OK (0) or a negative BPS_ERR_* code.
 *     Nothing throws across this boundary.  Arguments are validated before anything is
 *     launched; on a validation error nothing is enqueued and the context is unchanged.
 *   - "d_" pointers are device pointers, "h_" pointers host pointers.  The caller owns
 *     every buffer it passes in; the library never frees or keeps a caller buffer beyond
 *     the call, except the workspace given to bps_create (see there).
 *   - Work is enqueued on the CUDA stream given as `stream` (a cudaStream_t passed as
 *     void*; NULL = the legacy default stream) and is asynchronous unless stated.
 *   - Images are uint8 grayscale, row-major, `pitch` bytes between rows (pitch >= W).
 *     The left image is the reference: disparity d matches left pixel (x, y) with right
 *     pixel (x - d, y).  Disparities are int32 [H][W], row-major, pitch W.
 *   - A context is not thread-safe: calls on one context must be serialised by the caller.
 *
 * Numerical forms (msg_type)
 *   BPS_MSG_INT32  quantised int32 data costs, int32 messages, int32 arithmetic: the plain
 *                  integer min-sum method.  Bit-identical to the integer CPU oracle.
 *   BPS_MSG_U8     the same integer method with narrow storage: int16 costs and uint8
 *                  messages.  Exact (bit-identical to BPS_MSG_INT32) because a normalised
 *                  message lies in [0, lambda*trunc]; requires lambda*trunc <= 255 and
 *                  trunc_data * 4^(levels-1) <= 27000, otherwise BPS_ERR_UNSUPPORTED.
 *   BPS_MSG_FP16   unquantised float data costs clamp(trunc_data*(1-ncc), 0, trunc_data)
 *                  in fp32, fp16 messages, fp32 arithmetic, min-normalised per pixel.
 *                  Approximate; compared with the FP64 oracle by energy gap.
 */
#ifndef BPSTEREO_H
#define BPSTEREO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bps_ctx bps_ctx;

/* status codes */
#define BPS_OK 0
#define BPS_ERR_ARG (-1)         /* invalid argument (size, pointer, parameter range) */
#define BPS_ERR_UNSUPPORTED (-2) /* valid request outside what this build supports */
#define BPS_ERR_CUDA (-3)        /* a CUDA runtime call or kernel launch failed */
#define BPS_ERR_WORKSPACE (-4)   /* workspace missing, too small or misaligned */
#define BPS_ERR_TIMEOUT (-5)     /* a bounded device-side wait gave up */
#define BPS_ERR_STATE (-6)       /* call order violated (e.g. bp_solve before a cost volume) */
#define BPS_ERR_INTERNAL (-7)    /* a device-side consistency check of the debug build failed */

/* numerical forms */
#define BPS_MSG_INT32 0
#define BPS_MSG_U8 1
#define BPS_MSG_FP16 2

/* flags for bps_bp_solve / bps_stereo */
#define BPS_FLAG_FAST_SKIP 1  /* fast-converging BP: skip pixels whose inputs did not change */
#define BPS_FLAG_WARM_START 2 /* start the coarsest scale from d_init_msgs instead of zeros */
#define BPS_FLAG_GRAPH 4      /* bps_stereo*, bps_bp_solve: record the launch sequence once as a
                                 CUDA graph and replay it while the arguments and the kernel
                                 choices (variants, skip rule, candidates) stay the same */
#define BPS_FLAG_PROFILE 8    /* bps_bp_solve: time the BP launches with CUDA events (read with
                                 bps_read_profile / bps_read_launch_times); not with BPS_FLAG_GRAPH */
#define BPS_FLAG_PERSISTENT 16 /* run the whole solve as one persistent cooperative launch instead
                                  of one programmatically chained launch per half-sweep (same
                                  results) */
#define BPS_FLAG_TEST_TIMEOUT 32 /* test hook (with BPS_FLAG_PERSISTENT): the grid barrier waits for one
                                    block more than it has, gives up after 2 ms and the solve
                                    reports BPS_ERR_TIMEOUT through bps_get_error */
#define BPS_FLAG_ASYNC 64 /* bps_stereo_host / bps_batch_stereo_host: return once the work (copies
                             included) is queued on the stream instead of waiting for it; the host
                             outputs are valid, and the host inputs may be rewritten, only after
                             the stream has been synchronised (calls on one stream run in order).
                             With BPS_FLAG_PERSISTENT read the status with bps_get_error /
                             bps_batch_get_error after that synchronisation. */

/* Limits of this build. */
#define BPS_MAX_LEVELS 8
#define BPS_MAX_D 512
#define BPS_MAX_ITERS 1024
#define BPS_MAX_WINDOW 31

/* Human-readable name of a status code (static string, never NULL). */
const char *bps_status_string(int status);

/* The cudaError_t behind the calling thread's last BPS_ERR_CUDA (0 if none yet), and its
 * name as the CUDA runtime reports it (static string). */
int bps_last_cuda_error(void);
const char *bps_cuda_error_string(int code);

/*
 * Bytes of device workspace a context of this shape needs (cost pyramid, messages and
 * skip flags of every scale, reduction scratch, staging buffers of bps_stereo_host).
 * Returns 0 for invalid shapes (W, H >= 1; 1 <= D <= BPS_MAX_D; 1 <= levels <=
 * BPS_MAX_LEVELS; msg_type one of BPS_MSG_*).
 * Scale l has W_l = ceil(W_{l-1} / 2), H_l = ceil(H_{l-1} / 2) ("four scales", section
 * "GPU Implementation"); every scale keeps all D labels.
 */
size_t bps_workspace_bytes(int W, int H, int D, int levels, int msg_type);

/*
 * Create a context for W x H images, D disparity labels and `levels` scales.
 * d_workspace: device memory of at least bps_workspace_bytes(...) bytes, 256-byte aligned,
 * owned by the caller and used exclusively by this context until bps_destroy; or NULL, in
 * which case the context allocates (cudaMalloc) and frees it itself.
 * On success *out receives the context.  Errors: BPS_ERR_ARG (shape, out == NULL),
 * BPS_ERR_WORKSPACE (too small / misaligned), BPS_ERR_CUDA (allocation or stream creation).
 */
int bps_create(bps_ctx **out, int W, int H, int D, int levels, int msg_type, void *d_workspace,
               size_t workspace_bytes);

/*
 * Test hook, failure injection on the host: the next n resource acquisitions of bps_create and
 * bps_batch_create (device allocations, streams, events) succeed and the one after that fails as
 * if the CUDA runtime had refused it (the call then returns BPS_ERR_CUDA, having released
 * everything it had acquired); n < 0 cancels a planned failure.  Process-wide.  Returns BPS_OK.
 */
int bps_test_fail_resources(int n);

/* Destroy a context: synchronises its internal stream and frees what it allocated (cudaFree of
 * a context-owned workspace waits for the work in flight on the device; a caller-owned
 * workspace must not be reused before the context's work on the caller's streams is done).
 * NULL is a no-op. */
int bps_destroy(bps_ctx *ctx);

/*
 * Matching-cost volume (section "Correlation volume computation": normalized cross
 * correlation of the two views).  For every pixel p = (x, y) and label d < D:
 *   ncc(p, d) = (N S_ab - S_a S_b) / sqrt((N S_aa - S_a^2)(N S_bb - S_b^2)),  N = window^2,
 * over the window taps a = L(x+i, y+j), b = R(x-d+i, y+j), |i|, |j| <= window/2, with
 * replicate-clamped coordinates; ncc = 0 where either window is flat.  The data cost is
 *   integer forms:  c = clamp(floor(trunc_data * (1 - ncc) + 1/2), 0, trunc_data), decided
 *                   exactly as FP64 round-to-nearest arithmetic decides it;
 *   BPS_MSG_FP16:   c = clamp(trunc_data * (1 - ncc), 0, trunc_data) in fp32.
 * The coarser scales' costs are then built as the sum of each coarse pixel's existing 2x2
 * children.  d_ncc_out: nullable device float [H][W][D] receiving ncc (abs. error < 1e-5).
 * Errors: BPS_ERR_ARG (NULL images, pitch < W, window even or > BPS_MAX_WINDOW,
 * trunc_data < 0), BPS_ERR_UNSUPPORTED (BPS_MSG_U8 with trunc_data*4^(levels-1) > 27000).
 */
int bps_build_cost_volume(bps_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right, int pitch,
                          int window, int trunc_data, float *d_ncc_out, void *stream);

/*
 * Hierarchical min-sum loopy BP (sections "Fast Converging BP" and "GPU Implementation")
 * on the cost volume of the last bps_build_cost_volume.  Runs `levels` (<= the context's)
 * scales coarsest first; at each scale `iters` iterations of the red-black schedule (all
 * pixels with x + y even, then all odd).  A pixel sends to each existing 4-neighbour q
 *   m(d) = min_d' [h(d') + lambda * min(|d - d'|, trunc)] - min_d (same),
 *   h = its data cost + the messages from its other existing neighbours,
 * written in place into q's incoming slot.  The coarsest scale starts from zero messages
 * (or d_init_msgs with BPS_FLAG_WARM_START: [4][H_c][W_c][D] int32 for the integer forms,
 * float for BPS_MSG_FP16, direction = neighbour the message comes from: up, down, left,
 * right); every finer pixel starts from its parent's messages.  With BPS_FLAG_FAST_SKIP a
 * pixel is recomputed only if one of its incoming messages changed since its last update;
 * the result is identical to running without the skip.  With BPS_FLAG_GRAPH (not with
 * BPS_FLAG_PROFILE) the solve is recorded once as a CUDA graph and replayed while its
 * arguments (d_init_msgs included, as a pointer) and the context's kernel choices hold.
 * Errors: BPS_ERR_STATE (no cost volume yet), BPS_ERR_ARG (levels, iters > BPS_MAX_ITERS,
 * lambda < 0, trunc < 0, lambda*(D+trunc) >= 2^24, warm start without d_init_msgs),
 * BPS_ERR_UNSUPPORTED (BPS_MSG_U8 with lambda*trunc > 255).
 */
int bps_bp_solve(bps_ctx *ctx, int levels, int iters, int lambda, int trunc, int flags,
                 const void *d_init_msgs, void *stream);

/*
 * bps_bp_solve with its own iteration count at every scale: h_iters[l] iterations at scale l
 * (0 = the finest, levels - 1 = the coarsest; host array of `levels` entries, read during the
 * call).  A scale with no iterations passes its start messages down unchanged.  The trace holds
 * 2 h_iters[l] entries per scale, coarsest first.  Flags and errors as bps_bp_solve (each count
 * within [0, BPS_MAX_ITERS]); BPS_FLAG_PERSISTENT needs equal counts (BPS_ERR_UNSUPPORTED).
 */
int bps_bp_solve_schedule(bps_ctx *ctx, int levels, const int *h_iters, int lambda, int trunc, int flags,
                          const void *d_init_msgs, void *stream);

/*
 * Winner-take-all read-out at the finest scale: d(p) = argmin_d [c(p, d) + sum of the
 * messages into p], the lowest d on ties.  d_disp: device int32 [H][W].
 * Errors: BPS_ERR_STATE (no cost volume), BPS_ERR_ARG (NULL).
 */
int bps_wta_disparity(bps_ctx *ctx, int32_t *d_disp, void *stream);

/*
 * Energy E(d) = E_D(d) + E_S(d) (section "Approach Description"): the finest-scale data
 * cost of each pixel's label plus lambda * min(|d_p - d_q|, trunc) over every right and
 * down grid edge.  Integer forms write an exact int64 to d_energy_i64; BPS_MSG_FP16 writes
 * an FP64 sum (fixed reduction order, reproducible) to d_energy_f64.  Either output may be
 * NULL; for the integer forms d_energy_f64 receives the same value as a double.
 * Labels outside [0, D) are clamped to the nearest valid label.
 * Errors: BPS_ERR_STATE (no cost volume), BPS_ERR_ARG (NULL d_disp, lambda or trunc < 0).
 */
int bps_energy(bps_ctx *ctx, const int32_t *d_disp, int lambda, int trunc, int64_t *d_energy_i64,
               double *d_energy_f64, void *stream);

/*
 * The whole path in one call: bps_build_cost_volume, bps_bp_solve over all of the
 * context's scales, bps_wta_disparity.  flags: BPS_FLAG_FAST_SKIP, BPS_FLAG_GRAPH.
 * With BPS_FLAG_GRAPH the launch sequence is captured once into a CUDA graph kept by the
 * context and replayed while every argument is unchanged (a change re-captures).
 */
int bps_stereo(bps_ctx *ctx, const uint8_t *d_left, const uint8_t *d_right, int pitch, int window,
               int trunc_data, int iters, int lambda, int trunc, int flags, int32_t *d_disp,
               void *stream);

/*
 * The whole path from host buffers: copies h_left/h_right (pitch bytes per row) to the
 * context's staging buffers, runs bps_stereo, computes the energy and copies the
 * disparities (int32 [H][W]) and the energy back.  h_energy_i64 / h_energy_f64 nullable.
 * Synchronous: returns after the results are in host memory.  Pinned host memory makes
 * the copies asynchronous with respect to other streams.
 */
int bps_stereo_host(bps_ctx *ctx, const uint8_t *h_left, const uint8_t *h_right, int pitch,
                    int window, int trunc_data, int iters, int lambda, int trunc, int flags,
                    int32_t *h_disp, int64_t *h_energy_i64, double *h_energy_f64, void *stream);

/*
 * Status of this context's device-side checks: BPS_OK, BPS_ERR_TIMEOUT when a bounded wait gave
 * up (a grid barrier of the last persistent solve, or a stage wait of a bulk-copy sweep since the
 * last call; the results are then incomplete), or BPS_ERR_INTERNAL when a bounds check of the
 * debug build (libbpstereo_debug.so, compiled with -DBPS_DEBUG_BOUNDS) failed since the last call.
 * Reading reports the sweep and bounds errors once (they are cleared).  Synchronous.
 */
int bps_get_error(bps_ctx *ctx);
/*
 * The raw error word of the context's device-side checks, left as it is (bps_get_error clears it):
 * 0 none, 1 a bounded wait gave up, 2 and above the code of the largest failed check of the debug
 * build (2 list entry, 3 list append, 4 and 6 data-cost store, 5 read-out pixel, 7 scale-1 store,
 * 8 FP64 list entry, 9 accumulator column, 10 window record, 11 slab row, 12 FP64 pass store).
 */
int bps_peek_error_code(bps_ctx *ctx);

/*
 * Per half-sweep count of recomputed pixels of the last bps_bp_solve (coarsest scale
 * first, two entries per iteration): the fast-converging trace.  Synchronous.  Returns
 * the number of entries written (<= cap) or a negative status.
 */
int bps_get_trace(bps_ctx *ctx, int64_t *h_counts, int cap);

/*
 * Copy scale `level`'s messages to d_out in the natural layout [4][H_l][W_l][D]
 * (int32 for the integer forms, float for BPS_MSG_FP16; slots of missing neighbours are
 * written as 0).  Used for parity checks, checkpoints and warm starts.
 */
int bps_export_messages(bps_ctx *ctx, int level, void *d_out, void *stream);

/* Copy scale `level`'s data cost to d_out, natural layout [H_l][W_l][D] (int32 or float). */
int bps_export_cost(bps_ctx *ctx, int level, void *d_out, void *stream);

/*
 * Read the launch timings recorded by the last bps_bp_solve run with BPS_FLAG_PROFILE:
 * the number of finest-scale sweep launches, their summed duration in ms (CUDA events
 * on the launching stream), and the number of pixels they recomputed.  Synchronous.
 */
int bps_read_profile(bps_ctx *ctx, int *h_launches, double *h_total_ms, int64_t *h_pixels);

/*
 * Per-launch durations (ms, CUDA events on the launching stream) of every sweep launch of
 * the last bps_bp_solve run with BPS_FLAG_PROFILE, in launch order (coarsest scale first,
 * two per iteration).  Synchronous.  Returns the number written (<= cap) or a status.
 */
int bps_read_launch_times(bps_ctx *ctx, double *h_ms, int cap);

/*
 * Batches: several contexts (pairs of possibly different sizes and label counts, all with
 * the same number of scales and the same numerical form) processed together.
 * bps_batch_stereo runs, for every pair i, the whole path of bps_stereo on
 * (d_lefts[i], d_rights[i], pitches[i], windows[i]) into d_disps[i]:
 *   - by default each pair's launch chain runs on its own branch stream, forked from and
 *     joined back into `stream`, so the pairs' chains run concurrently;
 *   - with BPS_FLAG_PERSISTENT the cost volumes run on the branches, then ONE persistent
 *     cooperative launch solves every pair in lockstep and writes every read-out;
 *   - with BPS_FLAG_GRAPH the whole batch is recorded once as one CUDA graph and replayed
 *     while every argument is unchanged.
 * The host arrays (d_lefts ... d_disps) hold n entries each and are read during the call
 * only.  A batch keeps pointers to its contexts: destroy the batch before them.
 * bps_batch_get_error reports BPS_ERR_TIMEOUT when the last persistent launch gave up.
 */
typedef struct bps_batch bps_batch;
#define BPS_MAX_BATCH 256
int bps_batch_create(bps_batch **out, bps_ctx *const *ctxs, int n);
int bps_batch_destroy(bps_batch *batch);
int bps_batch_stereo(bps_batch *batch, const uint8_t *const *d_lefts, const uint8_t *const *d_rights,
                     const int *pitches, const int *windows, int trunc_data, int iters, int lambda, int trunc,
                     int flags, int32_t *const *d_disps, void *stream);
int bps_batch_get_error(bps_batch *batch);

/*
 * bps_batch_stereo from host buffers: copies every pair's images (pitches[i] bytes per row)
 * to its context's staging buffers, runs the batch, computes every pair's energy into
 * h_energies[i] (int64, integer forms; nullable) and copies every disparity map (int32
 * [H_i][W_i]) to h_disps[i].  Synchronous.  Pinned host memory makes the copies asynchronous.
 */
int bps_batch_stereo_host(bps_batch *batch, const uint8_t *const *h_lefts, const uint8_t *const *h_rights,
                          const int *pitches, const int *windows, int trunc_data, int iters, int lambda, int trunc,
                          int flags, int32_t *const *h_disps, int64_t *h_energies, void *stream);

/*
 * Kernel variant of the half-sweeps at one scale (integer u8 form; results are identical
 * for every variant, only the speed differs):
 *   BPS_VARIANT_GENERAL_DT  minimise with the forward/backward distance transform even
 *                           when trunc <= 2 allows the shorter stencil forms;
 *   BPS_VARIANT_LISTS       with the fast-converging skip, process only the listed dirty
 *                           pixels after the scale's first iteration;
 *   BPS_VARIANT_CLUSTER     run every iteration of the scale in one launch of one 16-CTA
 *                           thread-block cluster (hardware cluster barrier between the
 *                           half-sweeps); BPS_ERR_UNSUPPORTED where such a cluster does not fit;
 *   BPS_VARIANT_EAGER       (dense launches) issue every load of a half-sweep at once, before
 *                           the dirty flag is known, and the costs before the wait on the
 *                           preceding kernel: one round trip to memory per half-sweep instead
 *                           of two, at the price of loading clean pixels (small scales);
 *   BPS_VARIANT_DPAR        one group of lanes per (pixel, direction) instead of per pixel:
 *                           the four messages of a pixel side by side (up to 128 labels;
 *                           ignored above), for scales whose time is the latency of few pixels;
 *   BPS_VARIANT_DPAR_LISTS  the same on the list launches only (with BPS_VARIANT_LISTS);
 *   BPS_VARIANT_STAGED      dense launches: each thread copies the next pixel block's inputs
 *                           into shared memory (cp.async) while it computes the current one,
 *                           for HBM-bound scales (not combined with BPS_VARIANT_DPAR);
 *   BPS_VARIANT_STAGED_LISTS the same on the list launches (with BPS_VARIANT_LISTS; not
 *                           combined with BPS_VARIANT_DPAR_LISTS).
 *   BPS_VARIANT_BULK        dense launches: one warp of each CTA copies the whole records of
 *                           the pixels that need computing (cost, incoming messages, the
 *                           receivers' slots for the skip's change test) into a two-stage
 *                           shared-memory ring with 1-D bulk copies (cp.async.bulk, mbarrier
 *                           completion) while eight warps compute from the other stage; takes
 *                           precedence over BPS_VARIANT_STAGED (not combined with BPS_VARIANT_DPAR).
 *                           Its waits are bounded: one that gives up makes bps_get_error report
 *                           BPS_ERR_TIMEOUT for the solve;
 *   BPS_VARIANT_BULK_LISTS  the same on the list launches (with BPS_VARIANT_LISTS).
 *   BPS_VARIANT_BLOCK2      temporal blocking to depth 2 of the scale's first iteration (with
 *                           the fast-converging skip, on scales below the coarsest, without the
 *                           freeze rule): one launch runs both half-sweeps tile by tile (32 x 16
 *                           pixels), each tile's odd pixels reading back from L2 the messages
 *                           its even pixels (and the even pixels bordering it, computed again)
 *                           have just written; ignored elsewhere.
 * With BPS_FLAG_PROFILE a cluster launch's time is shared out evenly over its half-sweeps.
 * variant = -1 restores the default (chosen from the scale's size).  Setting a variant
 * drops a graph recorded by bps_stereo.  bps_get_sweep_variant returns the current one.
 * The autotuner (paper_1709_06509_gb300/autotune.py) picks them by measurement.
 */
/*
 * Shape of the NCC kernel's CTAs (windows up to 15): column_groups groups of 16 columns per
 * CTA (column_groups * D rounded up to 16 threads, between 32 and 512) and `rows` image rows
 * per strip (even).  0, 0 restores the default.  Results do not depend on it; the autotuner
 * picks it by measurement.  Drops a graph recorded by bps_stereo.
 */
int bps_set_ncc_shape(bps_ctx *ctx, int column_groups, int rows);

/*
 * Which kernel forms the NCC cost volume (section "Correlation volume computation"):
 *   BPS_NCC_DEFAULT  the tensor-core kernel where it applies, else a CUDA-core kernel;
 *   BPS_NCC_ROWS     a CUDA-core kernel (the row-streaming one for windows up to 15);
 *   BPS_NCC_TENSOR   the tensor-core kernel where it applies (as the default).
 * The tensor-core kernel forms every window sum of products S_ab of a 128-pixel tile and a block
 * of up to 128 labels as one banded matrix product on tcgen05 (BF16 image bytes, FP32
 * accumulation: exact, since every S_ab is an integer below 2^24), then quantises like the
 * row kernel: the costs are the same bits.  It applies to the integer cost forms (BPS_MSG_INT32,
 * BPS_MSG_U8), odd windows up to 9, trunc_data up to 127, and calls without ncc_out.
 * rows: image rows per strip of the tensor-core kernel (even; 0: strips that cover the SMs about
 * once).  Results do not depend on either choice.  Drops a graph recorded by bps_stereo.
 * bps_get_ncc_kernel returns the kernel (BPS_NCC_TENSOR or BPS_NCC_ROWS) that
 * bps_build_cost_volume would use for this window and trunc_data without ncc_out.
 */
#define BPS_NCC_DEFAULT 0
#define BPS_NCC_ROWS 1
#define BPS_NCC_TENSOR 2
int bps_set_ncc_kernel(bps_ctx *ctx, int kernel, int rows);
int bps_get_ncc_kernel(bps_ctx *ctx, int window, int trunc_data);

#define BPS_VARIANT_GENERAL_DT 1
#define BPS_VARIANT_LISTS 2
#define BPS_VARIANT_CLUSTER 4
#define BPS_VARIANT_EAGER 8
#define BPS_VARIANT_DPAR 16
#define BPS_VARIANT_DPAR_LISTS 32
#define BPS_VARIANT_STAGED 64
#define BPS_VARIANT_STAGED_LISTS 128
#define BPS_VARIANT_BULK 256
#define BPS_VARIANT_BULK_LISTS 512
#define BPS_VARIANT_BLOCK2 1024
int bps_set_sweep_variant(bps_ctx *ctx, int level, int variant);
int bps_get_sweep_variant(bps_ctx *ctx, int level);

/* The skip rule of the fast-converging variant (section "Fast Converging BP" does not fix the
 * convergence test; the default, eps = 0 and freeze = 0, is the exact rule whose results equal
 * those of no skip).  eps in [0, 255]: a recomputed pixel marks a receiver dirty only when the
 * new message differs from the stored one by more than eps at some label (the message itself
 * is always stored).  freeze = 1: a recomputed pixel that marked no receiver is frozen and not
 * recomputed again at that scale, even when marked later.  Both make the skip approximate
 * (judged by the energy gap).  u8 message form only: BPS_ERR_UNSUPPORTED otherwise for a
 * non-exact rule; BPS_ERR_ARG out of range.  Applies to later solves of this context,
 * including batches and persistent launches it takes part in. */
int bps_set_skip_rule(bps_ctx *ctx, int eps, int freeze);

/* Sparse candidates (the abstract: normalised cross correlation retrieves a sparse set of
 * candidate matches and belief propagation then chooses among them).  K = 0 (the default): the
 * dense solve.  1 <= K <= min(D, BPS_MAX_CANDIDATES): later solves of this context run the
 * scales above the finest densely; at the finest scale each pixel keeps the K labels of lowest
 * data cost (the lower label first among equal costs), each candidate starts from the parent's
 * message at its label, and messages are vectors over the receiver's candidates,
 *   m(j) = min over the sender's candidates i of h(i) + lambda*min(|label_i - label_j|, trunc),
 * minus their minimum.  bps_wta_disparity then picks the candidate of least belief (lowest
 * label on ties); bps_energy scores the labels with the dense cost.  K = D gives the dense
 * solve's results.  u8 form only, exact skip rule only (BPS_ERR_UNSUPPORTED otherwise, and for
 * BPS_FLAG_PERSISTENT, or BPS_FLAG_WARM_START with one scale); BPS_ERR_ARG out of range.
 * After a sparse solve bps_export_messages(level 0) returns BPS_ERR_STATE; read the finest
 * scale with bps_export_sparse: d_cand int32 [H][W][K] labels in increasing order, d_msgs
 * int32 [4][H][W][K] (direction as in bps_export_messages), both caller-owned device buffers. */
#define BPS_MAX_CANDIDATES 32
int bps_set_candidates(bps_ctx *ctx, int K);
int bps_export_sparse(bps_ctx *ctx, int32_t *d_cand, int32_t *d_msgs, void *stream);

/*
 * Learned warm start: kernels of a small convolutional network that predicts the coarsest
 * scale's messages from the coarsest cost volume (the start messages of bps_bp_solve with
 * BPS_FLAG_WARM_START).  The paper has no network; it is a way to start BP closer to its fixed
 * point, judged by the BP energy it leads to.  Activations are [B][C][H][W], BF16 (bf16 != 0)
 * or FP32; weights [Cout][Cin][3][3] BF16; biases and gradients FP32; every product is
 * accumulated in FP32.  3x3 convolutions with zero padding keep H x W.  All asynchronous on
 * `stream`; the caller owns every buffer.  Errors: BPS_ERR_ARG (NULL, sizes < 1), BPS_ERR_CUDA.
 *
 * bps_warmnet_conv3x3          out = conv(in, w) + bias, then max(., 0) when relu; with BF16 input
 *                              an implicit GEMM on the tensor cores (tcgen05, FP32 accumulator in
 *                              tensor memory); Cin * 9 <= 2^20, B * H * W <= 2^31 (BPS_ERR_ARG)
 * bps_warmnet_get_error        BPS_ERR_TIMEOUT when a bounded wait of a tensor-core convolution
 *                              gave up since the last call (its output is then unwritten), else
 *                              BPS_OK; synchronous
 * bps_warmnet_conv3x3_backward gradients of one such layer from d_gout (the gradient of its
 *                              output; masked by d_relu_out > 0 when the layer had a ReLU):
 *                              d_gw (and d_gb when not NULL) always, d_gin when not NULL
 * bps_warmnet_mse              grad = 2 (pred - target) mask / n and per-block partial sums of
 *                              the masked mean squared error (nparts blocks)
 * bps_warmnet_adam             one Adam step (Kingma & Ba 2015) of FP32 master weights, also
 *                              written as BF16 to d_w_bf16 when not NULL (step counts from 1)
 * bps_warmnet_features         network input from a natural int32 cost volume [H][W][D]:
 *                              channel g = (min of labels 8g..8g+7 - min of all labels) * scale,
 *                              BF16 [ceil(D/8)][H][W]
 * bps_warmnet_messages         start messages [4][H][W][D] int32 from the network output
 *                              [4 * D][H][W] FP32: rounded, clamped to [0, cap], minimum
 *                              shifted to 0, 0 for neighbours outside the image
 */
int bps_warmnet_conv3x3(const void *d_in, int in_bf16, int B, int Cin, int H, int W, const void *d_w,
                        const float *d_bias, int Cout, int relu, void *d_out, int out_bf16, void *stream);
int bps_warmnet_get_error(void);
int bps_warmnet_conv3x3_backward(const float *d_gout, const void *d_relu_out, const void *d_in, int in_bf16, int B,
                                 int Cin, int H, int W, const void *d_w, int Cout, float *d_gin, float *d_gw,
                                 float *d_gb, void *stream);
int bps_warmnet_mse(const float *d_pred, const float *d_target, const float *d_mask, int64_t n, float *d_grad,
                    float *d_loss_parts, int nparts, void *stream);
int bps_warmnet_adam(float *d_w, float *d_m, float *d_v, const float *d_g, int64_t n, float lr, float beta1,
                     float beta2, float eps, int step, void *d_w_bf16, void *stream);
int bps_warmnet_features(const int32_t *d_cost, int H, int W, int D, float scale, void *d_feat, void *stream);
int bps_warmnet_messages(const float *d_pred, int H, int W, int D, int cap, int32_t *d_init, void *stream);

/*
 * Diagnostic: what separating two phases of the solve costs on this GPU, as the chained and the
 * persistent launch forms pay it.  h_barrier_us receives the time per grid barrier of `phases`
 * barriers inside one cooperative launch of `ctas` 256-thread CTAs (the persistent kernel's
 * barrier, bounded wait included); h_boundary_us the time per kernel of `phases` empty kernels of
 * the same grid chained by programmatic dependent launch and replayed from a CUDA graph (the
 * boundary between two half-sweeps of the chained form).  Best of three after a warm-up each.
 * Synchronous; allocates and frees its own stream, events, graph and 16 bytes of device memory.
 * Errors: BPS_ERR_ARG (ctas < 1, phases outside [1, 100000], NULL outputs), BPS_ERR_UNSUPPORTED
 * (more CTAs than fit on the GPU at once), BPS_ERR_TIMEOUT (a barrier gave up), BPS_ERR_CUDA.
 */
int bps_measure_sync_costs(int ctas, int phases, double *h_barrier_us, double *h_boundary_us);

/*
 * Energy of a labelling without allocating any memory.  The paper has no counterpart:
 * this entry point serves callers that cannot allocate device memory when they need the
 * energy -- real-time loops that may not wait on an allocator (cudaMalloc and cudaFree may
 * synchronise the whole device), programs whose device memory belongs to an allocator this
 * library cannot reach, code under a fixed memory budget where a new allocation may fail.
 *
 * Computes E(d) = sum_p cost(p, d_p) + sum over right and down grid edges of
 * lambda * min(|d_p - d_q|, trunc), exactly, in int64, from
 *   d_cost   device int32 [H][W][D], natural layout (e.g. what bps_export_cost writes),
 *   d_disp   device int32 [H][W] labels (values outside [0, D) are clamped),
 * into d_energy (device int64).  Asynchronous on `stream`.  Caller owns all three buffers.
 *
 * Scratch: one partial sum per 1024 pixels in a fixed array compiled into the library
 * (BPS_NOALLOC_MAX_BLOCKS entries, 128 KiB of device memory on every GPU that loads the
 * library, held until the process exits); nothing is allocated, no cudaMalloc or cudaFree is
 * called.  Images with more than BPS_NOALLOC_MAX_PIXELS pixels are rejected with
 * BPS_ERR_UNSUPPORTED before anything is launched.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current: make that first
 * call before any stream capture.  cudaDeviceReset invalidates the looked-up address; a call
 * whose launch fails forgets it, and the next call looks it up again.  All calls share the array: calls whose kernels overlap on
 * the GPU (other streams, other host threads) race on it; calls in order on one stream are
 * safe.  Errors: BPS_ERR_ARG (NULL pointer, sizes < 1, lambda or trunc < 0),
 * BPS_ERR_UNSUPPORTED (too many pixels), BPS_ERR_CUDA.
 */
#define BPS_NOALLOC_MAX_BLOCKS 16384
#define BPS_NOALLOC_MAX_PIXELS (BPS_NOALLOC_MAX_BLOCKS * 1024)
int bps_energy_noalloc(const int32_t *d_cost, const int32_t *d_disp, int W, int H, int D, int lambda, int trunc,
                       int64_t *d_energy, void *stream);

#ifdef __cplusplus
}
#endif
#endif
