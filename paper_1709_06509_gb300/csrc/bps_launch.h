// bps_launch.h -- host-side launchers of the stereo kernels (internal to the library).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "bps_internal.cuh"

namespace bps {

// Launch `kernel` so that it may begin while the previous kernel on the stream finishes
// (programmatic stream serialisation; the kernel itself waits in pdl_enter()).  Also valid
// under stream capture, where it becomes a programmatic graph edge.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                            Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

// storage kinds
enum CostKind { COST_I32 = 0, COST_I16 = 1, COST_F32 = 2 };
enum MsgKind { MSG_I32 = 0, MSG_U8 = 1, MSG_F16 = 2 };

size_t ncc_smem_bytes(int D, int window);
// Allow the NCC kernel the shared memory of the largest window (call outside stream capture).
cudaError_t ncc_prepare(int cost_kind, int D, int max_window);
cudaError_t launch_ncc(int cost_kind, const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int D, int Dp,
                       int window, int T, int Wh, void *c0, void *c1, float *ncc_out, cudaStream_t st);
cudaError_t launch_pyramid(int cost_kind, const LevelView &fine, const LevelView &coarse, int Dp, cudaStream_t st);
// Scales l and l+1 from scale l-1 in one launch.
cudaError_t launch_pyramid2(int cost_kind, const LevelView &fine, const LevelView &mid, const LevelView &coarse, int Dp,
                            cudaStream_t st);

// Row-streaming NCC for windows up to NCC_ROWS_MAX_WINDOW; with l1 != NULL (integer forms)
// it also writes scale 1 of the pyramid.
constexpr int NCC_ROWS_MAX_WINDOW = 15;
// xs, tys: column groups of 16 per CTA and rows per strip (0: the default shape).
cudaError_t launch_ncc_rows(int cost_kind, const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int D, int Dp,
                            int window, int T, const LevelView &l0, const LevelView *l1, float *ncc_out,
                            cudaStream_t st, int xs = 0, int tys = 0);
cudaError_t ncc_rows_prepare(int cost_kind, int D, int Dp);

// Tensor-core NCC (integer forms, odd windows up to NCC_TC_MAX_WINDOW, trunc_data up to 8191):
// the same costs as the row kernel, and scale 1 with l1 != NULL.  rows: image rows per strip
// (0: the default, strips that cover the SMs about once).
constexpr int NCC_TC_MAX_WINDOW = 9;
bool ncc_tc_supported(int cost_kind, int Dp, int window, int T);
size_t ncc_tc_smem_bytes(int Dp, int window);
cudaError_t ncc_tc_prepare(int cost_kind, int Dp);
// fix: a workspace buffer of ncc_tc_fix_bytes (zeroed once) for the values the kernel leaves to a
// second, FP64 pass (null: every row decides them itself, slower).
size_t ncc_tc_fix_bytes(int W, int H, int Dp);
cudaError_t launch_ncc_tc(int cost_kind, const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int D, int Dp,
                          int window, int T, const LevelView &l0, const LevelView *l1, cudaStream_t st, int rows,
                          void *fix, size_t fix_bytes);

// Kernel variant of the u8 half-sweep at one scale (bit set; see bps_set_sweep_variant).
constexpr int VARIANT_GENERAL_DT = 1;  // the distance transform even where a stencil form exists
constexpr int VARIANT_LISTS = 2;       // active lists after the scale's first iteration (skip on)
constexpr int VARIANT_CLUSTER = 4;     // every iteration of the scale in one thread-block-cluster launch
constexpr int VARIANT_EAGER = 8;       // every load of a half-sweep issued at once (dense launches)
constexpr int VARIANT_DPAR = 16;       // one lane group per (pixel, direction), up to 128 labels
constexpr int VARIANT_DPAR_LISTS = 32; // ... on the list launches only
constexpr int VARIANT_STAGED = 64;     // dense launches stage the next block's inputs in shared memory
constexpr int VARIANT_STAGED_LISTS = 128; // ... list launches
constexpr int VARIANT_BULK = 256;      // dense launches fed by a copy warp's cp.async.bulk pipeline
constexpr int VARIANT_BULK_LISTS = 512; // ... list launches
constexpr int VARIANT_BLOCK2 = 1024;   // the first iteration temporally blocked: both half-sweeps in one launch

// Active lists of a half-sweep (u8 form with the skip on; all members nullable).
struct SweepLists {
    const unsigned *in;    // pixels to process (NULL: every pixel of the colour)
    const unsigned *n_in;  // device count of `in`
    unsigned *out;         // list of the other colour's newly dirty pixels
    unsigned *n_out;       // its device count (zeroed before the half-sweep)
};

// One red-black half-sweep of `colour` at one scale.  trace: nullable device counter of
// recomputed pixels.
cudaError_t launch_sweep(int msg_kind, const LevelView &lv, int colour, int D, int Dp, int Gp, int lambda,
                         int trunc, int skip, unsigned long long *trace, cudaStream_t st,
                         const SweepLists &lists = SweepLists{nullptr, nullptr, nullptr, nullptr}, int variant = 0);
// The first iteration of a scale with the fused coarse-to-fine start (u8 form, skip on) in one
// launch, tile by tile (temporal blocking to depth 2): `first` / `second` are the views of its two
// half-sweeps (start 1 and 2), trace0 / trace1 their trace counters, `lists` the list the second
// appends to (members nullable).  The even pixels' flags are cleared first (a second launch).
cudaError_t launch_sweep_block2(const LevelView &first, const LevelView &second, int D, int Dp, int Gp, int lambda,
                                int trunc, unsigned long long *trace0, unsigned long long *trace1,
                                const SweepLists &lists, cudaStream_t st);
// All iterations of one scale (u8 form) in one launch of one 16-CTA cluster; available only
// where such a cluster fits (cluster_sweep_available).
bool cluster_sweep_available();
cudaError_t launch_sweep_level_cluster(const LevelView &lv, int D, int Dp, int Gp, int lambda, int trunc, int skip,
                                       unsigned long long *trace, int iters, int variant, cudaStream_t st);

// Coarse-to-fine start: copy parent messages into the fine pixels of `colour` (and of the
// other colour too when both_colours), and mark every pixel of the fine scale dirty when
// set_dirty (fast-converging skip).
cudaError_t launch_upsample(int msg_kind, const LevelView &coarse, const LevelView &fine, int both_colours, int Dp,
                            int set_dirty, cudaStream_t st);
// Start of a solve at scale `top`: zero its messages (zero_msgs), mark its pixels dirty
// (set_dirty) and zero ntrace trace counters, in one kernel.
cudaError_t launch_solve_start(int msg_kind, const LevelView &top, int Dp, int zero_msgs, int set_dirty,
                               unsigned long long *trace, unsigned *list_counts, int ntrace, cudaStream_t st);
// Natural-layout [4][H][W][D] messages (int32 or float) into / out of colour-split storage.
cudaError_t launch_import_msgs(int msg_kind, const LevelView &lv, int D, int Dp, const void *src, cudaStream_t st);
cudaError_t launch_export_msgs(int msg_kind, const LevelView &lv, int D, int Dp, void *dst, cudaStream_t st);
cudaError_t launch_export_cost(int cost_kind, const LevelView &lv, int D, int Dp, void *dst, cudaStream_t st);

// ------------------------------------------------------------------ persistent batched solve
// One pair of a batch as the persistent kernel sees it (device memory).
struct PairDesc {
    LevelView lv[8];
    int D, Dp, Gp;
    unsigned long long *trace;  // per half-sweep counters of this pair (nullable)
    int32_t *disp;              // winner-take-all output (nullable: no read-out)
    unsigned *lists[2];         // active lists of the even / odd pixels (sized for the finest scale)
    unsigned *list_counts;      // entries appended during each half-sweep (zeroed before the launch)
};
struct PersistParams {
    const PairDesc *pairs;        // [npairs]
    const int *sweep_prefix;      // [levels][npairs + 1]: first work block of each pair in a half-sweep
    const int *wta_prefix;        // [npairs + 1]: first work block of each pair in the read-out
    int npairs, levels, iters, lam, lam_u8, trunc, skip;
    int lists;                    // after a scale's first iteration, sweep only the listed dirty pixels
    unsigned *barrier;            // {arrival count, error word}, zeroed before the launch
    unsigned extra_arrivals;      // test hook: > 0 makes every barrier wait for blocks that never come
    unsigned long long timeout_ns;
    int32_t *disp_override;       // single-pair launches: read-out target of pair 0 (nullable)
};
// Co-resident CTAs of the persistent kernel of this form and truncation (looked up once each).
cudaError_t persistent_grid(int form, int trunc, int *grid);
// Whether the persistent kernel of this form and truncation sweeps over active lists.
bool persistent_takes_lists(int form, int trunc);
cudaError_t launch_persistent(int form, const PersistParams &P, cudaStream_t st);

// Load every kernel a launch sequence may use (CUDA loads modules lazily on first use,
// which must not happen inside a stream capture).
cudaError_t preload_cost_kernels(int cost_kind);
cudaError_t preload_bp_kernels(int msg_kind);
cudaError_t preload_readout_kernels(int msg_kind);

// Winner-take-all disparity at the finest scale.
cudaError_t launch_wta(int msg_kind, const LevelView &lv, int D, int Dp, int Gp, int32_t *disp, cudaStream_t st);
// The rest of a read-out the finest scale's half-sweeps started (LevelView::disp): the even
// pixels dirtied by the last half-sweep, from the list of them (non-null `list`, device count
// n_list) or from the skip flags (every even pixel with the skip off).
cudaError_t launch_wta_rest(int msg_kind, const LevelView &lv, int D, int Dp, int Gp, int skip, const unsigned *list,
                            const unsigned *n_list, int32_t *disp, cudaStream_t st);

// Sparse candidates of the finest scale (sparse.cu): per colour, Kp uint16 labels a slot, then
// Kp int16 costs a slot (K candidates, Kp = K rounded up to a power of two).
struct SparseView {
    uint16_t *cand[2];
    int K, Kp;
};
cudaError_t launch_sparse_candidates(const LevelView &lv, const SparseView &sv, int D, int Dp, int Gp, cudaStream_t st);
cudaError_t launch_sparse_start(const LevelView &fine, const LevelView *coarse, const SparseView &sv, int Dp,
                                cudaStream_t st);
cudaError_t launch_sparse_sweep(const LevelView &lv, const SparseView &sv, int colour, int lambda, int trunc, int skip,
                                unsigned long long *trace, cudaStream_t st);
cudaError_t launch_sparse_wta(const LevelView &lv, const SparseView &sv, int32_t *disp, cudaStream_t st);
cudaError_t launch_sparse_export(const LevelView &lv, const SparseView &sv, int32_t *cand, int32_t *msg,
                                 cudaStream_t st);
cudaError_t preload_sparse_kernels();

// The fp16-message form's half-sweep in packed half2 arithmetic (sweep_f16.cu), for T <= 2.
bool sweep_f16_applies(int trunc);
cudaError_t launch_sweep_f16(const LevelView &lv, int colour, int D, int Dp, int Gp, int lambda, int trunc, int skip,
                             unsigned long long *trace, bool eager, const SweepLists &lists, cudaStream_t st);
cudaError_t preload_f16_kernels();
// Energy: per-block partial sums into `partials` (nblocks entries of 8 bytes), then one
// block sums them in a fixed order.
int energy_blocks(int W, int H);
cudaError_t launch_energy(int cost_kind, const LevelView &lv, int D, int Dp, const int32_t *disp, int lambda,
                          int trunc, void *partials, int64_t *out_i64, double *out_f64, cudaStream_t st);

}  // namespace bps
