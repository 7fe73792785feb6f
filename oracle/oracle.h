/*
 * oracle.h -- plain CPU reference of the stereo hot path of arXiv 1709.06509
 * ("A LBP based correspondence identification scheme for multi-view sensing network").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load this library.  It shares no code with the CUDA path.
 *
 * Everything is a direct, unblocked transcription of the definitions:
 *   - NCC matching cost (section "Correlation volume computation"), FP64 ratio of exact
 *     integer window sums, replicate-clamped borders;
 *   - quantised data cost c = clamp(floor(T_d (1 - ncc) + 1/2), 0, T_d);
 *   - cost pyramid: a coarse pixel's cost is the sum of its existing 2x2 children
 *     (section "GPU Implementation": four scales, same process at each scale);
 *   - min-sum message update on the 4-connected grid from the data term, the messages of
 *     the other three neighbours and the truncated-linear smoothness cost
 *     V(d, d') = lambda * min(|d - d'|, T) (section "Fast Converging BP"), normalised so
 *     that min_d m(d) = 0; O(D^2) minimisation exactly as the definition reads;
 *   - red-black schedule: one iteration = all pixels with (x + y) even, then all odd;
 *   - fast-converging BP: a pixel is recomputed only if one of its incoming messages
 *     changed since it was last computed (exact: identical output to no skipping);
 *   - coarse-to-fine: zero messages at the coarsest scale, each finer pixel starts from
 *     its parent's messages;
 *   - winner-take-all disparity (lowest d wins ties) and the energy
 *     E(d) = E_D(d) + E_S(d) (section "Approach Description"), each grid edge once.
 *
 * Array layouts (all row-major, D innermost):
 *   images        uint8  [H][W]
 *   ncc / cost    [H][W][D]
 *   messages      [4][H][W][D], direction index = neighbour the message comes FROM:
 *                 0 = up (x, y-1), 1 = down (x, y+1), 2 = left (x-1, y), 3 = right (x+1, y).
 *                 Slots of missing neighbours hold 0.
 *   trace         one count per half-sweep, coarsest scale first: number of pixels
 *                 recomputed in that half-sweep.
 * Functions returning int return 0 on success and -1 on bad arguments or allocation failure.
 */
#ifndef BPS_ORACLE_H
#define BPS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Threads of the OpenMP build (a timing build; same results): sets the count when n > 0 and
 * returns the count in use (1 in the serial build). */
int oracle_threads(int n);

/* ncc[H][W][D] in FP64.  window odd >= 1. */
int oracle_ncc(const uint8_t *L, const uint8_t *R, int W, int H, int D, int window, double *ncc);

/* c = clamp(floor(trunc*(1 - ncc) + 0.5), 0, trunc), FP64 round-to-nearest, no contraction. */
int oracle_quantise(const double *ncc, int64_t n, int trunc_data, int32_t *cost);

/* float data cost for the FP64 / FP16 message forms: clamp(trunc*(1 - ncc), 0, trunc). */
int oracle_cost_float(const double *ncc, int64_t n, int trunc_data, double *cost);

/* Scale sizes: Ws[0] = W, Ws[l+1] = ceil(Ws[l] / 2) (same for H).  Returns levels. */
int oracle_level_dims(int W, int H, int levels, int *Ws, int *Hs);

/* Cost pyramid, all scales concatenated finest first, each [H_l][W_l][D]. */
int oracle_pyramid_i32(const int32_t *cost0, int W, int H, int D, int levels, int32_t *out);
int oracle_pyramid_f64(const double *cost0, int W, int H, int D, int levels, double *out);

/* One message from the combined input h[D] (data term plus the three other incoming
 * messages): m(d) = min_d' (h(d') + lambda*min(|d - d'|, trunc)) - min_d (same). */
void oracle_message_i32(const int32_t *h, int D, int lambda, int trunc, int32_t *m);
void oracle_message_f64(const double *h, int D, double lambda, int trunc, double *m);

/* Hierarchical min-sum BP.  init_coarsest: nullable [4][H_c][W_c][D] start messages at the
 * coarsest scale (zero when NULL).  order_seed: 0 = raster order inside a half-sweep,
 * otherwise a seeded permutation (the result must not depend on it).  msg0_out receives
 * the finest-scale messages [4][H][W][D].  trace: nullable, levels*iters*2 entries. */
int oracle_bp_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda,
                  int trunc, int skip, const int32_t *init_coarsest, uint64_t order_seed,
                  int32_t *msg0_out, int64_t *trace);
int oracle_bp_f64(const double *cost0, int W, int H, int D, int levels, int iters, double lambda,
                  int trunc, int skip, const double *init_coarsest, uint64_t order_seed,
                  double *msg0_out, int64_t *trace);

/* Hierarchical BP with an iteration count per scale: iters[l] iterations at scale l (0 = the
 * finest, levels - 1 = the coarsest), the exact skip rule, raster order; otherwise as
 * oracle_bp_i32.  trace: nullable, sum over the scales of 2 iters[l] entries, coarsest first. */
int oracle_bp_schedule_i32(const int32_t *cost0, int W, int H, int D, int levels, const int *iters, int lambda,
                           int trunc, int skip, const int32_t *init_coarsest, int32_t *msg0_out, int64_t *trace);

/* Hierarchical BP (exact skip rule, zero start messages, raster order) followed by the
 * winner-take-all read-out, without handing the messages back: disp [H][W]; trace as above.
 * Same results as oracle_bp_* then oracle_wta_*, in half the host memory (for full-HD pairs
 * with many labels). */
int oracle_bp_wta_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda, int trunc,
                      int skip, int32_t *disp, int64_t *trace);
int oracle_bp_wta_f64(const double *cost0, int W, int H, int D, int levels, int iters, double lambda, int trunc,
                      int skip, int32_t *disp, int64_t *trace);

/* The same with an approximate skip rule (section "Fast Converging BP" leaves the convergence
 * test open): a receiver is marked dirty only when its new message differs from the stored one
 * by more than eps at some label, and with freeze a recomputed pixel that marked no receiver
 * is not recomputed again at that scale.  eps = 0, freeze = 0 is the exact skip above. */
int oracle_bp_rule_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda,
                       int trunc, int skip, int eps, int freeze, const int32_t *init_coarsest,
                       uint64_t order_seed, int32_t *msg0_out, int64_t *trace);
int oracle_bp_rule_f64(const double *cost0, int W, int H, int D, int levels, int iters, double lambda,
                       int trunc, int skip, double eps, int freeze, const double *init_coarsest,
                       uint64_t order_seed, double *msg0_out, int64_t *trace);

/* Sparse candidates (the abstract: NCC retrieves a sparse set of candidate matches and BP chooses
 * among them).  oracle_candidates: per pixel the K labels of lowest cost (the lower label first
 * among equal costs), listed in increasing label order, cand [H][W][K].  oracle_bp_sparse_i32:
 * scales levels-1 .. 1 run the dense solve above; at the finest scale each candidate starts from
 * the parent's message at its label, and red-black min-sum BP runs over the candidate sets:
 * m(j) = min over the sender's candidates i of h(i) + lambda*min(|label_i - label_j|, trunc),
 * minus its minimum, for each receiver candidate j.  msg_out [4][H][W][K]; trace as above.
 * oracle_wta_sparse_i32: the candidate of least belief (lowest label on ties). */
int oracle_candidates(const int32_t *cost0, int W, int H, int D, int K, int32_t *cand);
int oracle_bp_sparse_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda,
                         int trunc, int skip, int K, int32_t *cand_out, int32_t *msg_out, int64_t *trace);
int oracle_wta_sparse_i32(const int32_t *cost0, const int32_t *cand, const int32_t *msg, int W, int H, int D,
                          int K, int32_t *disp);

/* d*(p) = argmin_d [cost(p, d) + sum of incoming messages], lowest d on ties. */
int oracle_wta_i32(const int32_t *cost, const int32_t *msg, int W, int H, int D, int32_t *disp);
int oracle_wta_f64(const double *cost, const double *msg, int W, int H, int D, int32_t *disp);

/* E = sum_p cost(p, d_p) + sum over right and down edges of lambda*min(|d_p - d_q|, trunc).
 * Labels outside [0, D) make the call return INT64_MIN / NaN. */
int64_t oracle_energy_i32(const int32_t *cost, const int32_t *disp, int W, int H, int D,
                          int lambda, int trunc);
double oracle_energy_f64(const double *cost, const int32_t *disp, int W, int H, int D,
                         double lambda, int trunc);

#ifdef __cplusplus
}
#endif
#endif
