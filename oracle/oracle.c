/*
 * oracle.c -- plain CPU reference of the stereo hot path of arXiv 1709.06509.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  See oracle.h for the
 * definitions, layouts and the paper passages each function follows.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC oracle.c -lm
 * (-ffp-contract=off keeps every FP64 multiply and add separately rounded; gcc would
 * otherwise fuse them on aarch64.)  A second build adds -fopenmp, for timing only: the NCC
 * rows and the pixels of one colour in a half-sweep are then split over threads.  Every
 * output element is computed by the same operations either way (the pixels of one colour
 * are independent within a half-sweep, which the shuffled-order pin checks), so both builds
 * return the same bits.
 *
 * The message passing runs in FP64 for both forms.  With integer costs, lambda and trunc
 * every value stays an integer far below 2^53, so FP64 min/+/- are exact and the integer
 * entry points return exactly the integer min-sum result.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { UP = 0, DOWN = 1, LEFT = 2, RIGHT = 3 };

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* The OpenMP build's thread count (set when n > 0); returns the count in use, 1 in the
 * serial build. */
int oracle_threads(int n)
{
#ifdef _OPENMP
    if (n > 0)
        omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ---------------------------------------------------------------- NCC (Correlation volume) */

int oracle_ncc(const uint8_t *L, const uint8_t *R, int W, int H, int D, int window, double *ncc)
{
    if (!L || !R || !ncc || W < 1 || H < 1 || D < 1 || window < 1 || (window & 1) == 0)
        return -1;
    const int r = window / 2;
    const int64_t N = (int64_t)window * window;
#pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x)
            for (int d = 0; d < D; ++d) {
                int64_t Sa = 0, Sb = 0, Saa = 0, Sbb = 0, Sab = 0;
                for (int j = -r; j <= r; ++j)
                    for (int i = -r; i <= r; ++i) {
                        const int yy = clampi(y + j, 0, H - 1);
                        const int64_t a = L[(int64_t)yy * W + clampi(x + i, 0, W - 1)];
                        const int64_t b = R[(int64_t)yy * W + clampi(x - d + i, 0, W - 1)];
                        Sa += a;
                        Sb += b;
                        Saa += a * a;
                        Sbb += b * b;
                        Sab += a * b;
                    }
                const int64_t num = N * Sab - Sa * Sb;
                const int64_t va = N * Saa - Sa * Sa;
                const int64_t vb = N * Sbb - Sb * Sb;
                const double den = (double)va * (double)vb;
                ncc[((int64_t)y * W + x) * D + d] = den == 0.0 ? 0.0 : (double)num / sqrt(den);
            }
    return 0;
}

int oracle_quantise(const double *ncc, int64_t n, int trunc_data, int32_t *cost)
{
    if (!ncc || !cost || n < 0 || trunc_data < 0)
        return -1;
    const double T = (double)trunc_data;
    for (int64_t k = 0; k < n; ++k) {
        const double t = 1.0 - ncc[k];
        const double v = T * t;
        const double w = v + 0.5;
        const double f = floor(w);
        int c = f < 0.0 ? 0 : (f > T ? trunc_data : (int)f);
        cost[k] = c;
    }
    return 0;
}

int oracle_cost_float(const double *ncc, int64_t n, int trunc_data, double *cost)
{
    if (!ncc || !cost || n < 0 || trunc_data < 0)
        return -1;
    const double T = (double)trunc_data;
    for (int64_t k = 0; k < n; ++k) {
        const double v = T * (1.0 - ncc[k]);
        cost[k] = v < 0.0 ? 0.0 : (v > T ? T : v);
    }
    return 0;
}

/* ---------------------------------------------------------------- scales (GPU Implementation) */

int oracle_level_dims(int W, int H, int levels, int *Ws, int *Hs)
{
    if (W < 1 || H < 1 || levels < 1 || !Ws || !Hs)
        return -1;
    Ws[0] = W;
    Hs[0] = H;
    for (int l = 1; l < levels; ++l) {
        Ws[l] = (Ws[l - 1] + 1) / 2;
        Hs[l] = (Hs[l - 1] + 1) / 2;
    }
    return levels;
}

int oracle_pyramid_f64(const double *cost0, int W, int H, int D, int levels, double *out)
{
    int Ws[32], Hs[32];
    if (!cost0 || !out || D < 1 || levels > 32 || oracle_level_dims(W, H, levels, Ws, Hs) < 0)
        return -1;
    memcpy(out, cost0, sizeof(double) * (size_t)W * H * D);
    double *fine = out;
    for (int l = 1; l < levels; ++l) {
        double *coarse = fine + (size_t)Ws[l - 1] * Hs[l - 1] * D;
        for (int y = 0; y < Hs[l]; ++y)
            for (int x = 0; x < Ws[l]; ++x)
                for (int d = 0; d < D; ++d) {
                    double s = 0.0;
                    for (int dy = 0; dy < 2; ++dy)
                        for (int dx = 0; dx < 2; ++dx) {
                            const int fy = 2 * y + dy, fx = 2 * x + dx;
                            if (fy < Hs[l - 1] && fx < Ws[l - 1])
                                s += fine[((size_t)fy * Ws[l - 1] + fx) * D + d];
                        }
                    coarse[((size_t)y * Ws[l] + x) * D + d] = s;
                }
        fine = coarse;
    }
    return 0;
}

int oracle_pyramid_i32(const int32_t *cost0, int W, int H, int D, int levels, int32_t *out)
{
    int Ws[32], Hs[32];
    if (!cost0 || !out || D < 1 || levels > 32 || oracle_level_dims(W, H, levels, Ws, Hs) < 0)
        return -1;
    size_t total = 0;
    for (int l = 0; l < levels; ++l)
        total += (size_t)Ws[l] * Hs[l] * D;
    double *c = malloc(sizeof(double) * (size_t)W * H * D);
    double *p = malloc(sizeof(double) * total);
    if (!c || !p) {
        free(c);
        free(p);
        return -1;
    }
    for (size_t k = 0; k < (size_t)W * H * D; ++k)
        c[k] = cost0[k];
    oracle_pyramid_f64(c, W, H, D, levels, p);
    for (size_t k = 0; k < total; ++k)
        out[k] = (int32_t)p[k];
    free(c);
    free(p);
    return 0;
}

/* ---------------------------------------------------------------- message update (Fast Converging BP) */

void oracle_message_f64(const double *h, int D, double lambda, int trunc, double *m)
{
    double mn = INFINITY;
    for (int d = 0; d < D; ++d) {
        double best = INFINITY;
        for (int e = 0; e < D; ++e) {
            const int dist = abs(d - e);
            const double v = h[e] + lambda * (double)(dist < trunc ? dist : trunc);
            if (v < best)
                best = v;
        }
        m[d] = best;
        if (best < mn)
            mn = best;
    }
    for (int d = 0; d < D; ++d)
        m[d] -= mn;
}

void oracle_message_i32(const int32_t *h, int D, int lambda, int trunc, int32_t *m)
{
    if (D < 1)
        return;
    double *hd = malloc(sizeof(double) * 2 * (size_t)D);
    if (!hd)
        return;
    for (int d = 0; d < D; ++d)
        hd[d] = h[d];
    oracle_message_f64(hd, D, (double)lambda, trunc, hd + D);
    for (int d = 0; d < D; ++d)
        m[d] = (int32_t)hd[D + d];
    free(hd);
}

/* SplitMix64 step, used only to shuffle the update order inside a half-sweep. */
static uint64_t sm64(uint64_t *s)
{
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* One scale of red-black min-sum BP.  M: [4][H][W][D] incoming messages, updated in place.
 * Skip rule (with skip on): a pixel is recomputed while it is dirty.  A recomputed pixel
 * stores every outgoing message, and marks the receiver dirty when the new message differs
 * from the stored one by more than eps at some label (eps = 0: any change, the exact skip).
 * With freeze, a recomputed pixel that marked no receiver is frozen: it is not recomputed
 * again at this scale, dirty or not.  eps > 0 or freeze make the skip approximate. */
static int64_t *bp_level(const double *C, double *M, int W, int H, int D, int iters,
                         double lambda, int trunc, int skip, double eps, int freeze,
                         uint64_t order_seed, int64_t *trace)
{
    const size_t plane = (size_t)H * W * D;
    unsigned char *dirty = malloc((size_t)W * H);
    unsigned char *frozen = calloc((size_t)W * H, 1);
    int *order = malloc(sizeof(int) * ((size_t)W * H + 1));
    memset(dirty, 1, (size_t)W * H);
    uint64_t rng = order_seed;
    for (int it = 0; it < iters; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            /* the pixels of this colour, in raster order or a seeded permutation */
            int n = 0;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    if (((x + y) & 1) == colour)
                        order[n++] = y * W + x;
            if (order_seed)
                for (int k = n - 1; k > 0; --k) {
                    const int j = (int)(sm64(&rng) % (uint64_t)(k + 1));
                    const int t = order[k];
                    order[k] = order[j];
                    order[j] = t;
                }
            int64_t updated = 0;
#pragma omp parallel for schedule(static) reduction(+ : updated)
            for (int k = 0; k < n; ++k) {
                const int x = order[k] % W, y = order[k] / W;
                const size_t p = (size_t)y * W + x;
                if (skip && (!dirty[p] || frozen[p]))
                    continue;
                ++updated;
                int marked = 0;
                double b[D], h[D], m[D]; /* belief, message input, message */
                const int has[4] = {y > 0, y < H - 1, x > 0, x < W - 1};
                /* belief: data term plus every incoming message */
                for (int d = 0; d < D; ++d) {
                    double s = C[p * D + d];
                    for (int q = 0; q < 4; ++q)
                        if (has[q])
                            s += M[q * plane + p * D + d];
                    b[d] = s;
                }
                for (int q = 0; q < 4; ++q) {
                    if (!has[q])
                        continue;
                    /* the message to neighbour q leaves out what q sent */
                    for (int d = 0; d < D; ++d)
                        h[d] = b[d] - M[q * plane + p * D + d];
                    oracle_message_f64(h, D, lambda, trunc, m);
                    int qx = x, qy = y, slot;
                    switch (q) {
                    case UP: qy = y - 1; slot = DOWN; break;   /* p is q's lower neighbour */
                    case DOWN: qy = y + 1; slot = UP; break;
                    case LEFT: qx = x - 1; slot = RIGHT; break;
                    default: qx = x + 1; slot = LEFT; break;
                    }
                    double *dst = M + slot * plane + ((size_t)qy * W + qx) * D;
                    int changed = 0;
                    for (int d = 0; d < D; ++d) {
                        if (fabs(dst[d] - m[d]) > eps)
                            changed = 1;
                        dst[d] = m[d];
                    }
                    if (changed) {
                        /* q is of the other colour; several senders may mark it */
#pragma omp atomic write
                        dirty[(size_t)qy * W + qx] = 1;
                        marked = 1;
                    }
                }
                dirty[p] = 0;
                if (freeze && !marked)
                    frozen[p] = 1;
            }
            if (trace)
                *trace++ = updated;
        }
    free(dirty);
    free(frozen);
    free(order);
    return trace;
}

int oracle_bp_f64(const double *cost0, int W, int H, int D, int levels, int iters, double lambda,
                  int trunc, int skip, const double *init_coarsest, uint64_t order_seed,
                  double *msg0_out, int64_t *trace)
{
    return oracle_bp_rule_f64(cost0, W, H, D, levels, iters, lambda, trunc, skip, 0.0, 0, init_coarsest,
                              order_seed, msg0_out, trace);
}

/* The hierarchy of scales (section "GPU Implementation"): the cost pyramid, then every scale
 * coarsest first, each starting from its parent's messages.  Returns the finest scale's
 * messages [4][H][W][D] in a buffer the caller frees, or NULL on bad arguments or allocation
 * failure. */
static double *bp_hierarchy(const double *cost0, int W, int H, int D, int levels, const int *iters, double lambda,
                            int trunc, int skip, double eps, int freeze, const double *init_coarsest,
                            uint64_t order_seed, int64_t *trace)
{
    int Ws[32], Hs[32];
    if (!cost0 || !iters || D < 1 || levels > 32 || trunc < 0 || oracle_level_dims(W, H, levels, Ws, Hs) < 0)
        return NULL;
    for (int l = 0; l < levels; ++l)
        if (iters[l] < 0)
            return NULL;
    size_t off[33];
    off[0] = 0;
    for (int l = 0; l < levels; ++l)
        off[l + 1] = off[l] + (size_t)Ws[l] * Hs[l] * D;
    double *pyr = malloc(sizeof(double) * off[levels]);
    if (!pyr)
        return NULL;
    oracle_pyramid_f64(cost0, W, H, D, levels, pyr);
    double *parent = NULL;
    int64_t *tr = trace;
    for (int l = levels - 1; l >= 0; --l) {
        const int w = Ws[l], h = Hs[l];
        const size_t plane = (size_t)w * h * D;
        double *M = calloc(4 * plane, sizeof(double));
        if (!M) {
            free(pyr);
            free(parent);
            return NULL;
        }
        if (l == levels - 1) {
            if (init_coarsest)
                memcpy(M, init_coarsest, sizeof(double) * 4 * plane);
        } else {
            /* coarse-to-fine: each pixel starts from its parent's messages */
            const int pw = Ws[l + 1], ph = Hs[l + 1];
            const size_t pplane = (size_t)pw * ph * D;
            for (int q = 0; q < 4; ++q)
                for (int y = 0; y < h; ++y)
                    for (int x = 0; x < w; ++x)
                        memcpy(M + q * plane + ((size_t)y * w + x) * D,
                               parent + q * pplane + ((size_t)(y / 2) * pw + x / 2) * D,
                               sizeof(double) * D);
        }
        free(parent);
        tr = bp_level(pyr + off[l], M, w, h, D, iters[l], lambda, trunc, skip, eps, freeze, order_seed, tr);
        parent = M;
    }
    free(pyr);
    return parent;
}

int oracle_bp_rule_f64(const double *cost0, int W, int H, int D, int levels, int iters, double lambda,
                       int trunc, int skip, double eps, int freeze, const double *init_coarsest,
                       uint64_t order_seed, double *msg0_out, int64_t *trace)
{
    if (!msg0_out || iters < 0 || levels < 1 || levels > 32)
        return -1;
    int it[32];
    for (int l = 0; l < levels; ++l)
        it[l] = iters;
    double *M = bp_hierarchy(cost0, W, H, D, levels, it, lambda, trunc, skip, eps, freeze, init_coarsest,
                             order_seed, trace);
    if (!M)
        return -1;
    memcpy(msg0_out, M, sizeof(double) * 4 * (size_t)W * H * D);
    free(M);
    return 0;
}

int oracle_bp_wta_f64(const double *cost0, int W, int H, int D, int levels, int iters, double lambda, int trunc,
                      int skip, int32_t *disp, int64_t *trace)
{
    if (!disp || iters < 0 || levels < 1 || levels > 32)
        return -1;
    int it[32];
    for (int l = 0; l < levels; ++l)
        it[l] = iters;
    double *M = bp_hierarchy(cost0, W, H, D, levels, it, lambda, trunc, skip, 0.0, 0, NULL, 0, trace);
    if (!M)
        return -1;
    const int rc = oracle_wta_f64(cost0, M, W, H, D, disp);
    free(M);
    return rc;
}

int oracle_bp_schedule_i32(const int32_t *cost0, int W, int H, int D, int levels, const int *iters, int lambda,
                           int trunc, int skip, const int32_t *init_coarsest, int32_t *msg0_out, int64_t *trace)
{
    int Ws[32], Hs[32];
    if (!cost0 || !msg0_out || !iters || W < 1 || H < 1 || D < 1 || levels < 1 || levels > 32 ||
        oracle_level_dims(W, H, levels, Ws, Hs) < 0)
        return -1;
    const size_t n0 = (size_t)W * H * D;
    const size_t nc = (size_t)Ws[levels - 1] * Hs[levels - 1] * D;
    double *c = malloc(sizeof(double) * n0);
    double *init = init_coarsest ? malloc(sizeof(double) * 4 * nc) : NULL;
    if (!c || (init_coarsest && !init)) {
        free(c);
        free(init);
        return -1;
    }
    for (size_t k = 0; k < n0; ++k)
        c[k] = cost0[k];
    if (init)
        for (size_t k = 0; k < 4 * nc; ++k)
            init[k] = init_coarsest[k];
    double *M = bp_hierarchy(c, W, H, D, levels, iters, (double)lambda, trunc, skip, 0.0, 0, init, 0, trace);
    free(c);
    free(init);
    if (!M)
        return -1;
    for (size_t k = 0; k < 4 * n0; ++k)
        msg0_out[k] = (int32_t)M[k];
    free(M);
    return 0;
}

int oracle_bp_wta_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda, int trunc,
                      int skip, int32_t *disp, int64_t *trace)
{
    if (!cost0 || !disp || W < 1 || H < 1 || D < 1)
        return -1;
    const size_t n0 = (size_t)W * H * D;
    double *c = malloc(sizeof(double) * n0);
    if (!c)
        return -1;
    for (size_t k = 0; k < n0; ++k)
        c[k] = cost0[k];
    /* every value is an exact integer in FP64, so the FP64 argmin (lowest d on ties) is the
     * integer read-out */
    const int rc = oracle_bp_wta_f64(c, W, H, D, levels, iters, (double)lambda, trunc, skip, disp, trace);
    free(c);
    return rc;
}

int oracle_bp_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda,
                  int trunc, int skip, const int32_t *init_coarsest, uint64_t order_seed,
                  int32_t *msg0_out, int64_t *trace)
{
    return oracle_bp_rule_i32(cost0, W, H, D, levels, iters, lambda, trunc, skip, 0, 0, init_coarsest,
                              order_seed, msg0_out, trace);
}

int oracle_bp_rule_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda,
                       int trunc, int skip, int eps, int freeze, const int32_t *init_coarsest,
                       uint64_t order_seed, int32_t *msg0_out, int64_t *trace)
{
    int Ws[32], Hs[32];
    if (!cost0 || !msg0_out || D < 1 || levels > 32 || oracle_level_dims(W, H, levels, Ws, Hs) < 0)
        return -1;
    const size_t n0 = (size_t)W * H * D;
    const size_t nc = (size_t)Ws[levels - 1] * Hs[levels - 1] * D;
    double *c = malloc(sizeof(double) * n0);
    double *m = malloc(sizeof(double) * 4 * n0);
    double *init = init_coarsest ? malloc(sizeof(double) * 4 * nc) : NULL;
    if (!c || !m || (init_coarsest && !init)) {
        free(c);
        free(m);
        free(init);
        return -1;
    }
    for (size_t k = 0; k < n0; ++k)
        c[k] = cost0[k];
    if (init)
        for (size_t k = 0; k < 4 * nc; ++k)
            init[k] = init_coarsest[k];
    const int rc = oracle_bp_rule_f64(c, W, H, D, levels, iters, (double)lambda, trunc, skip, (double)eps,
                                      freeze, init, order_seed, m, trace);
    for (size_t k = 0; k < 4 * n0; ++k)
        msg0_out[k] = (int32_t)m[k];
    free(c);
    free(m);
    free(init);
    return rc;
}

/* ---------------------------------------------------------------- sparse candidates */

int oracle_candidates(const int32_t *cost0, int W, int H, int D, int K, int32_t *cand)
{
    if (!cost0 || !cand || W < 1 || H < 1 || K < 1 || K > D)
        return -1;
    unsigned char *taken = malloc((size_t)D);
    if (!taken)
        return -1;
    for (size_t p = 0; p < (size_t)W * H; ++p) {
        const int32_t *c = cost0 + p * D;
        int32_t *out = cand + p * K;
        memset(taken, 0, (size_t)D);
        /* the K smallest costs, the lower label first among equal costs */
        for (int k = 0; k < K; ++k) {
            int best = -1;
            for (int d = 0; d < D; ++d)
                if (!taken[d] && (best < 0 || c[d] < c[best]))
                    best = d;
            taken[best] = 1;
            out[k] = best;
        }
        /* listed in increasing label order */
        for (int a = 1; a < K; ++a)
            for (int b = a; b > 0 && out[b - 1] > out[b]; --b) {
                const int32_t t = out[b];
                out[b] = out[b - 1];
                out[b - 1] = t;
            }
    }
    free(taken);
    return 0;
}

/* The finest scale over candidate sets.  M: [4][H][W][K] incoming messages, indexed like the
 * candidates of the receiving pixel. */
static int64_t *bp_sparse_level(const double *C, const int32_t *cand, double *M, int W, int H, int D,
                                int K, int iters, double lambda, int trunc, int skip, int64_t *trace)
{
    const size_t plane = (size_t)H * W * K;
    double *b = malloc(sizeof(double) * (size_t)K);
    double *h = malloc(sizeof(double) * (size_t)K);
    double *m = malloc(sizeof(double) * (size_t)K);
    unsigned char *dirty = malloc((size_t)W * H);
    memset(dirty, 1, (size_t)W * H);
    for (int it = 0; it < iters; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            int64_t updated = 0;
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x) {
                    if (((x + y) & 1) != colour)
                        continue;
                    const size_t p = (size_t)y * W + x;
                    if (skip && !dirty[p])
                        continue;
                    ++updated;
                    const int has[4] = {y > 0, y < H - 1, x > 0, x < W - 1};
                    const int32_t *cp = cand + p * K;
                    for (int i = 0; i < K; ++i) {
                        double s = C[p * D + cp[i]];
                        for (int q = 0; q < 4; ++q)
                            if (has[q])
                                s += M[q * plane + p * K + i];
                        b[i] = s;
                    }
                    for (int q = 0; q < 4; ++q) {
                        if (!has[q])
                            continue;
                        int qx = x, qy = y, slot;
                        switch (q) {
                        case UP: qy = y - 1; slot = DOWN; break;
                        case DOWN: qy = y + 1; slot = UP; break;
                        case LEFT: qx = x - 1; slot = RIGHT; break;
                        default: qx = x + 1; slot = LEFT; break;
                        }
                        const size_t r = (size_t)qy * W + qx;
                        const int32_t *cr = cand + r * K;
                        for (int i = 0; i < K; ++i)
                            h[i] = b[i] - M[q * plane + p * K + i];
                        /* m(j) = min over p's candidates i of h(i) + lambda*min(|label_i - label_j|, T) */
                        double mn = INFINITY;
                        for (int j = 0; j < K; ++j) {
                            double v = INFINITY;
                            for (int i = 0; i < K; ++i) {
                                const int dd = abs(cp[i] - cr[j]);
                                const double t = h[i] + lambda * (double)(dd < trunc ? dd : trunc);
                                if (t < v)
                                    v = t;
                            }
                            m[j] = v;
                            if (v < mn)
                                mn = v;
                        }
                        double *dst = M + slot * plane + r * K;
                        int changed = 0;
                        for (int j = 0; j < K; ++j) {
                            const double v = m[j] - mn;
                            if (dst[j] != v)
                                changed = 1;
                            dst[j] = v;
                        }
                        if (changed)
                            dirty[r] = 1;
                    }
                    dirty[p] = 0;
                }
            if (trace)
                *trace++ = updated;
        }
    free(b);
    free(h);
    free(m);
    free(dirty);
    return trace;
}

int oracle_bp_sparse_i32(const int32_t *cost0, int W, int H, int D, int levels, int iters, int lambda,
                         int trunc, int skip, int K, int32_t *cand_out, int32_t *msg_out, int64_t *trace)
{
    int Ws[32], Hs[32];
    if (!cost0 || !cand_out || !msg_out || D < 1 || K < 1 || K > D || levels < 1 || levels > 32 || iters < 0 ||
        trunc < 0 || oracle_level_dims(W, H, levels, Ws, Hs) < 0)
        return -1;
    if (oracle_candidates(cost0, W, H, D, K, cand_out) != 0)
        return -1;
    size_t off[33];
    off[0] = 0;
    for (int l = 0; l < levels; ++l)
        off[l + 1] = off[l] + (size_t)Ws[l] * Hs[l] * D;
    const size_t n0 = (size_t)W * H * D;
    double *c = malloc(sizeof(double) * n0);
    double *pyr = malloc(sizeof(double) * off[levels]);
    if (!c || !pyr) {
        free(c);
        free(pyr);
        return -1;
    }
    for (size_t k = 0; k < n0; ++k)
        c[k] = cost0[k];
    oracle_pyramid_f64(c, W, H, D, levels, pyr);
    /* scales levels-1 .. 1: the dense hierarchical solve */
    double *parent = NULL;
    int64_t *tr = trace;
    for (int l = levels - 1; l >= 1; --l) {
        const int w = Ws[l], h = Hs[l];
        const size_t plane = (size_t)w * h * D;
        double *M = calloc(4 * plane, sizeof(double));
        if (l < levels - 1) {
            const int pw = Ws[l + 1], ph = Hs[l + 1];
            const size_t pplane = (size_t)pw * ph * D;
            for (int q = 0; q < 4; ++q)
                for (int y = 0; y < h; ++y)
                    for (int x = 0; x < w; ++x)
                        memcpy(M + q * plane + ((size_t)y * w + x) * D,
                               parent + q * pplane + ((size_t)(y / 2) * pw + x / 2) * D, sizeof(double) * D);
        }
        free(parent);
        tr = bp_level(pyr + off[l], M, w, h, D, iters, (double)lambda, trunc, skip, 0.0, 0, 0, tr);
        parent = M;
    }
    /* the finest scale: each candidate starts from the parent's message at its label */
    const size_t splane = (size_t)W * H * K;
    double *M = calloc(4 * splane, sizeof(double));
    if (parent) {
        const int pw = Ws[1], ph = Hs[1];
        const size_t pplane = (size_t)pw * ph * D;
        for (int q = 0; q < 4; ++q)
            for (int y = 0; y < H; ++y)
                for (int x = 0; x < W; ++x)
                    for (int j = 0; j < K; ++j) {
                        const size_t p = (size_t)y * W + x;
                        M[q * splane + p * K + j] =
                            parent[q * pplane + ((size_t)(y / 2) * pw + x / 2) * D + cand_out[p * K + j]];
                    }
    }
    free(parent);
    bp_sparse_level(pyr, cand_out, M, W, H, D, K, iters, (double)lambda, trunc, skip, tr);
    for (size_t k = 0; k < 4 * splane; ++k)
        msg_out[k] = (int32_t)M[k];
    free(M);
    free(pyr);
    free(c);
    return 0;
}

int oracle_wta_sparse_i32(const int32_t *cost0, const int32_t *cand, const int32_t *msg, int W, int H, int D,
                          int K, int32_t *disp)
{
    if (!cost0 || !cand || !msg || !disp || W < 1 || H < 1 || K < 1 || K > D)
        return -1;
    const size_t plane = (size_t)W * H * K;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const int has[4] = {y > 0, y < H - 1, x > 0, x < W - 1};
            int64_t best = INT64_MAX;
            int arg = 0;
            for (int j = 0; j < K; ++j) { /* increasing labels: the lowest label wins ties */
                int64_t s = cost0[p * D + cand[p * K + j]];
                for (int q = 0; q < 4; ++q)
                    if (has[q])
                        s += msg[q * plane + p * K + j];
                if (s < best) {
                    best = s;
                    arg = cand[p * K + j];
                }
            }
            disp[p] = arg;
        }
    return 0;
}

/* ---------------------------------------------------------------- read-out and energy */

int oracle_wta_f64(const double *cost, const double *msg, int W, int H, int D, int32_t *disp)
{
    if (!cost || !msg || !disp || W < 1 || H < 1 || D < 1)
        return -1;
    const size_t plane = (size_t)W * H * D;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const int has[4] = {y > 0, y < H - 1, x > 0, x < W - 1};
            double best = INFINITY;
            int arg = 0;
            for (int d = 0; d < D; ++d) {
                double s = cost[p * D + d];
                for (int q = 0; q < 4; ++q)
                    if (has[q])
                        s += msg[q * plane + p * D + d];
                if (s < best) {
                    best = s;
                    arg = d;
                }
            }
            disp[p] = arg;
        }
    return 0;
}

int oracle_wta_i32(const int32_t *cost, const int32_t *msg, int W, int H, int D, int32_t *disp)
{
    if (!cost || !msg || !disp || W < 1 || H < 1 || D < 1)
        return -1;
    const size_t plane = (size_t)W * H * D;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const int has[4] = {y > 0, y < H - 1, x > 0, x < W - 1};
            int64_t best = INT64_MAX;
            int arg = 0;
            for (int d = 0; d < D; ++d) {
                int64_t s = cost[p * D + d];
                for (int q = 0; q < 4; ++q)
                    if (has[q])
                        s += msg[q * plane + p * D + d];
                if (s < best) {
                    best = s;
                    arg = d;
                }
            }
            disp[p] = arg;
        }
    return 0;
}

static int smooth_cost(int a, int b, int trunc)
{
    const int dist = abs(a - b);
    return dist < trunc ? dist : trunc;
}

int64_t oracle_energy_i32(const int32_t *cost, const int32_t *disp, int W, int H, int D,
                          int lambda, int trunc)
{
    if (!cost || !disp || W < 1 || H < 1 || D < 1)
        return INT64_MIN;
    int64_t e = 0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const int d = disp[p];
            if (d < 0 || d >= D)
                return INT64_MIN;
            e += cost[p * D + d];
            if (x + 1 < W)
                e += (int64_t)lambda * smooth_cost(d, disp[p + 1], trunc);
            if (y + 1 < H)
                e += (int64_t)lambda * smooth_cost(d, disp[p + W], trunc);
        }
    return e;
}

double oracle_energy_f64(const double *cost, const int32_t *disp, int W, int H, int D,
                         double lambda, int trunc)
{
    if (!cost || !disp || W < 1 || H < 1 || D < 1)
        return NAN;
    double e = 0.0;
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            const size_t p = (size_t)y * W + x;
            const int d = disp[p];
            if (d < 0 || d >= D)
                return NAN;
            e += cost[p * D + d];
            if (x + 1 < W)
                e += lambda * smooth_cost(d, disp[p + 1], trunc);
            if (y + 1 < H)
                e += lambda * smooth_cost(d, disp[p + W], trunc);
        }
    return e;
}
