// ncc.cu -- matching-cost volume (section "Correlation volume computation") and the
// cost pyramid of the hierarchical scheme (section "GPU Implementation").
//
// ncc_cost_kernel: one CTA per 32 x 4 pixel tile, all labels.  The left tile and the right
// strip it can match ([x0 - r - (D-1), x0 + 32 + r)) are staged in shared memory with
// replicate-clamped coordinates.  Window sums are exact integers: S_a, S_aa per left
// pixel and S_b, S_bb per right position; S_ab per (pixel, label) is separable: first a
// vertical sum of L*R over the window rows for every staged column, then a horizontal
// sum over the window columns.
//
// Quantiser c = clamp(floor(T (1 - ncc) + 1/2), 0, T).  GB300's FP64 rate is low, so the
// decision is taken in fp32 first, with correctly rounded operations whose worst-case
// error on v = T (1 - ncc) + 1/2 is below 2^-19 (T + 1) (each rounded step adds at most
// 2^-24 relative, the reciprocal square root halves its input's error; |ncc| <= 1).  Only where v lies within (T + 1) 2^-13 of an integer
// is the decision re-taken with the exact FP64 sequence (correctly rounded multiply,
// square root, divide, subtract, multiply, add, floor).  Outside that margin both
// computations fall on the same side of every integer, so the result equals the FP64
// decision everywhere.
#include <algorithm>
#include <type_traits>

#include "bps_internal.cuh"
#include "bps_launch.h"
#include "ncc_quant.cuh"

namespace bps {

constexpr int NCC_TX = 32, NCC_TY = 4, NCC_DC = 32, NCC_THREADS = 256;

__device__ inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <typename CostT> struct CostOut;
template <> struct CostOut<int32_t> { static constexpr bool is_float = false; };
template <> struct CostOut<int16_t> { static constexpr bool is_float = false; };
template <> struct CostOut<float> { static constexpr bool is_float = true; };

__device__ inline int quantise_exact(long long num, long long va, long long vb, int T, float *ncc_f) {
    if (va == 0 || vb == 0) {
        *ncc_f = 0.f;
        return T;  // floor(T + 1/2) for an integer T
    }
    const float pf = __fmul_rn((float)va, (float)vb);
    const float nccf = __fmul_rn((float)num, __frsqrt_rn(pf));
    *ncc_f = nccf;
    const float v = __fadd_rn(__fmul_rn((float)T, __fsub_rn(1.f, nccf)), 0.5f);
    const float fl = floorf(v);
    const float dist = fminf(v - fl, fl + 1.f - v);
    int c;
    if (dist > (float)(T + 1) * (1.f / 8192.f)) {
        c = (int)fl;
    } else {
        const double den = __dmul_rn((double)va, (double)vb);
        const double n64 = __ddiv_rn((double)num, __dsqrt_rn(den));
        const double w = __dadd_rn(__dmul_rn((double)T, __dadd_rn(1.0, -n64)), 0.5);
        c = (int)floor(w);
    }
    return c < 0 ? 0 : (c > T ? T : c);
}

template <typename CostT>
__global__ void __launch_bounds__(NCC_THREADS)
ncc_cost_kernel(const uint8_t *__restrict__ L, const uint8_t *__restrict__ R, int pitch, int W, int H,
                int D, int Dp, int window, int T, int Wh, CostT *cost0, CostT *cost1, float *ncc_out) {
    extern __shared__ __align__(16) unsigned char smem[];
    pdl_enter();
    const int r = window / 2;
    const int TW = NCC_TX + 2 * r;          // staged left columns
    const int RW = TW + D - 1;              // staged right columns
    const int SH = NCC_TY + 2 * r;          // staged rows
    const int UW = NCC_TX + D - 1;          // right window positions u = x0 - (D-1) + uu
    const int CS = NCC_TY * TW + 1;         // padded stride of one label's column sums
    const int x0 = blockIdx.x * NCC_TX, y0 = blockIdx.y * NCC_TY;
    const long long N = (long long)window * window;

    int *SA = reinterpret_cast<int *>(smem);
    int *SAA = SA + NCC_TY * NCC_TX;
    int *SB = SAA + NCC_TY * NCC_TX;
    int *SBB = SB + NCC_TY * UW;
    int *colsum = SBB + NCC_TY * UW;                                       // [NCC_DC][CS]
    uint8_t *Ls = reinterpret_cast<uint8_t *>(colsum + NCC_DC * CS);        // [SH][TW]
    uint8_t *Rs = Ls + SH * TW;                                            // [SH][RW]

    for (int k = threadIdx.x; k < SH * TW; k += blockDim.x) {
        const int jj = k / TW, ii = k % TW;
        Ls[k] = L[(size_t)clampi(y0 - r + jj, 0, H - 1) * pitch + clampi(x0 - r + ii, 0, W - 1)];
    }
    for (int k = threadIdx.x; k < SH * RW; k += blockDim.x) {
        const int jj = k / RW, ii = k % RW;
        Rs[k] = R[(size_t)clampi(y0 - r + jj, 0, H - 1) * pitch + clampi(x0 - r - (D - 1) + ii, 0, W - 1)];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < NCC_TY * NCC_TX; k += blockDim.x) {
        const int ty = k / NCC_TX, tx = k % NCC_TX;
        int s = 0, ss = 0;
        for (int j = 0; j < window; ++j)
            for (int i = 0; i < window; ++i) {
                const int a = Ls[(ty + j) * TW + tx + i];
                s += a;
                ss += a * a;
            }
        SA[k] = s;
        SAA[k] = ss;
    }
    for (int k = threadIdx.x; k < NCC_TY * UW; k += blockDim.x) {
        const int ty = k / UW, uu = k % UW;
        int s = 0, ss = 0;
        for (int j = 0; j < window; ++j)
            for (int i = 0; i < window; ++i) {
                const int b = Rs[(ty + j) * RW + uu + i];
                s += b;
                ss += b * b;
            }
        SB[k] = s;
        SBB[k] = ss;
    }
    __syncthreads();

    for (int d0 = 0; d0 < Dp; d0 += NCC_DC) {
        const int dc = min(NCC_DC, Dp - d0);
        // vertical sums of L * R over the window rows, every staged column, dc labels
        for (int k = threadIdx.x; k < dc * NCC_TY * TW; k += blockDim.x) {
            const int col = k % TW, rest = k / TW;
            const int ty = rest % NCC_TY, dd = rest / NCC_TY;
            const int d = min(d0 + dd, D - 1);
            int s = 0;
            for (int j = 0; j < window; ++j)
                s += (int)Ls[(ty + j) * TW + col] * (int)Rs[(ty + j) * RW + col + (D - 1) - d];
            colsum[dd * CS + ty * TW + col] = s;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < dc * NCC_TY * NCC_TX; k += blockDim.x) {
            const int dd = k % dc, px = k / dc;
            const int tx = px % NCC_TX, ty = px / NCC_TX;
            const int x = x0 + tx, y = y0 + ty, d = d0 + dd;
            if (x >= W || y >= H) continue;
            const int c = colour_of(x, y);
            CostT *dst = (c ? cost1 : cost0) + slot_of(x, y, Wh) * Dp + label_pos<CostT>(d);
            if (d >= D) {
                *dst = CostT(0);
                continue;
            }
            int sab = 0;
            const int *cs = colsum + dd * CS + ty * TW + tx;
            for (int i = 0; i < window; ++i) sab += cs[i];
            const int uu = tx - d + (D - 1);
            const long long sa = SA[ty * NCC_TX + tx], saa = SAA[ty * NCC_TX + tx];
            const long long sb = SB[ty * UW + uu], sbb = SBB[ty * UW + uu];
            const long long num = N * sab - sa * sb;
            const long long va = N * saa - sa * sa;
            const long long vb = N * sbb - sb * sb;
            float nccf;
            if constexpr (CostOut<CostT>::is_float) {
                nccf = (va == 0 || vb == 0) ? 0.f
                                            : __fmul_rn((float)num, __frsqrt_rn(__fmul_rn((float)va, (float)vb)));
                const float v = (float)T * (1.f - nccf);
                *dst = fminf(fmaxf(v, 0.f), (float)T);
            } else {
                *dst = (CostT)quantise_exact(num, va, vb, T, &nccf);
            }
            if (ncc_out) ncc_out[((size_t)y * W + x) * D + d] = nccf;
        }
        __syncthreads();
    }
}

// The dynamic shared-memory limit is a property of the kernel function, shared by every
// context in the process, so it is raised once to the device's opt-in maximum; each launch
// still requests only what its shape needs.
static int smem_optin() {
    int dev = 0, v = 48 * 1024;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

// ------------------------------------------------------------------ row-streaming NCC (windows up to 15)
// ncc_rows_kernel: a CTA owns a strip of rows [y0, y0 + TYS) and XS * 16 columns; thread
// (label d, column group xs) owns 16 consecutive columns at one label.
//
// Every staged column (left: the CTA's columns and the horizontal window margin; right: the
// positions those can match) keeps the 2R + 1 image bytes of its current window rows packed
// in NW = ceil((2R + 1) / 4) 32-bit words, a shift register held by the thread that owns the
// column: one byte enters per row.  The owner publishes the words to shared memory each row,
// with the column's sum and sum of squares (4-way byte dot products with ones and with the
// words themselves).  The vertical window sum of L(x') R(x' - d) of a column is then NW
// byte dot products (dp4a) of the left and the right words, with no running state, so a
// strip needs no per-label warm-up rows (only the owners shift in the 2R rows above the
// strip).  Each thread slides the horizontal window over those column sums for its 16
// outputs.  Per pixel and per right position the CTA forms once the window sum S, the
// variance term N S_xx - S_x^2 and its reciprocal square root (correctly rounded).  The data
// cost of each (pixel, label) then needs one multiply-add for the numerator and two
// multiplies for the correlation.  The 2x2 sum of the next scale is accumulated over row
// pairs in registers and written directly (scale 1 of the pyramid).
//
// Quantiser: one fused multiply-add forms v = T (1 - ncc) + 1/2 in fp32 within (T + 1) 2^-20
// of its exact value (see quantise_fp32); the FP64 sequence decides only where v lies within
// (T + 1) 2^-17 of an integer, after the row, for the few outputs that need it.
constexpr int NR_TX = 16;
constexpr int NR_ITEMS_MAX = 4;  // staged columns per thread at most (checked by the launcher)
#ifndef NCC_ROWS_MAXNREG
#define NCC_ROWS_MAXNREG 80  // registers a thread: 24 warps on an SM, CTAs of up to 512 threads
#endif

// Words of a packed column window: (2R + 1) bytes, padded to 1, 2 or 4 words so that one
// shared load fetches a column.
template <int R> struct WinWords {
    static constexpr int NW = (2 * R + 1 + 3) / 4;
    static constexpr int NWP = NW <= 1 ? 1 : (NW <= 2 ? 2 : 4);
};
template <int NWP> struct alignas(4 * NWP) Win { uint32_t w[NWP]; };

// A store under a predicate, without a branch around it.
__device__ __forceinline__ void store_if(int16_t *p, int16_t v, bool pred) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.u16 [%0], %1;\n\t}" ::"l"(p),
                 "h"(v), "r"((unsigned)pred)
                 : "memory");
}
__device__ __forceinline__ void store_if(int32_t *p, int32_t v, bool pred) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.u32 [%0], %1;\n\t}" ::"l"(p),
                 "r"(v), "r"((unsigned)pred)
                 : "memory");
}

template <typename CostT, int R, bool NCC_OUT, int NR_ITEMS>
__global__ void __maxnreg__(NCC_ROWS_MAXNREG)
ncc_rows_kernel(const uint8_t *__restrict__ Limg, const uint8_t *__restrict__ Rimg, int pitch, int W, int H, int D,
                int Dp, int T, int TYS, LevelView l0, LevelView l1, int write_l1, float *ncc_out) {
    // blockDim.x = XS * Dp: XS column groups of 16, all labels.  Rows are processed in pairs
    // (y, y + 1), y even: one shift-and-publish phase and one record phase per pair, each followed
    // by a CTA barrier, then the outputs of both rows, whose 2x2 sums complete scale 1 at once.
    using Num = typename NccInt<R>::type;
    constexpr int WIN = 2 * R + 1;
    constexpr int NW = WinWords<R>::NW, NWP = WinWords<R>::NWP;
    constexpr bool FLOAT_COST = CostOut<CostT>::is_float;
    using WinT = Win<NWP>;
    extern __shared__ __align__(16) unsigned char smem[];
    const int XS = blockDim.x / Dp;
    const int CW = XS * NR_TX;
    const int LW = CW + 2 * R, RW = CW + 2 * R + D - 1, UW = CW + D - 1;
    const int dl = threadIdx.x % Dp, xs = threadIdx.x / Dp;
    const int d = min(dl, D - 1);
    const int x0 = blockIdx.x * CW, y0 = blockIdx.y * TYS, y1 = min(H, y0 + TYS);
    const int N = WIN * WIN;

    // per row h of the pair: the records the outputs read, {S, T / sqrt(N S_xx - S_x^2)} per left
    // pixel and {S, 1 / sqrt(...)} per right position (8 bytes: one shared load each per output),
    // and the ones only the FP64 decision and the correlation output read, {N S_xx - S_x^2, 1 / sqrt}
    int2 *PA = reinterpret_cast<int2 *>(smem);       // [2][CW]  left window at pixel x0 + i
    int2 *PB = PA + 2 * CW;                          // [2][UW]  right window at u = x0 - (D-1) + i
    int2 *QA = PB + 2 * UW;                          // [2][CW]
    int2 *QB = QA + 2 * CW;                          // [2][UW]
    WinT *LWn = reinterpret_cast<WinT *>(QB + 2 * UW);  // [4][LW] packed left column windows (by row & 3)
    WinT *RWn = LWn + 4 * LW;                        // [4][RW] ... right
    int *colA = reinterpret_cast<int *>(RWn + 4 * RW);  // [2][LW]  column sums of L over the window rows
    int *colAA = colA + 2 * LW;                      // [2][LW]
    int *colB = colAA + 2 * LW;                      // [2][RW]
    int *colBB = colB + 2 * RW;                      // [2][RW]

    // the staged columns this thread owns: item k is column tid + k * blockDim of the left
    // (index < LW) or the right (index - LW) image
    const int items = LW + RW;
    const int nk = (items - (int)threadIdx.x + (int)blockDim.x - 1) / (int)blockDim.x;  // items of this thread
    uint32_t win[NR_ITEMS][NWP];
    int col[NR_ITEMS];  // the item's clamped image column
#pragma unroll
    for (int k = 0; k < NR_ITEMS; ++k) {
#pragma unroll
        for (int w = 0; w < NWP; ++w) win[k][w] = 0u;
        const int it = threadIdx.x + k * blockDim.x;
        col[k] = it < LW ? clampi(x0 - R + it, 0, W - 1) : clampi(x0 - R - (D - 1) + (it - LW), 0, W - 1);
    }
    auto load_row = [&](int e, uint32_t (&bytes)[NR_ITEMS]) {
        const int row = clampi(e, 0, H - 1) * pitch;
#pragma unroll
        for (int k = 0; k < NR_ITEMS; ++k) {
            const int it = threadIdx.x + k * blockDim.x;
            bytes[k] = k < nk ? (uint32_t)__ldg((it < LW ? Limg : Rimg) + row + col[k]) : 0u;
        }
    };
    auto shift_in = [&](const uint32_t (&bytes)[NR_ITEMS]) {
#pragma unroll
        for (int k = 0; k < NR_ITEMS; ++k) {
#pragma unroll
            for (int w = 0; w < NWP; ++w) win[k][w] = __funnelshift_r(win[k][w], w + 1 < NWP ? win[k][w + 1] : 0u, 8);
            win[k][(WIN - 1) / 4] |= bytes[k] << (8 * ((WIN - 1) % 4));
        }
    };
    // publish the owned windows (row buffer wb) and their column sums (column buffer h)
    auto publish = [&](int wb, int h) {
#pragma unroll
        for (int k = 0; k < NR_ITEMS; ++k) {
            if (k >= nk) break;
            const int it = threadIdx.x + k * blockDim.x;
            unsigned s = 0u, ss = 0u;
            WinT wv;
#pragma unroll
            for (int w = 0; w < NWP; ++w) {
                wv.w[w] = win[k][w];
                if (w < NW) {
                    s = __dp4a(win[k][w], 0x01010101u, s);
                    ss = __dp4a(win[k][w], win[k][w], ss);
                }
            }
            if (it < LW) {
                LWn[wb * LW + it] = wv;
                colA[h * LW + it] = (int)s;
                colAA[h * LW + it] = (int)ss;
            } else {
                RWn[wb * RW + it - LW] = wv;
                colB[h * RW + it - LW] = (int)s;
                colBB[h * RW + it - LW] = (int)ss;
            }
        }
    };

    pdl_enter();
    // the 2R rows above the strip enter the owners' windows first
    uint32_t next0[NR_ITEMS], next1[NR_ITEMS];
    for (int e = y0 - R; e < y0 + R; ++e) {
        load_row(e, next0);
        shift_in(next0);
    }
    load_row(y0 + R, next0);
    load_row(y0 + 1 + R, next1);

    int acc[NR_TX / 2];
    const int lbase = xs * NR_TX;               // this thread's first staged left column
    const int rbase = xs * NR_TX + D - 1 - d;   // ... and the right column matching it at label d
    const int xb = x0 + lbase;
    const int nvalid = min(NR_TX, W - xb);      // columns of this thread inside the image
    const bool lab = dl < D;
    const float T_half = (float)T + 0.5f, half_m = 0.5f - (float)(T + 1) * (1.f / 131072.f);

    for (int y = y0; y < y1; y += 2) {
        const int nrows = min(2, y1 - y);  // 1 only for the last row of an odd image height
        // phase 1: the owners shift rows y + R and y + 1 + R in, publish the words and the column sums
        {
            uint32_t cur0[NR_ITEMS], cur1[NR_ITEMS];
#pragma unroll
            for (int k = 0; k < NR_ITEMS; ++k) {
                cur0[k] = next0[k];
                cur1[k] = next1[k];
            }
            if (y + 2 < y1) {  // the next pair's rows are in flight during this pair
                load_row(y + 2 + R, next0);
                load_row(y + 3 + R, next1);
            }
            shift_in(cur0);
            publish(y & 3, 0);
            if (nrows == 2) {
                shift_in(cur1);
                publish((y + 1) & 3, 1);
            }
        }
        __syncthreads();
        // phase 2: window records of every left pixel and every right position, both rows
        for (int i = threadIdx.x; i < nrows * (CW + UW); i += blockDim.x) {
            const int h = i >= CW + UW ? 1 : 0;
            const int k = i - h * (CW + UW);
            const bool left = k < CW;
            const int c = left ? k : k - CW;
            const int *cs = left ? colA + h * LW + c : colB + h * RW + c;
            const int *css = left ? colAA + h * LW + c : colBB + h * RW + c;
            int s = 0, ss = 0;
#pragma unroll
            for (int q = 0; q < WIN; ++q) {
                s += cs[q];
                ss += css[q];
            }
            const unsigned v = (unsigned)N * (unsigned)ss - (unsigned)s * (unsigned)s;
            const float r = v ? rsqrtf((float)v) : 0.f;
            if (left) {
                PA[h * CW + c] = make_int2(s, __float_as_int(__fmul_rn((float)T, r)));
                QA[h * CW + c] = make_int2((int)v, __float_as_int(r));
            } else {
                PB[h * UW + c] = make_int2(s, __float_as_int(r));
                QB[h * UW + c] = make_int2((int)v, 0);
            }
        }
        __syncthreads();
        // phase 3: this thread's 16 outputs at label dl, in each row of the pair
        if constexpr (!FLOAT_COST) {
#pragma unroll
            for (int i = 0; i < NR_TX / 2; ++i) acc[i] = 0;
        }
        for (int h = 0; h < nrows; ++h) {
            const int yy = y + h;
            const WinT *Lrow = LWn + (yy & 3) * LW + lbase;
            const WinT *Rrow = RWn + (yy & 3) * RW + rbase;
            const int2 *pa_row = PA + h * CW + lbase;
            const int2 *pb_row = PB + h * UW + lbase + D - 1 - d;
            // the window's column dot products (L x R over the 2R + 1 rows): a ring of the last
            // 2R + 1, each formed when it enters the horizontal window (fewer live registers)
            auto dot = [&](int i) {
                const WinT a = Lrow[i], b = Rrow[i];
                unsigned v = 0u;
#pragma unroll
                for (int w = 0; w < NW; ++w) v = __dp4a(a.w[w], b.w[w], v);
                return (int)v;
            };
            int V[WIN];
#pragma unroll
            for (int i = 0; i < WIN; ++i) V[i] = dot(i);
            // destinations: x0 + lbase is even, so column j has colour (j + yy) & 1 and slot
            // row_slot + j / 2 in that colour's array
            const int64_t row_slot = (int64_t)yy * l0.Wh + (xb >> 1);
            CostT *const base_even = reinterpret_cast<CostT *>((yy & 1) ? l0.cost[1] : l0.cost[0]) + row_slot * Dp +
                                     label_pos<CostT>(dl);
            CostT *const base_odd = reinterpret_cast<CostT *>((yy & 1) ? l0.cost[0] : l0.cost[1]) + row_slot * Dp +
                                    label_pos<CostT>(dl);
            unsigned near_mask = 0u;  // outputs whose level the FP64 sequence must decide
            int S = 0;
#pragma unroll
            for (int i = 0; i < WIN; ++i) S += V[i];
#pragma unroll
            for (int j = 0; j < NR_TX; ++j) {
                if (j) {  // column j + 2R enters, column j - 1 leaves (its slot in the ring)
                    const int vn = dot(j + 2 * R);
                    S += vn - V[(j - 1) % WIN];
                    V[(j - 1) % WIN] = vn;
                }
                const int2 pa = pa_row[j];
                const int2 pb = pb_row[j];
                const Num num = (Num)N * (Num)S - (Num)pa.x * (Num)pb.x;
                bool near;
                const int c = quantise_fp32((float)num, __int_as_float(pa.y), __int_as_float(pb.y), T_half, half_m, T,
                                            &near);
                float nccf = 0.f;
                if constexpr (NCC_OUT || FLOAT_COST)
                    nccf = __fmul_rn(__fmul_rn((float)num, __int_as_float(QA[h * CW + lbase + j].y)),
                                     __int_as_float(pb.y));
                const bool inside = j < nvalid;
                CostT *dst = ((j & 1) ? base_odd : base_even) + (int64_t)(j >> 1) * Dp;
                if constexpr (FLOAT_COST) {
                    const float cf = fminf(fmaxf((float)T * (1.f - nccf), 0.f), (float)T);
                    if (inside) *dst = lab ? cf : 0.f;
                } else {
                    const int cs = lab ? c : 0;
                    store_if(dst, (CostT)cs,
                             inside && BPS_CHECK(row_slot + (j >> 1) < (int64_t)l0.H * l0.Wh, l0.err, 4u));
                    acc[j >> 1] += inside ? cs : 0;
                    near_mask |= (near ? 1u : 0u) << j;
                }
                if constexpr (NCC_OUT) {
                    if (inside && lab) ncc_out[((size_t)yy * W + xb + j) * D + dl] = nccf;
                }
            }
            if constexpr (!FLOAT_COST) {
                // rare: outputs whose fp32 value lies too near a level boundary are decided again
                // in FP64, and their stores and scale-1 sums corrected
                while (near_mask) {
                    const int j = __ffs(near_mask) - 1;
                    near_mask &= near_mask - 1;
                    int Sj = 0;
                    for (int i = j; i < j + WIN; ++i) {
                        const WinT a = Lrow[i], b = Rrow[i];
                        unsigned v = 0u;
#pragma unroll
                        for (int w = 0; w < NW; ++w) v = __dp4a(a.w[w], b.w[w], v);
                        Sj += (int)v;
                    }
                    const int2 pa = pa_row[j];
                    const int2 pb = pb_row[j];
                    const Num num = (Num)N * (Num)Sj - (Num)pa.x * (Num)pb.x;
                    bool near;
                    const int c32 = quantise_fp32((float)num, __int_as_float(pa.y), __int_as_float(pb.y), T_half,
                                                  half_m, T, &near);
                    const unsigned va = (unsigned)QA[h * CW + lbase + j].x;
                    const unsigned vb = (unsigned)QB[h * UW + lbase + j + D - 1 - d].x;
                    int c = quantise_fp64<Num>(num, va, vb, T);
                    c = c < 0 ? 0 : (c > T ? T : c);
                    if (j < nvalid && lab && c != c32) {
                        (((j & 1) ? base_odd : base_even) + (int64_t)(j >> 1) * Dp)[0] = (CostT)c;
#pragma unroll
                        for (int i = 0; i < NR_TX / 2; ++i)
                            if (i == (j >> 1)) acc[i] += c - c32;
                    }
                }
            }
        }
        if constexpr (!FLOAT_COST) {
            if (write_l1) {  // the coarse pixels of this row pair are complete
                const int cy = y >> 1;
#pragma unroll
                for (int jj = 0; jj < NR_TX / 2; ++jj) {
                    const int cx = (x0 + lbase) / 2 + jj;
                    if (cx < l1.W) {
                        CostT *dst = reinterpret_cast<CostT *>(colour_of(cx, cy) ? l1.cost[1] : l1.cost[0]) +
                                     slot_of(cx, cy, l1.Wh) * Dp + label_pos<CostT>(dl);
                        *dst = (CostT)acc[jj];
                    }
                }
            }
        }
    }
}

static int win_bytes(int window) {
    const int nw = (window + 3) / 4;
    return 4 * (nw <= 1 ? 1 : (nw <= 2 ? 2 : 4));
}

size_t ncc_rows_smem_bytes(int D, int XS, int window) {
    const int R = window / 2;
    const int CW = XS * NR_TX, LW = CW + 2 * R, RW = CW + 2 * R + D - 1, UW = CW + D - 1;
    // records [2 rows][hot, cold] 8 bytes each, windows [4 row buffers], column sums [2 rows][2]
    return (size_t)32 * (CW + UW) + (size_t)4 * win_bytes(window) * (LW + RW) + (size_t)16 * (LW + RW);
}

// Staged columns a thread owns at most for this shape (2 or 4: the kernel keeps that many
// windows in registers), or 0 when the shape needs more.
static int ncc_rows_items(int D, int Dp, int XS, int window) {
    const int R = window / 2, CW = XS * NR_TX;
    const int items = (CW + 2 * R) + (CW + 2 * R + D - 1);
    return items <= 2 * XS * Dp ? 2 : (items <= NR_ITEMS_MAX * XS * Dp ? NR_ITEMS_MAX : 0);
}

// Default CTA shape: every label of 256 / Dp column groups (256 threads), strips short
// enough that the grid covers the GPU (each strip re-reads 2R + 1 rows to fill its window),
// even for the 2x2 sums of scale 1.  bps_set_ncc_shape / the autotuner can replace it.
static void ncc_rows_default_shape(int W, int H, int Dp, int *XS, int *tys) {
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int xs = Dp >= 256 ? 1 : 256 / Dp;
    const int nx = (W + xs * NR_TX - 1) / (xs * NR_TX);
    int rows = (int)(((int64_t)H * nx + sms - 1) / sms);
    *XS = xs;
    *tys = std::max(8, std::min(64, (rows + 1) & ~1));
}

template <typename CostT, int R>
static cudaError_t launch_rows_t(const uint8_t *L, const uint8_t *Rim, int pitch, int W, int H, int D, int Dp, int T,
                                 const LevelView &l0, const LevelView *l1, float *ncc_out, cudaStream_t st, bool prep,
                                 int xs_req = 0, int tys_req = 0) {
    if (prep) {
        const int XSmax = std::max(1, 512 / Dp);
        if ((int)ncc_rows_smem_bytes(D, XSmax, 2 * R + 1) > smem_optin()) return cudaErrorInvalidValue;
        cudaError_t e = cudaFuncSetAttribute(ncc_rows_kernel<CostT, R, false, 2>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ncc_rows_kernel<CostT, R, true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     smem_optin());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ncc_rows_kernel<CostT, R, false, NR_ITEMS_MAX>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(ncc_rows_kernel<CostT, R, true, NR_ITEMS_MAX>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin());
        return e;
    }
    int XS = 1, tys = 16;
    ncc_rows_default_shape(W, H, Dp, &XS, &tys);
    if (xs_req > 0) XS = xs_req;
    if (tys_req > 0) tys = tys_req;
    const int items = ncc_rows_items(D, Dp, XS, 2 * R + 1);
    if (!items) return cudaErrorInvalidConfiguration;
    const size_t smem = ncc_rows_smem_bytes(D, XS, 2 * R + 1);
    const int threads = XS * Dp;
    const int CW = XS * NR_TX;
    const int nx = (W + CW - 1) / CW;
    const int ny = (H + tys - 1) / tys;
    LevelView none = l0;
    const dim3 grid(nx, ny);
    const LevelView l1v = l1 ? *l1 : none;
    const int w1 = l1 ? 1 : 0;
    if (items == 2) {
        if (ncc_out)
            return launch_k(ncc_rows_kernel<CostT, R, true, 2>, grid, dim3(threads), smem, st, L, Rim, pitch, W, H, D,
                            Dp, T, tys, l0, l1v, w1, ncc_out);
        return launch_k(ncc_rows_kernel<CostT, R, false, 2>, grid, dim3(threads), smem, st, L, Rim, pitch, W, H, D, Dp,
                        T, tys, l0, l1v, w1, ncc_out);
    }
    if (ncc_out)
        return launch_k(ncc_rows_kernel<CostT, R, true, NR_ITEMS_MAX>, grid, dim3(threads), smem, st, L, Rim, pitch, W,
                        H, D, Dp, T, tys, l0, l1v, w1, ncc_out);
    return launch_k(ncc_rows_kernel<CostT, R, false, NR_ITEMS_MAX>, grid, dim3(threads), smem, st, L, Rim, pitch, W, H,
                    D, Dp, T, tys, l0, l1v, w1, ncc_out);
}

template <typename CostT>
static cudaError_t launch_rows(int R, const uint8_t *L, const uint8_t *Rim, int pitch, int W, int H, int D, int Dp,
                               int T, const LevelView &l0, const LevelView *l1, float *ncc_out, cudaStream_t st,
                               bool prep, int xs = 0, int tys = 0) {
    switch (R) {
    case 0: return launch_rows_t<CostT, 0>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    case 1: return launch_rows_t<CostT, 1>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    case 2: return launch_rows_t<CostT, 2>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    case 3: return launch_rows_t<CostT, 3>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    case 4: return launch_rows_t<CostT, 4>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    case 5: return launch_rows_t<CostT, 5>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    case 6: return launch_rows_t<CostT, 6>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    default: return launch_rows_t<CostT, 7>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, prep, xs, tys);
    }
}

cudaError_t launch_ncc_rows(int cost_kind, const uint8_t *L, const uint8_t *Rim, int pitch, int W, int H, int D, int Dp,
                            int window, int T, const LevelView &l0, const LevelView *l1, float *ncc_out,
                            cudaStream_t st, int xs, int tys) {
    const int R = window / 2;
    switch (cost_kind) {
    case COST_I32: return launch_rows<int32_t>(R, L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, false, xs, tys);
    case COST_I16: return launch_rows<int16_t>(R, L, Rim, pitch, W, H, D, Dp, T, l0, l1, ncc_out, st, false, xs, tys);
    default: return launch_rows<float>(R, L, Rim, pitch, W, H, D, Dp, T, l0, nullptr, ncc_out, st, false, xs, tys);
    }
}

cudaError_t ncc_rows_prepare(int cost_kind, int D, int Dp) {
    for (int R = 0; R <= NCC_ROWS_MAX_WINDOW / 2; ++R) {
        const LevelView none{};
        cudaError_t e;
        switch (cost_kind) {
        case COST_I32: e = launch_rows<int32_t>(R, nullptr, nullptr, 0, 1, 1, D, Dp, 0, none, nullptr, nullptr, 0, true); break;
        case COST_I16: e = launch_rows<int16_t>(R, nullptr, nullptr, 0, 1, 1, D, Dp, 0, none, nullptr, nullptr, 0, true); break;
        default: e = launch_rows<float>(R, nullptr, nullptr, 0, 1, 1, D, Dp, 0, none, nullptr, nullptr, 0, true); break;
        }
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

size_t ncc_smem_bytes(int D, int window) {
    const int r = window / 2;
    const int TW = NCC_TX + 2 * r, RW = TW + D - 1, SH = NCC_TY + 2 * r, UW = NCC_TX + D - 1;
    const int CS = NCC_TY * TW + 1;
    size_t ints = 2 * NCC_TY * NCC_TX + 2 * NCC_TY * UW + NCC_DC * CS;
    return ints * 4 + (size_t)SH * TW + (size_t)SH * RW;
}

template <typename CostT>
static cudaError_t launch_ncc_t(const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int D, int Dp,
                                int window, int T, int Wh, void *c0, void *c1, float *ncc_out, cudaStream_t st) {
    const size_t smem = ncc_smem_bytes(D, window);
    dim3 grid((W + NCC_TX - 1) / NCC_TX, (H + NCC_TY - 1) / NCC_TY);
    return launch_k(ncc_cost_kernel<CostT>, grid, dim3(NCC_THREADS), smem, st, L, R, pitch, W, H, D, Dp, window, T,
                    Wh, (CostT *)c0, (CostT *)c1, ncc_out);
}

cudaError_t ncc_prepare(int cost_kind, int D, int max_window) {
    if ((int)ncc_smem_bytes(D, max_window) > smem_optin()) return cudaErrorInvalidValue;
    const int smem = smem_optin();
    switch (cost_kind) {
    case COST_I32: return cudaFuncSetAttribute(ncc_cost_kernel<int32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    case COST_I16: return cudaFuncSetAttribute(ncc_cost_kernel<int16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    default: return cudaFuncSetAttribute(ncc_cost_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    }
}

cudaError_t launch_ncc(int cost_kind, const uint8_t *L, const uint8_t *R, int pitch, int W, int H, int D, int Dp,
                       int window, int T, int Wh, void *c0, void *c1, float *ncc_out, cudaStream_t st) {
    switch (cost_kind) {
    case COST_I32: return launch_ncc_t<int32_t>(L, R, pitch, W, H, D, Dp, window, T, Wh, c0, c1, ncc_out, st);
    case COST_I16: return launch_ncc_t<int16_t>(L, R, pitch, W, H, D, Dp, window, T, Wh, c0, c1, ncc_out, st);
    default: return launch_ncc_t<float>(L, R, pitch, W, H, D, Dp, window, T, Wh, c0, c1, ncc_out, st);
    }
}

// ------------------------------------------------------------------ cost pyramid
// C_{l+1}(x, y, d) = sum of C_l over the existing children (2x + a, 2y + b), a, b in {0, 1}.
// Children (2x, 2y) and (2x+1, 2y+1) are even-coloured, the other two odd; child (2x + a,
// 2y + b) sits at fine slot (2y + b) * Wh_f + x.
template <typename CostT>
__global__ void pyramid_kernel(LevelView fine, LevelView coarse, int Dp) {
    pdl_enter();
    using Acc = typename std::conditional<CostOut<CostT>::is_float, float, int>::type;
    const int64_t n = (int64_t)coarse.H * coarse.W * Dp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(k % Dp);
        const int64_t p = k / Dp;
        const int x = (int)(p % coarse.W), y = (int)(p / coarse.W);
        Acc s = Acc(0);
        for (int b = 0; b < 2; ++b)
            for (int a = 0; a < 2; ++a) {
                const int fx = 2 * x + a, fy = 2 * y + b;
                if (fx < fine.W && fy < fine.H) {
                    const CostT *src = (const CostT *)fine.cost[(a + b) & 1];
                    s += (Acc)src[((int64_t)fy * fine.Wh + x) * Dp + d];
                }
            }
        CostT *dst = (CostT *)coarse.cost[colour_of(x, y)];
        dst[slot_of(x, y, coarse.Wh) * Dp + d] = (CostT)s;
    }
}

// Two scales in one launch: a thread per (pixel of scale l+1, label) forms its four children
// at scale l from their 2x2 blocks at scale l-1, writes them, and writes their sum.  Every
// pixel of scale l has its parent at scale l+1 (ceil halving), so each is written once.
template <typename CostT>
__global__ void pyramid2_kernel(LevelView fine, LevelView mid, LevelView coarse, int Dp) {
    pdl_enter();
    using Acc = typename std::conditional<CostOut<CostT>::is_float, float, int>::type;
    const int64_t n = (int64_t)coarse.H * coarse.W * Dp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(k % Dp);
        const int64_t p = k / Dp;
        const int X = (int)(p % coarse.W), Y = (int)(p / coarse.W);
        Acc S = Acc(0);
        for (int bb = 0; bb < 2; ++bb)
            for (int aa = 0; aa < 2; ++aa) {
                const int mx = 2 * X + aa, my = 2 * Y + bb;
                if (mx >= mid.W || my >= mid.H) continue;
                Acc s = Acc(0);
                for (int b = 0; b < 2; ++b)
                    for (int a = 0; a < 2; ++a) {
                        const int fx = 2 * mx + a, fy = 2 * my + b;
                        if (fx < fine.W && fy < fine.H) {
                            const CostT *src = (const CostT *)fine.cost[(a + b) & 1];
                            s += (Acc)src[((int64_t)fy * fine.Wh + mx) * Dp + d];
                        }
                    }
                ((CostT *)mid.cost[colour_of(mx, my)])[slot_of(mx, my, mid.Wh) * Dp + d] = (CostT)s;
                S += s;
            }
        ((CostT *)coarse.cost[colour_of(X, Y)])[slot_of(X, Y, coarse.Wh) * Dp + d] = (CostT)S;
    }
}

cudaError_t preload_cost_kernels(int cost_kind) {
    cudaFuncAttributes a;
    switch (cost_kind) {
    case COST_I32:
        return cudaFuncGetAttributes(&a, pyramid_kernel<int32_t>) == cudaSuccess
                   ? cudaFuncGetAttributes(&a, pyramid2_kernel<int32_t>)
                   : cudaErrorUnknown;
    case COST_I16:
        return cudaFuncGetAttributes(&a, pyramid_kernel<int16_t>) == cudaSuccess
                   ? cudaFuncGetAttributes(&a, pyramid2_kernel<int16_t>)
                   : cudaErrorUnknown;
    default:
        return cudaFuncGetAttributes(&a, pyramid_kernel<float>) == cudaSuccess
                   ? cudaFuncGetAttributes(&a, pyramid2_kernel<float>)
                   : cudaErrorUnknown;
    }
}

cudaError_t launch_pyramid2(int cost_kind, const LevelView &fine, const LevelView &mid, const LevelView &coarse, int Dp,
                            cudaStream_t st) {
    const int64_t n = (int64_t)coarse.H * coarse.W * Dp;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    switch (cost_kind) {
    case COST_I32: return launch_k(pyramid2_kernel<int32_t>, dim3(blocks), dim3(256), 0, st, fine, mid, coarse, Dp);
    case COST_I16: return launch_k(pyramid2_kernel<int16_t>, dim3(blocks), dim3(256), 0, st, fine, mid, coarse, Dp);
    default: return launch_k(pyramid2_kernel<float>, dim3(blocks), dim3(256), 0, st, fine, mid, coarse, Dp);
    }
}

cudaError_t launch_pyramid(int cost_kind, const LevelView &fine, const LevelView &coarse, int Dp, cudaStream_t st) {
    const int64_t n = (int64_t)coarse.H * coarse.W * Dp;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    switch (cost_kind) {
    case COST_I32: return launch_k(pyramid_kernel<int32_t>, dim3(blocks), dim3(256), 0, st, fine, coarse, Dp);
    case COST_I16: return launch_k(pyramid_kernel<int16_t>, dim3(blocks), dim3(256), 0, st, fine, coarse, Dp);
    default: return launch_k(pyramid_kernel<float>, dim3(blocks), dim3(256), 0, st, fine, coarse, Dp);
    }
}

}  // namespace bps
