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
    ncc_cost_kernel<CostT><<<grid, NCC_THREADS, smem, st>>>(L, R, pitch, W, H, D, Dp, window, T, Wh,
                                                            (CostT *)c0, (CostT *)c1, ncc_out);
    return cudaGetLastError();
}

cudaError_t ncc_prepare(int cost_kind, int D, int max_window) {
    const int smem = (int)ncc_smem_bytes(D, max_window);
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

cudaError_t launch_pyramid(int cost_kind, const LevelView &fine, const LevelView &coarse, int Dp, cudaStream_t st) {
    const int64_t n = (int64_t)coarse.H * coarse.W * Dp;
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
    switch (cost_kind) {
    case COST_I32: pyramid_kernel<int32_t><<<blocks, 256, 0, st>>>(fine, coarse, Dp); break;
    case COST_I16: pyramid_kernel<int16_t><<<blocks, 256, 0, st>>>(fine, coarse, Dp); break;
    default: pyramid_kernel<float><<<blocks, 256, 0, st>>>(fine, coarse, Dp); break;
    }
    return cudaGetLastError();
}

}  // namespace bps
