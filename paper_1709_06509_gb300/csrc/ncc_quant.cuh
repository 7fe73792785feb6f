// ncc_quant.cuh -- the data-cost quantiser shared by the NCC kernels (section "Correlation
// volume computation"; the data cost c = clamp(floor(T (1 - ncc) + 1/2), 0, T)): a fast fp32
// step that is exact away from the level boundaries, and the FP64 sequence that decides near them.
#pragma once

#include <stdint.h>

namespace bps {

template <int R> struct NccInt { using type = int; };
template <> struct NccInt<7> { using type = long long; };  // 15x15: N S_ab - S_a S_b needs 33 bits


// The rare exact decision of the quantiser, out of line: the fp32 path is the hot one.
template <typename Num>
__device__ __noinline__ int quantise_fp64(Num num, unsigned va, unsigned vb, int T) {
    const double den = __dmul_rn((double)va, (double)vb);
    const double n64 = __ddiv_rn((double)num, __dsqrt_rn(den));
    return (int)floor(__dadd_rn(__dmul_rn((double)T, __dadd_rn(1.0, -n64)), 0.5));
}

// The fp32 quantiser step of one (pixel, label): the level c = min(floor(v), T) of
// v = (T + 1/2) - (T ra) rb num, one fused multiply-add, and whether v lies within the margin
// m = (T + 1) 2^-17 of an integer (then only the FP64 sequence may decide).  ra, rb are the
// reciprocal square roots of the two variance terms (rsqrtf, at most 2 ulp = 4 2^-24 relative
// error, plus half the conversion's 2^-24), T ra is rounded once more, the product once more
// and the numerator's conversion once: at most 12 2^-24 relative error in the product, and with
// the fused multiply-add's rounding v is within (T + 1) 14 2^-24 < (T + 1) 2^-20 of its exact
// value: outside the margin (8 times wider) the fp32 and the exact decision agree.
// v >= 1/2 - (T + 1) 2^-20 > 0, so the lower clamp at 0 is never needed.  A zero variance has a zero reciprocal
// square root, so v = T + 1/2 and c = T, the value the definition gives for ncc = 0.
__device__ __forceinline__ int quantise_fp32(float numf, float tra, float rb, float T_half, float half_m, int T,
                                             bool *near) {
    const float v = __fmaf_rn(-__fmul_rn(tra, rb), numf, T_half);
    const float fl = floorf(v);
    *near = !(fabsf((v - fl) - 0.5f) < half_m);  // v - fl is exact
    return min((int)fl, T);
}

}  // namespace bps
