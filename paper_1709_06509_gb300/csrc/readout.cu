// readout.cu -- winner-take-all disparity and the energy E(d) = E_D(d) + E_S(d)
// (section "Approach Description").
//
// wta_kernel: a group of Gp lanes per pixel (natural raster order) forms the belief
// cost + sum of the existing incoming messages and takes the argmin, the lowest label on
// ties (per-lane scan, then a butterfly that prefers the smaller label on equal values).
//
// energy: each thread walks pixels with a grid stride and adds the data cost of its label
// and lambda * min(|d_p - d_q|, trunc) for the right and lower neighbours (each grid edge
// once).  Integer forms sum in int64 (exact); the float form sums in FP64.  Per-block
// partials go to scratch, then one block adds them in a fixed order, so the FP64 result
// is reproducible run to run.
#include <algorithm>
#include <type_traits>

#include "bps_launch.h"
#include "sweep_body.cuh"

namespace bps {

template <typename CostT, typename MsgT>
__global__ void __launch_bounds__(256) wta_kernel(LevelView lv, int D, int Dp, int Gp, int32_t *disp) {
    pdl_enter();
    wta_group<CostT, MsgT>(lv, D, Dp, Gp, disp, blockIdx.x);
}

// The rest of a read-out that the finest scale's half-sweeps started (u8 form, or the fp16 form's
// packed sweep; exact skip rule):
// every recomputed pixel already wrote the label of the belief it formed, and a pixel's belief
// changes only when an incoming message does.  After the last half-sweep (the odd pixels) the
// odd pixels' labels are final, and so are the even pixels' whose incoming messages did not
// change since their own last update; the even pixels that the last half-sweep marked dirty
// (with the skip off: every even pixel) are read out here, from the listed entries (`list`
// non-null, `n_list` entries) or by their skip flags.  Grid-stride over the even pixels.
template <typename CostT, typename MsgT>
__global__ void __launch_bounds__(256)
wta_rest_kernel(LevelView lv, int D, int Dp, int Gp, int skip, const unsigned *list, const unsigned *n_list,
                int32_t *disp) {
    pdl_enter();
    const int groups = blockDim.x / Gp;
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    const int64_t n = list ? (int64_t)*n_list : nslot;
    for (int64_t b = blockIdx.x; b * groups < n; b += gridDim.x) {
        const int64_t i = b * groups + threadIdx.x / Gp;
        int64_t s = i < n ? (list ? (int64_t)list[i] : i) : nslot;
        int x = 0, y = 0;
        bool need = false;
        if (s < nslot) {
            y = (int)(s / lv.Wh);
            x = 2 * (int)(s - (int64_t)y * lv.Wh) + (y & 1);  // even pixels: (x + y) & 1 == 0
            need = x < lv.W && (list || !skip || lv.dirty[0][s] == 1u);
        }
        if (__ballot_sync(FULL, need) == 0u) continue;
        wta_pixel<CostT, MsgT>(lv, D, Dp, Gp, disp, need ? x : 0, need ? y : 0, need);
    }
}

cudaError_t preload_readout_kernels(int msg_kind) {
    cudaFuncAttributes a;
    switch (msg_kind) {
    case MSG_I32: return cudaFuncGetAttributes(&a, wta_kernel<int32_t, int32_t>);
    case MSG_U8: {
        const cudaError_t e = cudaFuncGetAttributes(&a, wta_kernel<int16_t, uint8_t>);
        return e == cudaSuccess ? cudaFuncGetAttributes(&a, wta_rest_kernel<int16_t, uint8_t>) : e;
    }
    default: {
        const cudaError_t e = cudaFuncGetAttributes(&a, wta_kernel<float, __half>);
        return e == cudaSuccess ? cudaFuncGetAttributes(&a, wta_rest_kernel<float, __half>) : e;
    }
    }
}

cudaError_t launch_wta_rest(int msg_kind, const LevelView &lv, int D, int Dp, int Gp, int skip, const unsigned *list,
                            const unsigned *n_list, int32_t *disp, cudaStream_t st) {
    const int groups = 256 / Gp;
    const int64_t blocks = ((int64_t)lv.H * lv.Wh + groups - 1) / groups;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)sms * 8));
    if (msg_kind == MSG_F16)
        return launch_k(wta_rest_kernel<float, __half>, dim3(grid), dim3(256), 0, st, lv, D, Dp, Gp, skip, list, n_list,
                        disp);
    return launch_k(wta_rest_kernel<int16_t, uint8_t>, dim3(grid), dim3(256), 0, st, lv, D, Dp, Gp, skip, list, n_list,
                    disp);
}

cudaError_t launch_wta(int msg_kind, const LevelView &lv, int D, int Dp, int Gp, int32_t *disp, cudaStream_t st) {
    const int groups = 256 / Gp;
    const int64_t blocks = ((int64_t)lv.W * lv.H + groups - 1) / groups;
    switch (msg_kind) {
    case MSG_I32: return launch_k(wta_kernel<int32_t, int32_t>, dim3((unsigned)blocks), dim3(256), 0, st, lv, D, Dp, Gp, disp);
    case MSG_U8: return launch_k(wta_kernel<int16_t, uint8_t>, dim3((unsigned)blocks), dim3(256), 0, st, lv, D, Dp, Gp, disp);
    default: return launch_k(wta_kernel<float, __half>, dim3((unsigned)blocks), dim3(256), 0, st, lv, D, Dp, Gp, disp);
    }
}

// ------------------------------------------------------------------ energy
constexpr int E_THREADS = 256, E_MAX_BLOCKS = 1024;

int energy_blocks(int W, int H) {
    const int64_t n = (int64_t)W * H;
    return (int)std::max<int64_t>(1, std::min<int64_t>((n + E_THREADS - 1) / E_THREADS, E_MAX_BLOCKS));
}

template <typename Sum>
__device__ inline Sum block_sum(Sum v, Sum *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    Sum t = Sum(0);
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : Sum(0);
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(FULL, t, o);
    }
    return t;  // valid in thread 0
}

template <typename CostT>
__global__ void __launch_bounds__(E_THREADS)
energy_partial_kernel(LevelView lv, int D, int Dp, const int32_t *disp, int lambda, int trunc, void *partials) {
    pdl_enter();
    using Sum = typename std::conditional<std::is_same<CostT, float>::value, double, long long>::type;
    __shared__ Sum sh[E_THREADS / 32];
    Sum acc = Sum(0);
    const int64_t n = (int64_t)lv.W * lv.H;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(p % lv.W), y = (int)(p / lv.W);
        const int d = min(max(disp[p], 0), D - 1);
        acc += (Sum) reinterpret_cast<const CostT *>(lv.cost[colour_of(x, y)])[slot_of(x, y, lv.Wh) * Dp +
                                                                               label_pos<CostT>(d)];
        if (x + 1 < lv.W) {
            const int e = min(max(disp[p + 1], 0), D - 1);
            acc += (Sum)((long long)lambda * min(abs(d - e), trunc));
        }
        if (y + 1 < lv.H) {
            const int e = min(max(disp[p + lv.W], 0), D - 1);
            acc += (Sum)((long long)lambda * min(abs(d - e), trunc));
        }
    }
    const Sum t = block_sum(acc, sh);
    if (threadIdx.x == 0) reinterpret_cast<Sum *>(partials)[blockIdx.x] = t;
}

template <typename Sum>
__global__ void __launch_bounds__(E_THREADS)
energy_final_kernel(const void *partials, int nblocks, int64_t *out_i64, double *out_f64) {
    pdl_enter();
    __shared__ Sum sh[E_THREADS / 32];
    Sum acc = Sum(0);
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) acc += reinterpret_cast<const Sum *>(partials)[k];
    const Sum t = block_sum(acc, sh);
    if (threadIdx.x == 0) {
        if (out_i64) *out_i64 = (int64_t)t;
        if (out_f64) *out_f64 = (double)t;
    }
}

cudaError_t launch_energy(int cost_kind, const LevelView &lv, int D, int Dp, const int32_t *disp, int lambda,
                          int trunc, void *partials, int64_t *out_i64, double *out_f64, cudaStream_t st) {
    const int nb = energy_blocks(lv.W, lv.H);
    cudaError_t e = cudaSuccess;
    switch (cost_kind) {
    case COST_I32:
        e = launch_k(energy_partial_kernel<int32_t>, dim3(nb), dim3(E_THREADS), 0, st, lv, D, Dp, disp, lambda, trunc,
                     partials);
        if (e == cudaSuccess)
            e = launch_k(energy_final_kernel<long long>, dim3(1), dim3(E_THREADS), 0, st, (const void *)partials, nb,
                         out_i64, out_f64);
        break;
    case COST_I16:
        e = launch_k(energy_partial_kernel<int16_t>, dim3(nb), dim3(E_THREADS), 0, st, lv, D, Dp, disp, lambda, trunc,
                     partials);
        if (e == cudaSuccess)
            e = launch_k(energy_final_kernel<long long>, dim3(1), dim3(E_THREADS), 0, st, (const void *)partials, nb,
                         out_i64, out_f64);
        break;
    default:
        e = launch_k(energy_partial_kernel<float>, dim3(nb), dim3(E_THREADS), 0, st, lv, D, Dp, disp, lambda, trunc,
                     partials);
        if (e == cudaSuccess)
            e = launch_k(energy_final_kernel<double>, dim3(1), dim3(E_THREADS), 0, st, (const void *)partials, nb,
                         (int64_t *)nullptr, out_f64);
        break;
    }
    return e;
}

}  // namespace bps
