// sweep_f16.cu -- the red-black half-sweep of the fp16-message form in packed half2 arithmetic
// (truncation T <= 2; larger T keeps the generic kernel): one launch per half-sweep, the body in
// sweep_f16_body.cuh.  Skip and trace as in the other forms; the flag and every input may be
// loaded at once (EAGER); with the skip on, the active lists of the u8 form (a dense launch that
// appends, then launches over the lists).
#include <cuda_fp16.h>

#include <algorithm>

#include "bps_launch.h"
#include "sweep_f16_body.cuh"

namespace bps {

template <bool PADDED, int TS, bool EAGER, bool APPEND>
__global__ void __launch_bounds__(256, 2)
sweep_f16_kernel(LevelView lv, int colour, int D, int Dp, int Gp, float lam, float lamT, int skip,
                 unsigned long long *trace, int nblocks, ActiveList al) {
    unsigned *abuf = nullptr;
    if constexpr (APPEND) {
        BPS_LIST_BUFFER(list_buf);
        abuf = list_buf[threadIdx.x >> 5];
    }
    pdl_enter();
    Tally tally(trace, abuf);
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x)
        sweep_group_f16<PADDED, TS, EAGER, APPEND>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b, al);
    if constexpr (APPEND) tally.flush_appends(al.out, al.n_out, (unsigned)lv.H * (unsigned)lv.Wh, lv.err);
    tally.flush();
}

// Over the pixels of an active list (its length read on the device), like the u8 list sweep.
template <bool PADDED, int TS>
__global__ void __launch_bounds__(256, 2)
sweep_f16_list_kernel(LevelView lv, int colour, int D, int Dp, int Gp, float lam, float lamT,
                      unsigned long long *trace, ActiveList al) {
    pdl_enter();
    const int groups = blockDim.x / Gp;
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    const int64_t stride = (int64_t)gridDim.x * groups;
    int64_t idx = (int64_t)blockIdx.x * groups + threadIdx.x / Gp;
    unsigned e = idx < nslot ? al.in[idx] : 0u;
    const int64_t n = *al.n_in;
    BPS_LIST_BUFFER(list_buf);
    Tally tally(trace, list_buf[threadIdx.x >> 5]);
    for (int64_t b = blockIdx.x; b * groups < n; b += gridDim.x, idx += stride) {
        const int64_t s = idx < n ? (int64_t)e : nslot;
        if (idx + stride < n) e = al.in[idx + stride];
        sweep_group_f16<PADDED, TS, false, true, true>(lv, colour, D, Dp, Gp, lam, lamT, 1, tally, b, al, s);
    }
    tally.flush_appends(al.out, al.n_out, (unsigned)nslot, lv.err);
    tally.flush();
}

static int resident_f16() {  // CTAs of the fp16 sweep resident at once (looked up once per process)
    static int resident = 0;
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_f16_kernel<false, 2, false, false>, 256, 0);
        resident = std::max(1, sms * std::max(1, per_sm));
    }
    return resident;
}

template <bool PADDED, int TS>
static cudaError_t launch_f16_t(const LevelView &lv, int colour, int D, int Dp, int Gp, float lam, float lamT, int skip,
                                unsigned long long *trace, bool eager, const SweepLists &lists, cudaStream_t st) {
    const int groups = 256 / Gp;
    const int64_t blocks = ((int64_t)lv.H * lv.Wh + groups - 1) / groups;
    if (blocks == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>(blocks, resident_f16());
    const ActiveList al{lists.in, lists.n_in, skip ? lists.out : nullptr, lists.n_out};
    if (skip && al.in)
        return launch_k(sweep_f16_list_kernel<PADDED, TS>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp, lam,
                        lamT, trace, al);
    const ActiveList dense{nullptr, nullptr, al.out, al.n_out};
    if (al.out)
        return launch_k(sweep_f16_kernel<PADDED, TS, false, true>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp,
                        lam, lamT, skip, trace, (int)blocks, dense);
    if (eager)
        return launch_k(sweep_f16_kernel<PADDED, TS, true, false>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp,
                        lam, lamT, skip, trace, (int)blocks, dense);
    return launch_k(sweep_f16_kernel<PADDED, TS, false, false>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp,
                    lam, lamT, skip, trace, (int)blocks, dense);
}

bool sweep_f16_applies(int trunc) { return trunc <= 2; }

cudaError_t launch_sweep_f16(const LevelView &lv, int colour, int D, int Dp, int Gp, int lambda, int trunc, int skip,
                             unsigned long long *trace, bool eager, const SweepLists &lists, cudaStream_t st) {
    const float lam = trunc == 0 ? 0.f : (float)lambda, lamT = lam * (float)trunc;
    const bool padded = (D & 15) != 0;
    if (trunc <= 1) {
        if (padded) return launch_f16_t<true, 1>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, eager, lists, st);
        return launch_f16_t<false, 1>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, eager, lists, st);
    }
    if (padded) return launch_f16_t<true, 2>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, eager, lists, st);
    return launch_f16_t<false, 2>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, eager, lists, st);
}

template <bool PADDED, int TS> static cudaError_t preload_f16_t() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, sweep_f16_kernel<PADDED, TS, false, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sweep_f16_kernel<PADDED, TS, true, false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sweep_f16_kernel<PADDED, TS, false, true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sweep_f16_list_kernel<PADDED, TS>);
    return e;
}

cudaError_t preload_f16_kernels() {
    cudaError_t e = preload_f16_t<false, 1>();
    if (e == cudaSuccess) e = preload_f16_t<false, 2>();
    if (e == cudaSuccess) e = preload_f16_t<true, 1>();
    if (e == cudaSuccess) e = preload_f16_t<true, 2>();
    return e;
}

}  // namespace bps
