// persist.cu -- the whole hierarchical BP solve (sections "Fast Converging BP" and "GPU
// Implementation") for a batch of stereo pairs in ONE cooperative launch, followed by the
// winner-take-all read-out.
//
// All pairs advance in lockstep through the same phase sequence (every pair of a batch
// has the same number of scales and iterations):
//   for scale l = coarsest .. 0:
//       prep:   coarse-to-fine copy of the parents' messages (l < coarsest) and the skip
//               flags set to "dirty" (fast-converging skip on)            -> grid barrier
//       for it < iters, colour 0 then 1:
//               red-black half-sweep of every pair                        -> grid barrier
//   winner-take-all of every pair.
// Inside a half-sweep the work of all pairs is one list of 256-thread blocks (a prefix
// sum per scale maps a block index to its pair); each CTA takes blocks grid-stride.  One
// launch replaces the 2 * iters * levels dependent launches of the per-sweep path, and a
// batch shares each barrier.
//
// Grid barrier: a monotonically increasing arrival counter (barrier k completes when it
// reaches (k + 1) * gridDim.x), so it never needs a reset.  The wait is bounded by a
// deadline on %globaltimer: a block that waits past it sets the error word and the whole
// grid returns; the host reports BPS_ERR_TIMEOUT.  Co-residency of all CTAs comes from the
// cooperative launch.
#include <algorithm>

#include "bps_launch.h"
#include "sweep_body.cuh"

namespace bps {

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Returns false (in every thread of the block) once any block has given up.
__device__ __forceinline__ bool grid_barrier(unsigned *state, unsigned target, unsigned long long timeout_ns) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        volatile unsigned *count = state;
        volatile unsigned *error = state + 1;
        __threadfence();
        atomicAdd(state, 1u);
        const unsigned long long t0 = global_ns();
        while (*count < target) {
            if (*error) {
                ok = 0;
                break;
            }
            if (global_ns() - t0 > timeout_ns) {
                atomicExch(state + 1, 1u);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

__device__ __forceinline__ int find_pair(const int *prefix, int npairs, int v) {
    int lo = 0, hi = npairs - 1;  // last p with prefix[p] <= v
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= v) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int FORM>
__global__ void __launch_bounds__(256, FORM == MSG_U8 ? 3 : 1) bp_persistent_kernel(PersistParams P) {
    const int top = P.levels - 1;
    unsigned target = 0;
    auto sync = [&]() {
        target += gridDim.x;
        return grid_barrier(P.barrier, target + P.extra_arrivals, P.timeout_ns);
    };
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    for (int l = top; l >= 0; --l) {
        for (int p = 0; p < P.npairs; ++p) {
            const PairDesc &pd = P.pairs[p];
            const LevelView &v = pd.lv[l];
            if (l < top) {
                const int rec_chunks = 4 * pd.Dp * (FORM == MSG_I32 ? 4 : FORM == MSG_U8 ? 1 : 2) / 16;
                const int64_t n = (int64_t)v.H * v.Wh * rec_chunks;
                // the odd pixels' start messages matter only without sweeps, or under the freeze
                // rule, whose first half-sweep compares the even pixels' messages with them
                for (int colour = 0; colour < ((P.iters == 0 || v.freeze) ? 2 : 1); ++colour)
                    for (int64_t k = tid; k < n; k += nthreads) upsample_chunk(pd.lv[l + 1], v, colour, rec_chunks, k);
            }
            if (P.skip) {
                const int64_t n = (int64_t)v.H * v.Wh;
                for (int64_t k = tid; k < n; k += nthreads) v.dirty[0][k] = v.dirty[1][k] = 1;
            }
        }
        if (!sync()) return;
        const int *prefix = P.sweep_prefix + l * (P.npairs + 1);
        const int nblocks = prefix[P.npairs];
        for (int it = 0; it < P.iters; ++it)
            for (int colour = 0; colour < 2; ++colour) {
                const int t = (top - l) * P.iters * 2 + it * 2 + colour;
                for (int vb = blockIdx.x; vb < nblocks; vb += gridDim.x) {
                    const int p = find_pair(prefix, P.npairs, vb);
                    const PairDesc &pd = P.pairs[p];
                    const int64_t b = vb - prefix[p];
                    unsigned long long *trace = pd.trace ? pd.trace + t : nullptr;
                    if constexpr (FORM == MSG_U8) {
                        if (pd.D & 15)
                            sweep_group_u8<true, false, 0, true>(pd.lv[l], colour, pd.D, pd.Dp, pd.Gp, P.lam_u8, P.lam_u8 * P.trunc,
                                                 P.skip, trace, b);
                        else
                            sweep_group_u8<false, false, 0, true>(pd.lv[l], colour, pd.D, pd.Dp, pd.Gp, P.lam_u8, P.lam_u8 * P.trunc,
                                                  P.skip, trace, b);
                    } else if constexpr (FORM == MSG_I32) {
                        sweep_group<int32_t, int32_t, true>(pd.lv[l], colour, pd.D, pd.Dp, pd.Gp, P.lam, P.lam * P.trunc,
                                                      P.skip, trace, b);
                    } else {
                        sweep_group<float, __half, true>(pd.lv[l], colour, pd.D, pd.Dp, pd.Gp, (float)P.lam,
                                                   (float)P.lam * (float)P.trunc, P.skip, trace, b);
                    }
                }
                if (!sync()) return;
            }
    }
    const int *wp = P.wta_prefix;
    for (int vb = blockIdx.x; vb < wp[P.npairs]; vb += gridDim.x) {
        const int p = find_pair(wp, P.npairs, vb);
        const PairDesc &pd = P.pairs[p];
        int32_t *disp = (p == 0 && P.disp_override) ? P.disp_override : pd.disp;
        if (!disp) continue;
        if constexpr (FORM == MSG_U8) wta_group<int16_t, uint8_t, true>(pd.lv[0], pd.D, pd.Dp, pd.Gp, disp, vb - wp[p]);
        else if constexpr (FORM == MSG_I32) wta_group<int32_t, int32_t, true>(pd.lv[0], pd.D, pd.Dp, pd.Gp, disp, vb - wp[p]);
        else wta_group<float, __half, true>(pd.lv[0], pd.D, pd.Dp, pd.Gp, disp, vb - wp[p]);
    }
}

static const void *persistent_fn(int form) {
    switch (form) {
    case MSG_I32: return (const void *)bp_persistent_kernel<MSG_I32>;
    case MSG_U8: return (const void *)bp_persistent_kernel<MSG_U8>;
    default: return (const void *)bp_persistent_kernel<MSG_F16>;
    }
}

cudaError_t persistent_grid(int form, int *grid) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_fn(form), 256, 0);
    if (e != cudaSuccess) return e;
    *grid = std::max(1, sms * per_sm);
    return cudaSuccess;
}

cudaError_t launch_persistent(int form, const PersistParams &P, int grid, cudaStream_t st) {
    PersistParams copy = P;
    void *args[] = {&copy};
    return cudaLaunchCooperativeKernel(persistent_fn(form), dim3(grid), dim3(256), args, 0, st);
}

}  // namespace bps
