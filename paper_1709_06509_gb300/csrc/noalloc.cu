// noalloc.cu -- an energy entry point that allocates no memory at all.
//
// Some callers cannot allocate device memory when they need the energy of a labelling:
// real-time loops whose latency budget forbids an allocator (cudaMalloc and cudaFree may
// synchronise the whole device), programs that run this library inside a framework owning
// all device memory through an allocator the library cannot reach, and code running under a
// fixed memory budget where any new allocation may fail.  For them bps_energy_noalloc
// computes E(d) = E_D(d) + E_S(d) from a cost volume and a labelling the caller already
// holds, with its scratch (one partial sum per block) in a fixed array compiled into this
// library instead of a workspace or a cudaMalloc.
//
// The scratch array lives in device memory of every GPU that loads the library and stays
// there until the process exits.  Every call shares it, so two calls whose kernels overlap
// on the GPU (different streams, or different host threads) race on it; calls that follow
// each other on one stream are safe.  Each call writes all the partial sums it reads, so
// nothing needs clearing between calls.  The array's device address is looked up once per
// device and cached; cudaDeviceReset invalidates it, and a failed launch drops the cached
// address so that the next call looks it up again.
#include <mutex>

#include "../../include/bpstereo.h"
#include "bps_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_PIXELS_PER_BLOCK = 1024;  // each block adds 1024 pixels (4 per thread)

// One int64 partial sum per block, in static device memory: 128 KiB per GPU.
static __device__ __align__(256) long long g_energy_partials[BPS_NOALLOC_MAX_BLOCKS];

__device__ inline long long block_sum_i64(long long v, long long *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    long long t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    return t;
}

__global__ void __launch_bounds__(NA_THREADS)
energy_volume_partial_kernel(const int32_t *__restrict__ cost, const int32_t *__restrict__ disp, int W, int H, int D,
                             int lambda, int trunc, long long *partials) {
    __shared__ long long sh[NA_THREADS / 32];
    const int64_t n = (int64_t)W * H;
    const int64_t p0 = (int64_t)blockIdx.x * NA_PIXELS_PER_BLOCK;
    long long acc = 0;
    for (int k = threadIdx.x; k < NA_PIXELS_PER_BLOCK; k += blockDim.x) {
        const int64_t p = p0 + k;
        if (p >= n) break;
        const int x = (int)(p % W), y = (int)(p / W);
        const int d = min(max(disp[p], 0), D - 1);
        acc += cost[p * D + d];
        if (x + 1 < W) acc += (long long)lambda * min(abs(d - min(max(disp[p + 1], 0), D - 1)), trunc);
        if (y + 1 < H) acc += (long long)lambda * min(abs(d - min(max(disp[p + W], 0), D - 1)), trunc);
    }
    const long long t = block_sum_i64(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

__global__ void __launch_bounds__(NA_THREADS)
energy_volume_final_kernel(const long long *partials, int nblocks, int64_t *out) {
    __shared__ long long sh[NA_THREADS / 32];
    long long acc = 0;
    for (int k = threadIdx.x; k < nblocks; k += blockDim.x) acc += partials[k];
    const long long t = block_sum_i64(acc, sh);
    if (threadIdx.x == 0) *out = (int64_t)t;
}

// Device address of the scratch array, looked up once per device with that device current.
constexpr int NA_MAX_DEVICES = 64;
long long *g_scratch_addr[NA_MAX_DEVICES] = {};
std::mutex g_scratch_mutex;

int scratch_for_current_device(long long **out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return BPS_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_energy_partials) != cudaSuccess || !ptr) return BPS_ERR_CUDA;
        g_scratch_addr[dev] = static_cast<long long *>(ptr);
    }
    *out = g_scratch_addr[dev];
    return BPS_OK;
}

// After a failed launch (e.g. following a cudaDeviceReset) the cached address is looked up again.
void forget_scratch_for_current_device() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) return;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    g_scratch_addr[dev] = nullptr;
}

}  // namespace

extern "C" int bps_energy_noalloc(const int32_t *d_cost, const int32_t *d_disp, int W, int H, int D, int lambda,
                                  int trunc, int64_t *d_energy, void *stream) {
    if (!d_cost || !d_disp || !d_energy || W < 1 || H < 1 || D < 1 || lambda < 0 || trunc < 0) return BPS_ERR_ARG;
    const int64_t blocks = ((int64_t)W * H + NA_PIXELS_PER_BLOCK - 1) / NA_PIXELS_PER_BLOCK;
    if (blocks > BPS_NOALLOC_MAX_BLOCKS) return BPS_ERR_UNSUPPORTED;  // more pixels than the scratch covers
    long long *scratch = nullptr;
    const int rc = scratch_for_current_device(&scratch);
    if (rc != BPS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    energy_volume_partial_kernel<<<(unsigned)blocks, NA_THREADS, 0, st>>>(d_cost, d_disp, W, H, D, lambda, trunc,
                                                                          scratch);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) {
        energy_volume_final_kernel<<<1, NA_THREADS, 0, st>>>(scratch, (int)blocks, d_energy);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        forget_scratch_for_current_device();
        return BPS_ERR_CUDA;
    }
    return BPS_OK;
}
