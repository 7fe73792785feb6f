// conv_tc.cu -- the learned warm start's 3x3 convolution (BF16 activations and weights, FP32
// accumulation) as an implicit GEMM on the fifth-generation tensor cores (tcgen05).
//
// out[b][co][y][x] = bias[co] + sum_{ci,ky,kx} in[b][ci][y+ky-1][x+kx-1] w[co][ci][ky][kx]
// is D[m][n] = sum_k A[m][k] B[n][k] with m a pixel (b, y, x), n an output channel and
// k = (ci, ky, kx) = ci * 9 + ky * 3 + kx (the weights' own row-major order).  A CTA owns 128
// consecutive pixels (M = 128) and up to 256 output channels (N): its accumulator is a
// 128-lane x N-column FP32 tile of tensor memory.  K runs in chunks of 32: the CTA's threads
// write the chunk of A (the im2col of the input, zero outside the image and past K) and of B
// (the weights) into shared memory in the canonical K-major layout without swizzle (8-row x
// 16-byte core matrices; 128 bytes between core matrices along K, 512 bytes along M / N), one
// thread issues the chunk's two MMAs (K = 16 each) and commits them to an mbarrier, and the CTA
// waits for it before reusing the buffers.  The epilogue reads the accumulator with tcgen05.ld
// (warp w holds lanes 32w .. 32w + 31, i.e. pixels), adds the bias, applies the ReLU and stores
// NCHW (consecutive pixels of a channel: coalesced).  The wait is bounded; a wait that gives up
// sets the error word (bps_warmnet_get_error), skips the epilogue and still frees the tensor
// memory.
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "../../include/bpstereo.h"
#include "bps_internal.cuh"

namespace {

constexpr int TC_M = 128;          // pixels a CTA
constexpr int TC_KC = 32;          // K a chunk (two MMAs of K = 16)
constexpr int TC_NMAX = 256;       // output channels a CTA
constexpr int TC_THREADS = 128;    // four warps: one per 32 lanes of tensor memory
constexpr unsigned TC_WAIT_LIMIT = 1u << 24;

static __device__ unsigned g_conv_tc_error;  // 1 when a bounded wait of the kernel gave up

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor of a K-major operand without swizzle: start address, the byte
// offset between core matrices adjacent along K (leading) and along M / N (stride), the
// descriptor version of this architecture (bits 46-47 = 1), no base offset, layout 0.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16 A and B (bits 7-9
// and 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 in bits 17-22, M / 16 in bits 24-28.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ bool wait_phase(uint64_t *bar, unsigned parity) {
    for (unsigned it = 0; it < TC_WAIT_LIMIT; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    atomicExch(&g_conv_tc_error, 1u);
    return false;
}

__global__ void __launch_bounds__(TC_THREADS)
conv3x3_tc_kernel(const __nv_bfloat16 *__restrict__ in, int B, int Cin, int H, int W,
                  const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias, int Cout, int relu, void *out,
                  int out_bf16, int ncols) {
    // A chunk [16 row groups][4 k groups][8 rows][16 B], B chunk [N / 8 row groups][4][8][16 B]
    __shared__ __align__(128) unsigned char smA[TC_M * TC_KC * 2];
    __shared__ __align__(128) unsigned char smB[TC_NMAX * TC_KC * 2];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int HW = H * W;
    const int64_t npix = (int64_t)B * HW;
    const int64_t p0 = (int64_t)blockIdx.x * TC_M;
    const int n0 = blockIdx.y * TC_NMAX;
    const int NT = min(TC_NMAX, ((Cout - n0) + 15) / 16 * 16);  // this CTA's N, a multiple of 16
    const int K = Cin * 9;
    const int nchunks = (K + TC_KC - 1) / TC_KC;

    if (warp == 0) {  // the accumulator: `ncols` (a power of two >= 32 and >= NT) FP32 columns
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_slot)),
                     "r"(ncols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = tmem_slot;

    // this thread's pixel (row m = tid of A)
    const int64_t p = p0 + tid;
    const bool pix_ok = p < npix;
    const int b = pix_ok ? (int)(p / HW) : 0;
    const int pp = pix_ok ? (int)(p % HW) : 0;
    const int y = pp / W, x = pp % W;
    const __nv_bfloat16 *inb = in + (int64_t)b * Cin * HW;
    const uint32_t idesc = instr_desc(TC_M, NT);
    bool ok = true;

    for (int c = 0; c < nchunks && ok; ++c) {
        const int k0 = c * TC_KC;
        // A: row m = tid, four 16-byte k groups
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t v[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
                unsigned short h[2];
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int k = k0 + 8 * j + e + t;
                    unsigned short bits = 0;
                    if (pix_ok && k < K) {
                        const int ci = k / 9, r = k - ci * 9, ky = r / 3, kx = r - ky * 3;
                        const int yy = y + ky - 1, xx = x + kx - 1;
                        if (yy >= 0 && yy < H && xx >= 0 && xx < W)
                            bits = __bfloat16_as_ushort(inb[(int64_t)ci * HW + yy * W + xx]);
                    }
                    h[t] = bits;
                }
                v[e >> 1] = (uint32_t)h[0] | ((uint32_t)h[1] << 16);
            }
            *reinterpret_cast<uint4 *>(smA + (tid >> 3) * 512 + j * 128 + (tid & 7) * 16) = make_uint4(v[0], v[1], v[2], v[3]);
        }
        // B: rows n of this CTA's NT channels (zero past Cout and past K)
        for (int n = tid; n < NT; n += TC_THREADS) {
            const int co = n0 + n;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                uint32_t v[4];
#pragma unroll
                for (int e = 0; e < 8; e += 2) {
                    const int k = k0 + 8 * j + e;
                    const unsigned short lo =
                        (co < Cout && k < K) ? __bfloat16_as_ushort(w[(int64_t)co * K + k]) : (unsigned short)0;
                    const unsigned short hi =
                        (co < Cout && k + 1 < K) ? __bfloat16_as_ushort(w[(int64_t)co * K + k + 1]) : (unsigned short)0;
                    v[e >> 1] = (uint32_t)lo | ((uint32_t)hi << 16);
                }
                *reinterpret_cast<uint4 *>(smB + (n >> 3) * 512 + j * 128 + (n & 7) * 16) =
                    make_uint4(v[0], v[1], v[2], v[3]);
            }
        }
        // the tensor core reads shared memory through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int s = 0; s < 2; ++s) {  // K = 16 each: two core matrices along K
                const uint64_t ad = smem_desc(smem_addr(smA) + s * 256, 128, 512);
                const uint64_t bd = smem_desc(smem_addr(smB) + s * 256, 128, 512);
                const uint32_t acc = (c > 0 || s > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&mbar))
                         : "memory");
        }
        // the MMAs of this chunk have read the buffers (and written the accumulator)
        ok = wait_phase(&mbar, (unsigned)(c & 1));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        __syncthreads();
    }

    if (ok) {
        // epilogue: lane (pixel) 32 warp + lane, eight columns (channels) a load
        const uint32_t lane_base = tmem + ((uint32_t)(32 * warp) << 16);
        for (int nc = 0; nc < NT; nc += 8) {
            uint32_t r[8];
            // the load and its wait in one statement: the load writes its registers asynchronously
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
                "tcgen05.wait::ld.sync.aligned;"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                : "r"(lane_base + (uint32_t)nc)
                : "memory");
            const int64_t q = p0 + 32 * warp + lane;
            if (q < npix) {
                const int qb = (int)(q / HW), qp = (int)(q % HW);
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const int co = n0 + nc + t;
                    if (co >= Cout) break;
                    float v = __uint_as_float(r[t]) + (bias ? bias[co] : 0.f);
                    if (relu) v = fmaxf(v, 0.f);
                    const int64_t o = ((int64_t)qb * Cout + co) * HW + qp;
                    if (out_bf16) reinterpret_cast<__nv_bfloat16 *>(out)[o] = __float2bfloat16_rn(v);
                    else reinterpret_cast<float *>(out)[o] = v;
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(ncols) : "memory");
}

std::mutex g_err_mutex;
unsigned *g_err_addr[64] = {};

}  // namespace

namespace bps {

// The forward 3x3 convolution of BF16 activations on the tensor cores (see the file comment).
cudaError_t launch_conv3x3_tc(const void *in, int B, int Cin, int H, int W, const void *w, const float *bias, int Cout,
                              int relu, void *out, int out_bf16, cudaStream_t st) {
    const int64_t npix = (int64_t)B * H * W;
    const dim3 grid((unsigned)((npix + TC_M - 1) / TC_M), (unsigned)((Cout + TC_NMAX - 1) / TC_NMAX));
    const int nt = std::min(TC_NMAX, (std::min(Cout, TC_NMAX) + 15) / 16 * 16);
    int ncols = 32;
    while (ncols < nt) ncols *= 2;
    conv3x3_tc_kernel<<<grid, TC_THREADS, 0, st>>>(reinterpret_cast<const __nv_bfloat16 *>(in), B, Cin, H, W,
                                                     reinterpret_cast<const __nv_bfloat16 *>(w), bias, Cout, relu, out,
                                                     out_bf16, ncols);
    return cudaGetLastError();
}

// 1 when a bounded wait of the tensor-core convolution gave up since the last call (cleared).
int conv3x3_tc_error(int *flag) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return BPS_ERR_CUDA;
    unsigned *addr = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_err_mutex);
        if (!g_err_addr[dev]) {
            void *p = nullptr;
            if (cudaGetSymbolAddress(&p, g_conv_tc_error) != cudaSuccess) return BPS_ERR_CUDA;
            g_err_addr[dev] = static_cast<unsigned *>(p);
        }
        addr = g_err_addr[dev];
    }
    unsigned v = 0;
    if (cudaMemcpy(&v, addr, sizeof(v), cudaMemcpyDeviceToHost) != cudaSuccess) return BPS_ERR_CUDA;
    if (v && cudaMemset(addr, 0, sizeof(v)) != cudaSuccess) return BPS_ERR_CUDA;
    *flag = v ? 1 : 0;
    return BPS_OK;
}

}  // namespace bps
