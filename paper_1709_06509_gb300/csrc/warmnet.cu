// warmnet.cu -- kernels of the learned warm start: a small convolutional network that
// predicts the coarsest scale's messages from the coarsest cost volume, so that the
// hierarchical BP starts closer to its fixed point.  The paper has no such network; its
// role is the warm start the solve accepts (bps_bp_solve with BPS_FLAG_WARM_START).
//
// Layout: activations [B][C][H][W] in BF16, weights [Cout][Cin][3][3] in BF16 (training keeps
// FP32 master copies), biases, gradients and optimiser state in FP32; every product is
// accumulated in FP32.  3x3 convolutions with zero padding ("same" size).  The forward
// convolution of BF16 activations (every layer of the network) runs on the tensor cores
// (conv_tc.cu); the FP32-input forward and the backward kernels below are direct convolutions
// on the CUDA cores, one thread per output element (training only).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "../../include/bpstereo.h"
#include "bps_internal.cuh"

namespace {

constexpr int WN_THREADS = 256;

inline unsigned blocks_for(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + WN_THREADS - 1) / WN_THREADS); }

__device__ inline float ld_act(const void *p, int64_t i, int bf16) {
    return bf16 ? __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]) : reinterpret_cast<const float *>(p)[i];
}

// out[b][co][y][x] = bias[co] + sum_{ci,ky,kx} in[b][ci][y+ky-1][x+kx-1] * w[co][ci][ky][kx]
__global__ void conv3x3_fwd_kernel(const void *in, int in_bf16, int B, int Cin, int H, int W,
                                   const __nv_bfloat16 *__restrict__ w, const float *__restrict__ bias, int Cout,
                                   int relu, void *out, int out_bf16) {
    const int64_t n = (int64_t)B * Cout * H * W;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % W);
        int64_t r = k / W;
        const int y = (int)(r % H);
        r /= H;
        const int co = (int)(r % Cout);
        const int b = (int)(r / Cout);
        float acc = bias ? bias[co] : 0.f;
        for (int ci = 0; ci < Cin; ++ci) {
            const int64_t ib = ((int64_t)b * Cin + ci) * H * W;
            const __nv_bfloat16 *wk = w + ((int64_t)co * Cin + ci) * 9;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int yy = y + ky - 1;
                if (yy < 0 || yy >= H) continue;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int xx = x + kx - 1;
                    if (xx < 0 || xx >= W) continue;
                    acc += ld_act(in, ib + (int64_t)yy * W + xx, in_bf16) * __bfloat162float(wk[ky * 3 + kx]);
                }
            }
        }
        if (relu) acc = fmaxf(acc, 0.f);
        if (out_bf16) reinterpret_cast<__nv_bfloat16 *>(out)[k] = __float2bfloat16_rn(acc);
        else reinterpret_cast<float *>(out)[k] = acc;
    }
}

// din[b][ci][y][x] = sum_{co,ky,kx} g[b][co][y-ky+1][x-kx+1] * w[co][ci][ky][kx], where g is the
// output gradient, masked by the forward ReLU (out > 0) when relu_out is given.
__global__ void conv3x3_bwd_data_kernel(const float *__restrict__ gout, const void *relu_out, int B, int Cout, int H,
                                        int W, const __nv_bfloat16 *__restrict__ w, int Cin, float *din) {
    const int64_t n = (int64_t)B * Cin * H * W;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % W);
        int64_t r = k / W;
        const int y = (int)(r % H);
        r /= H;
        const int ci = (int)(r % Cin);
        const int b = (int)(r / Cin);
        float acc = 0.f;
        for (int co = 0; co < Cout; ++co) {
            const int64_t gb = ((int64_t)b * Cout + co) * H * W;
            const __nv_bfloat16 *wk = w + ((int64_t)co * Cin + ci) * 9;
#pragma unroll
            for (int ky = 0; ky < 3; ++ky) {
                const int yy = y - ky + 1;
                if (yy < 0 || yy >= H) continue;
#pragma unroll
                for (int kx = 0; kx < 3; ++kx) {
                    const int xx = x - kx + 1;
                    if (xx < 0 || xx >= W) continue;
                    const int64_t gi = gb + (int64_t)yy * W + xx;
                    float g = gout[gi];
                    if (relu_out && __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(relu_out)[gi]) <= 0.f)
                        g = 0.f;
                    acc += g * __bfloat162float(wk[ky * 3 + kx]);
                }
            }
        }
        din[k] = acc;
    }
}

// One CTA per (co, ci): dw[co][ci][ky][kx] = sum_{b,y,x} g[b][co][y][x] in[b][ci][y+ky-1][x+kx-1]
// (g masked by the forward ReLU as above); CTAs with ci == 0 also form db[co] = sum g.
__global__ void __launch_bounds__(WN_THREADS)
conv3x3_bwd_weight_kernel(const float *__restrict__ gout, const void *relu_out, const void *in, int in_bf16, int B,
                          int Cin, int H, int W, int Cout, float *dw, float *db) {
    const int co = blockIdx.x / Cin, ci = blockIdx.x % Cin;
    float acc[10];
#pragma unroll
    for (int t = 0; t < 10; ++t) acc[t] = 0.f;
    const int64_t n = (int64_t)B * H * W;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) {
        const int x = (int)(k % W);
        const int y = (int)((k / W) % H);
        const int b = (int)(k / ((int64_t)H * W));
        const int64_t gi = ((int64_t)b * Cout + co) * H * W + (int64_t)y * W + x;
        float g = gout[gi];
        if (relu_out && __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(relu_out)[gi]) <= 0.f) g = 0.f;
        if (g == 0.f) continue;
        const int64_t ib = ((int64_t)b * Cin + ci) * H * W;
#pragma unroll
        for (int ky = 0; ky < 3; ++ky) {
            const int yy = y + ky - 1;
            if (yy < 0 || yy >= H) continue;
#pragma unroll
            for (int kx = 0; kx < 3; ++kx) {
                const int xx = x + kx - 1;
                if (xx < 0 || xx >= W) continue;
                acc[ky * 3 + kx] += g * ld_act(in, ib + (int64_t)yy * W + xx, in_bf16);
            }
        }
        acc[9] += g;
    }
    __shared__ float sh[WN_THREADS / 32][10];
#pragma unroll
    for (int t = 0; t < 10; ++t) {
        float v = acc[t];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5][t] = v;
    }
    __syncthreads();
    if (threadIdx.x < 10) {
        float v = 0.f;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) v += sh[wv][threadIdx.x];
        if (threadIdx.x < 9) dw[((int64_t)co * Cin + ci) * 9 + threadIdx.x] = v;
        else if (ci == 0 && db) db[co] = v;
    }
}

// Masked mean squared error: loss_part[block] partial sums, grad = 2 (pred - target) mask / count.
__global__ void __launch_bounds__(WN_THREADS)
mse_kernel(const float *__restrict__ pred, const float *__restrict__ target, const float *__restrict__ mask, int64_t n,
           float inv_count, float *grad, float *loss_part) {
    float acc = 0.f;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float m = mask ? mask[k] : 1.f;
        const float d = (pred[k] - target[k]) * m;
        acc += d * d;
        grad[k] = 2.f * d * inv_count;
    }
    __shared__ float sh[WN_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = 0.f;
        for (int wv = 0; wv < (int)(blockDim.x >> 5); ++wv) v += sh[wv];
        loss_part[blockIdx.x] = v * inv_count;
    }
}

// Adam (Kingma & Ba 2015) on FP32 master weights; the BF16 copy used by the kernels follows.
__global__ void adam_kernel(float *w, float *m, float *v, const float *g, int64_t n, float lr, float b1, float b2,
                            float eps, float bc1, float bc2, __nv_bfloat16 *w_bf16) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float gk = g[k];
        const float mk = b1 * m[k] + (1.f - b1) * gk;
        const float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        const float wk = w[k] - lr * (mk / bc1) / (sqrtf(vk / bc2) + eps);
        w[k] = wk;
        if (w_bf16) w_bf16[k] = __float2bfloat16_rn(wk);
    }
}

// Network input from a natural-layout int32 cost volume [H][W][D]: channel g is the minimum of
// labels [8g, 8g + 8) minus the pixel's minimum over all labels, times `scale`.
__global__ void features_kernel(const int32_t *__restrict__ cost, int H, int W, int D, float scale,
                                __nv_bfloat16 *feat) {
    const int C = (D + 7) / 8;
    const int64_t n = (int64_t)H * W;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x) {
        const int32_t *c = cost + p * D;
        int mn = c[0];
        for (int d = 1; d < D; ++d) mn = min(mn, c[d]);
        for (int g = 0; g < C; ++g) {
            int gm = c[8 * g];
            for (int d = 8 * g + 1; d < min(D, 8 * g + 8); ++d) gm = min(gm, c[d]);
            feat[(int64_t)g * n + p] = __float2bfloat16_rn((float)(gm - mn) * scale);
        }
    }
}

// Start messages from the network output pred[4 * D][H][W] (channel q * D + d): rounded to
// integers, clamped to [0, cap], shifted so that each message's minimum is 0, and 0 in the
// slots of neighbours outside the image; natural layout [4][H][W][D].
__global__ void messages_kernel(const float *__restrict__ pred, int H, int W, int D, int cap, int32_t *init) {
    const int64_t n = 4LL * H * W;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(k % W);
        const int y = (int)((k / W) % H);
        const int q = (int)(k / ((int64_t)H * W));
        const bool has = q == 0 ? y > 0 : q == 1 ? y < H - 1 : q == 2 ? x > 0 : x < W - 1;
        int32_t *dst = init + k * D;
        if (!has) {
            for (int d = 0; d < D; ++d) dst[d] = 0;
            continue;
        }
        int mn = cap;
        for (int d = 0; d < D; ++d) {
            const int v = min(max(__float2int_rn(pred[((int64_t)q * D + d) * H * W + (int64_t)y * W + x]), 0), cap);
            dst[d] = v;
            mn = min(mn, v);
        }
        for (int d = 0; d < D; ++d) dst[d] -= mn;
    }
}

}  // namespace

#define WN_CK(x)                                                 \
    do {                                                         \
        if ((x) != cudaSuccess) return BPS_ERR_CUDA;             \
    } while (0)

namespace bps {
cudaError_t launch_conv3x3_tc(const void *in, int B, int Cin, int H, int W, const void *w, const float *bias, int Cout,
                              int relu, void *out, int out_bf16, cudaStream_t st);
int conv3x3_tc_error(int *flag);
}  // namespace bps

extern "C" int bps_warmnet_conv3x3(const void *d_in, int in_bf16, int B, int Cin, int H, int W, const void *d_w,
                                   const float *d_bias, int Cout, int relu, void *d_out, int out_bf16, void *stream) {
    if (!d_in || !d_w || !d_out || B < 1 || Cin < 1 || Cout < 1 || H < 1 || W < 1) return BPS_ERR_ARG;
    if ((int64_t)Cin * 9 > (1 << 20) || (int64_t)B * H * W > ((int64_t)1 << 31)) return BPS_ERR_ARG;
    if (in_bf16) {  // BF16 activations: an implicit GEMM on the tensor cores (conv_tc.cu)
        WN_CK(bps::launch_conv3x3_tc(d_in, B, Cin, H, W, d_w, d_bias, Cout, relu, d_out, out_bf16,
                                     (cudaStream_t)stream));
        return BPS_OK;
    }
    const int64_t n = (int64_t)B * Cout * H * W;
    conv3x3_fwd_kernel<<<std::min<unsigned>(blocks_for(n), 152 * 64), WN_THREADS, 0, (cudaStream_t)stream>>>(
        d_in, in_bf16, B, Cin, H, W, (const __nv_bfloat16 *)d_w, d_bias, Cout, relu, d_out, out_bf16);
    WN_CK(cudaGetLastError());
    return BPS_OK;
}

extern "C" int bps_warmnet_get_error(void) {
    int flag = 0;
    const int rc = bps::conv3x3_tc_error(&flag);
    if (rc != BPS_OK) return rc;
    return flag ? BPS_ERR_TIMEOUT : BPS_OK;
}

extern "C" int bps_warmnet_conv3x3_backward(const float *d_gout, const void *d_relu_out, const void *d_in, int in_bf16,
                                            int B, int Cin, int H, int W, const void *d_w, int Cout, float *d_gin,
                                            float *d_gw, float *d_gb, void *stream) {
    if (!d_gout || !d_in || !d_w || !d_gw || B < 1 || Cin < 1 || Cout < 1 || H < 1 || W < 1) return BPS_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    conv3x3_bwd_weight_kernel<<<Cout * Cin, WN_THREADS, 0, st>>>(d_gout, d_relu_out, d_in, in_bf16, B, Cin, H, W, Cout,
                                                                 d_gw, d_gb);
    WN_CK(cudaGetLastError());
    if (d_gin) {
        const int64_t n = (int64_t)B * Cin * H * W;
        conv3x3_bwd_data_kernel<<<std::min<unsigned>(blocks_for(n), 152 * 64), WN_THREADS, 0, st>>>(
            d_gout, d_relu_out, B, Cout, H, W, (const __nv_bfloat16 *)d_w, Cin, d_gin);
        WN_CK(cudaGetLastError());
    }
    return BPS_OK;
}

extern "C" int bps_warmnet_mse(const float *d_pred, const float *d_target, const float *d_mask, int64_t n,
                               float *d_grad, float *d_loss_parts, int nparts, void *stream) {
    if (!d_pred || !d_target || !d_grad || !d_loss_parts || n < 1 || nparts < 1) return BPS_ERR_ARG;
    float count = (float)n;
    mse_kernel<<<nparts, WN_THREADS, 0, (cudaStream_t)stream>>>(d_pred, d_target, d_mask, n, 1.f / count, d_grad,
                                                                d_loss_parts);
    WN_CK(cudaGetLastError());
    return BPS_OK;
}

extern "C" int bps_warmnet_adam(float *d_w, float *d_m, float *d_v, const float *d_g, int64_t n, float lr, float beta1,
                                float beta2, float eps, int step, void *d_w_bf16, void *stream) {
    if (!d_w || !d_m || !d_v || !d_g || n < 1 || step < 1) return BPS_ERR_ARG;
    const float bc1 = 1.f - powf(beta1, (float)step), bc2 = 1.f - powf(beta2, (float)step);
    adam_kernel<<<std::min<unsigned>(blocks_for(n), 4096), WN_THREADS, 0, (cudaStream_t)stream>>>(
        d_w, d_m, d_v, d_g, n, lr, beta1, beta2, eps, bc1, bc2, (__nv_bfloat16 *)d_w_bf16);
    WN_CK(cudaGetLastError());
    return BPS_OK;
}

extern "C" int bps_warmnet_features(const int32_t *d_cost, int H, int W, int D, float scale, void *d_feat,
                                    void *stream) {
    if (!d_cost || !d_feat || H < 1 || W < 1 || D < 1) return BPS_ERR_ARG;
    features_kernel<<<blocks_for((int64_t)H * W), WN_THREADS, 0, (cudaStream_t)stream>>>(d_cost, H, W, D, scale,
                                                                                        (__nv_bfloat16 *)d_feat);
    WN_CK(cudaGetLastError());
    return BPS_OK;
}

extern "C" int bps_warmnet_messages(const float *d_pred, int H, int W, int D, int cap, int32_t *d_init, void *stream) {
    if (!d_pred || !d_init || H < 1 || W < 1 || D < 1 || cap < 0) return BPS_ERR_ARG;
    messages_kernel<<<blocks_for(4LL * H * W), WN_THREADS, 0, (cudaStream_t)stream>>>(d_pred, H, W, D, cap, d_init);
    WN_CK(cudaGetLastError());
    return BPS_OK;
}
