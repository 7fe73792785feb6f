// sparse.cu -- belief propagation over sparse candidate sets at the finest scale (the abstract:
// normalised cross correlation retrieves a sparse set of candidate matches, and BP chooses among
// them).  Scales above the finest run the dense solve; at the finest scale each pixel keeps the K
// labels of lowest data cost (the lower label first among equal costs), listed in increasing
// label order, and messages are vectors over the receiver's candidates:
//     m(j) = min over the sender's candidates i of h(i) + lambda*min(|label_i - label_j|, T),
// minus their minimum, with h = cost + the incoming messages other than the receiver's.  Messages
// stay in [0, lambda*T] (the difference of two values of the minimum is at most lambda*T), so the
// u8 storage is exact, and the exact skip of the dense solve applies unchanged.
//
// Layout (colour-split like the dense arrays, slot y*Wh + x/2):
//   cand[c]  [H][Wh][Kp] uint16 labels, then costK[c] [H][Wh][Kp] int16 costs (Kp = K rounded up
//            to a power of two; entries K.. unused);
//   messages in the finest scale's dense message arrays, [H][Wh][4][Kp] bytes per colour.
// One group of Kp lanes per pixel, lane j holding candidate j.
#include <algorithm>

#include "bps_launch.h"
#include "sweep_body.cuh"

namespace bps {

__device__ __forceinline__ uint16_t *sp_labels(const SparseView &sv, int colour) { return sv.cand[colour]; }
__device__ __forceinline__ int16_t *sp_costs(const SparseView &sv, const LevelView &lv, int colour) {
    return reinterpret_cast<int16_t *>(sv.cand[colour] + (size_t)lv.H * lv.Wh * sv.Kp);
}

// ------------------------------------------------------------------ candidate selection
// Group of Gp lanes (16 labels each, the dense int16 storage order) per pixel of colour
// `colour`: K rounds of a group-wide argmin over (cost, label) pick the candidates; their rank
// in label order is the count of picked labels below them.
__global__ void candidates_kernel(LevelView lv, SparseView sv, int colour, int D, int Dp, int Gp, int K) {
    pdl_enter();
    const int g = threadIdx.x & (Gp - 1);
    const int64_t s = (int64_t)blockIdx.x * (blockDim.x / Gp) + threadIdx.x / Gp;
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    const bool in_range = s < nslot;
    const int64_t sc = in_range ? s : 0;
    const int dbase = g * VEC;
    const int16_t *cost = reinterpret_cast<const int16_t *>(colour ? lv.cost[1] : lv.cost[0]) + sc * Dp + dbase;
    unsigned key[VEC];  // cost << 16 | label, all ones for labels outside [0, D)
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        const int lab = dbase + k;
        key[k] = (dbase < Dp && lab < D) ? ((unsigned)(uint16_t)cost[label_pos<int16_t>(k)] << 16) | (unsigned)lab
                                         : 0xffffffffu;
    }
    unsigned picked = 0u;  // bit k: label dbase + k is a candidate
    for (int r = 0; r < K; ++r) {
        unsigned best = 0xffffffffu;
#pragma unroll
        for (int k = 0; k < VEC; ++k)
            if (!((picked >> k) & 1u)) best = min(best, key[k]);
        for (int o = 1; o < Gp; o <<= 1) best = min(best, __shfl_xor_sync(FULL, best, o, Gp));
        const int lab = (int)(best & 0xffffu);
        if (best != 0xffffffffu && lab >= dbase && lab < dbase + VEC) picked |= 1u << (lab - dbase);
    }
    // count of picked labels in the lower lanes of the group (inclusive scan, minus its own)
    const int mine = __popc(picked);
    int incl = mine;
    for (int o = 1; o < Gp; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o, Gp);
        if (g >= o) incl += t;
    }
    const int below = incl - mine;
    if (!in_range) return;
    uint16_t *labels = sp_labels(sv, colour) + sc * sv.Kp;
    int16_t *costs = sp_costs(sv, lv, colour) + sc * sv.Kp;
    int rank = below;
#pragma unroll
    for (int k = 0; k < VEC; ++k)
        if ((picked >> k) & 1u) {
            labels[rank] = (uint16_t)(dbase + k);
            costs[rank] = (int16_t)(key[k] >> 16);
            ++rank;
        }
}

// ------------------------------------------------------------------ coarse-to-fine gather
// Candidate j of a finest pixel starts from its parent's dense message at label_j; with no
// coarser scale, from zero.  Also sets every skip flag of the finest scale.
__global__ void sparse_start_kernel(LevelView fine, LevelView coarse, SparseView sv, int Dp_coarse, int has_parent) {
    pdl_enter();
    const int64_t nslot = (int64_t)fine.H * fine.Wh;
    const int64_t n = 2 * nslot * sv.Kp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(k % sv.Kp);
        const int64_t t = k / sv.Kp;
        const int colour = (int)(t / nslot);
        const int64_t s = t - (int64_t)colour * nslot;
        if (j == 0) fine.dirty[colour][s] = 1u;
        const int y = (int)(s / fine.Wh);
        const int x = 2 * (int)(s - (int64_t)y * fine.Wh) + ((y + colour) & 1);
        if (x >= fine.W) continue;
        uint8_t *dst = reinterpret_cast<uint8_t *>(fine.msg[colour]) + s * 4 * sv.Kp + j;
        const int lab = sp_labels(sv, colour)[s * sv.Kp + j];
        for (int q = 0; q < 4; ++q) {
            uint8_t v = 0;
            if (has_parent && j < sv.K) {
                const int px = x >> 1, py = y >> 1;
                const uint8_t *src = reinterpret_cast<const uint8_t *>(colour_of(px, py) ? coarse.msg[1] : coarse.msg[0]) +
                                     (slot_of(px, py, coarse.Wh) * 4 + q) * Dp_coarse;
                v = src[(lab / VEC) * VEC + label_pos<uint8_t>(lab % VEC)];
            }
            dst[q * sv.Kp] = v;
        }
    }
}

// ------------------------------------------------------------------ the sweep
// One block of blockDim / Kp pixels of the half-sweep.
__device__ __forceinline__ void sparse_group(const LevelView &lv, const SparseView &sv, int colour, int lam, int trunc,
                                             int skip, Tally &trace, int64_t block) {
    const int Kp = sv.Kp, K = sv.K;
    const int lane = threadIdx.x & 31;
    const int j = threadIdx.x & (Kp - 1);
    const int64_t s = block * (blockDim.x / Kp) + threadIdx.x / Kp;
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    int x = 0, y = 0;
    bool valid = false;
    if (s < nslot) {
        const unsigned su = (unsigned)s, wh = (unsigned)lv.Wh;  // slots stay below 2^31: 32-bit division
        y = (int)(su / wh);
        x = 2 * (int)(su - (unsigned)y * wh) + ((y + colour) & 1);
        valid = x < lv.W;
    }
    const int64_t sc = valid ? s : 0;
    const bool cand_lane = j < K;
    const bool has[4] = {valid && y > 0, valid && y < lv.H - 1, valid && x > 0, valid && x < lv.W - 1};
    const int nbx[4] = {x, x, x - 1, x + 1};
    const int nby[4] = {y - 1, y + 1, y, y};
    const int opp[4] = {DIR_DOWN, DIR_UP, DIR_RIGHT, DIR_LEFT};
    unsigned *dirty_in = colour ? lv.dirty[1] : lv.dirty[0];
    unsigned *dirty_out = colour ? lv.dirty[0] : lv.dirty[1];
    const uint8_t *msg_in = reinterpret_cast<const uint8_t *>(colour ? lv.msg[1] : lv.msg[0]) + sc * 4 * Kp + j;
    uint8_t *msg_out = reinterpret_cast<uint8_t *>(colour ? lv.msg[0] : lv.msg[1]);
    const uint16_t *lab_out = sp_labels(sv, colour ^ 1);
    // every load at once: flag, own candidate, incoming, receivers' candidates and old messages
    const unsigned flag = valid ? dirty_in[s] : 0u;
    const int lab = (int)sp_labels(sv, colour)[sc * Kp + j];
    int b = cand_lane ? (int)sp_costs(sv, lv, colour)[sc * Kp + j] : 0;
    int in[4], rlab[4], old[4];
    int64_t rs[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        in[q] = has[q] ? (int)msg_in[q * Kp] : 0;
        rs[q] = has[q] ? slot_of(nbx[q], nby[q], lv.Wh) : 0;
        rlab[q] = (int)lab_out[rs[q] * Kp + j];
        old[q] = (skip && has[q]) ? (int)msg_out[(rs[q] * 4 + opp[q]) * Kp + j] : 0;
    }
    const bool active = valid && (!skip || flag == 1u);
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) return;
    trace.add(act, Kp);
#pragma unroll
    for (int q = 0; q < 4; ++q) b += in[q];
    const int BIG = 1 << 28;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int h = cand_lane ? b - in[q] : BIG;
        int v = BIG;
        for (int i = 0; i < K; ++i) {
            const int hi = __shfl_sync(FULL, h, i, Kp);
            const int li = __shfl_sync(FULL, lab, i, Kp);
            v = min(v, hi + lam * min(abs(li - rlab[q]), trunc));
        }
        int mn = cand_lane ? v : BIG;
        for (int o = 1; o < Kp; o <<= 1) mn = min(mn, __shfl_xor_sync(FULL, mn, o, Kp));
        const int m = v - mn;  // in [0, lambda*T] on candidate lanes
        const bool send = active && has[q];
        if (skip) {
            const unsigned dm = __ballot_sync(FULL, send && cand_lane && m != old[q]);
            const bool changed = ((dm >> (lane & ~(Kp - 1))) & group_bits(Kp)) != 0u;
            if (send && changed) {
                if (cand_lane) msg_out[(rs[q] * 4 + opp[q]) * Kp + j] = (uint8_t)m;
                if (j == 0) dirty_out[rs[q]] = 1u;
            }
        } else if (send && cand_lane) {
            msg_out[(rs[q] * 4 + opp[q]) * Kp + j] = (uint8_t)m;
        }
    }
    if (skip && active && j == 0) dirty_in[s] = 0u;
}

// Grid-stride over the pixel blocks with the CTAs resident at once (the trace count of a warp is
// added once, at the end).
__global__ void __launch_bounds__(256)
sparse_sweep_kernel(LevelView lv, SparseView sv, int colour, int lam, int trunc, int skip, unsigned long long *trace,
                    int64_t nblocks) {
    pdl_enter();
    Tally tally(trace);
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) sparse_group(lv, sv, colour, lam, trunc, skip, tally, b);
    tally.flush();
}

// ------------------------------------------------------------------ read-out
// Pixels in raster order, Kp lanes each: the candidate of least belief, the lowest label on ties.
__global__ void sparse_wta_kernel(LevelView lv, SparseView sv, int32_t *disp) {
    pdl_enter();
    const int Kp = sv.Kp;
    const int j = threadIdx.x & (Kp - 1);
    const int64_t p = (int64_t)blockIdx.x * (blockDim.x / Kp) + threadIdx.x / Kp;
    const bool valid = p < (int64_t)lv.W * lv.H;
    const int x = valid ? (int)(p % lv.W) : 0, y = valid ? (int)(p / lv.W) : 0;
    const int c = colour_of(x, y);
    const int64_t s = slot_of(x, y, lv.Wh);
    long long key = 0x7fffffffffffffffLL;  // belief << 16 | label
    if (valid && j < sv.K) {
        int b = sp_costs(sv, lv, c)[s * Kp + j];
        const uint8_t *mp = reinterpret_cast<const uint8_t *>(c ? lv.msg[1] : lv.msg[0]) + s * 4 * Kp + j;
        const bool has[4] = {y > 0, y < lv.H - 1, x > 0, x < lv.W - 1};
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (has[q]) b += mp[q * Kp];
        key = ((long long)b << 16) | (long long)sp_labels(sv, c)[s * Kp + j];
    }
    for (int o = 1; o < Kp; o <<= 1) key = min(key, __shfl_xor_sync(FULL, key, o, Kp));
    if (valid && j == 0) disp[p] = (int32_t)(key & 0xffff);
}

// ------------------------------------------------------------------ export (natural layout)
__global__ void sparse_export_kernel(LevelView lv, SparseView sv, int32_t *cand, int32_t *msg) {
    pdl_enter();  // launched with programmatic serialisation: wait for the solve's last kernel
    const int64_t n = (int64_t)lv.W * lv.H * sv.K;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int j = (int)(k % sv.K);
        const int64_t p = k / sv.K;
        const int x = (int)(p % lv.W), y = (int)(p / lv.W);
        const int c = colour_of(x, y);
        const int64_t s = slot_of(x, y, lv.Wh);
        cand[k] = sp_labels(sv, c)[s * sv.Kp + j];
        const uint8_t *mp = reinterpret_cast<const uint8_t *>(c ? lv.msg[1] : lv.msg[0]) + s * 4 * sv.Kp + j;
        for (int q = 0; q < 4; ++q) msg[(int64_t)q * n + k] = mp[q * sv.Kp];
    }
}

static unsigned grid_of(int64_t threads) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((threads + 255) / 256, 65535)); }

cudaError_t launch_sparse_candidates(const LevelView &lv, const SparseView &sv, int D, int Dp, int Gp, cudaStream_t st) {
    const int groups = 256 / Gp;
    const int64_t blocks = ((int64_t)lv.H * lv.Wh + groups - 1) / groups;
    for (int colour = 0; colour < 2; ++colour) {
        const cudaError_t e =
            launch_k(candidates_kernel, dim3((unsigned)blocks), dim3(256), 0, st, lv, sv, colour, D, Dp, Gp, sv.K);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_sparse_start(const LevelView &fine, const LevelView *coarse, const SparseView &sv, int Dp,
                                cudaStream_t st) {
    const int64_t n = 2 * (int64_t)fine.H * fine.Wh * sv.Kp;
    return launch_k(sparse_start_kernel, dim3(grid_of(n)), dim3(256), 0, st, fine, coarse ? *coarse : fine, sv, Dp,
                    coarse ? 1 : 0);
}

cudaError_t launch_sparse_sweep(const LevelView &lv, const SparseView &sv, int colour, int lambda, int trunc, int skip,
                                unsigned long long *trace, cudaStream_t st) {
    const int groups = 256 / sv.Kp;
    const int64_t blocks = ((int64_t)lv.H * lv.Wh + groups - 1) / groups;
    if (blocks == 0) return cudaSuccess;
    static int resident = 0;  // CTAs resident at once (looked up once per process)
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sparse_sweep_kernel, 256, 0);
        resident = std::max(1, sms * std::max(1, per_sm));
    }
    const int lam = trunc == 0 ? 0 : lambda;
    return launch_k(sparse_sweep_kernel, dim3((unsigned)std::min<int64_t>(blocks, resident)), dim3(256), 0, st, lv, sv,
                    colour, lam, trunc, skip, trace, blocks);
}

cudaError_t launch_sparse_wta(const LevelView &lv, const SparseView &sv, int32_t *disp, cudaStream_t st) {
    const int groups = 256 / sv.Kp;
    const int64_t blocks = ((int64_t)lv.W * lv.H + groups - 1) / groups;
    return launch_k(sparse_wta_kernel, dim3((unsigned)blocks), dim3(256), 0, st, lv, sv, disp);
}

cudaError_t launch_sparse_export(const LevelView &lv, const SparseView &sv, int32_t *cand, int32_t *msg,
                                 cudaStream_t st) {
    return launch_k(sparse_export_kernel, dim3(grid_of((int64_t)lv.W * lv.H * sv.K)), dim3(256), 0, st, lv, sv, cand,
                    msg);
}

cudaError_t preload_sparse_kernels() {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, candidates_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sparse_start_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sparse_sweep_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sparse_wta_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sparse_export_kernel);
    return e;
}

}  // namespace bps
