// sweep_f16_body.cuh -- the per-pixel work of the fp16-message form's red-black half-sweep in
// packed half2 arithmetic (truncation T <= 2), shared by the one-launch-per-half-sweep kernels
// (sweep_f16.cu) and the persistent batched kernel (persist.cu).
//
// Same layout and label order as the generic form: float costs, fp16 messages, labels 2j and
// 2j+1 in one half2 register j of a lane's 16.  Per pixel the belief is formed from the costs
// minus their minimum over the pixel's labels: a constant per pixel changes no message and no
// read-out, and it keeps every value that can decide a message small: the minimum of h is at
// most three messages, 3 lambda T, above zero, so those values lie below 4 lambda T (80 at
// lambda T = 20, where half precision steps by 1/16 at most; a message itself, at most
// lambda T, by 1/64).  The truncated-linear minimisation is the stencil of the u8 form:
// m(d) = min(h(d), h(d±1) + lambda, min h + lambda T) - min h for T = 2,
// min(h(d), min h + lambda T) - min h for T <= 1.
#pragma once

#include <cuda_fp16.h>

#include "sweep_body.cuh"

namespace bps {

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *reinterpret_cast<uint32_t *>(&h); }
__device__ __forceinline__ __half2 u2h(uint32_t u) { return *reinterpret_cast<__half2 *>(&u); }
__device__ __forceinline__ uint32_t word(const uint4 (&v)[2], int j) {
    const uint4 &w = v[j >> 2];
    return (j & 3) == 0 ? w.x : (j & 3) == 1 ? w.y : (j & 3) == 2 ? w.z : w.w;
}

// APPEND: newly dirty neighbours are appended to the other colour's active list (one
// reservation a warp).  LISTED: the slot is the caller's list entry (nslot for none); a listed
// pixel is dirty by construction, so its flag is not read.  RW: messages are read with coherent
// loads (a kernel that wrote them earlier in the same launch, across a grid barrier).
template <bool PADDED, int TS, bool EAGER, bool APPEND = false, bool LISTED = false, bool RW = false>
__device__ __forceinline__ void sweep_group_f16(const LevelView &lv, int colour, int D, int Dp, int Gp, float lam,
                                                float lamT, int skip, Tally &trace, int64_t block,
                                                const ActiveList &al = ActiveList{nullptr, nullptr, nullptr, nullptr},
                                                int64_t s_listed = 0) {
    const int lane = threadIdx.x & 31;
    const int g = threadIdx.x & (Gp - 1);
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    const int64_t s = LISTED ? s_listed : block * (blockDim.x / Gp) + threadIdx.x / Gp;
    int x = 0, y = 0;
    bool valid = false;
    if (s < nslot) {
        const unsigned su = (unsigned)s, wh = (unsigned)lv.Wh;  // slots stay below 2^31: 32-bit division
        y = (int)(su / wh);
        x = 2 * (int)(su - (unsigned)y * wh) + ((y + colour) & 1);
        valid = x < lv.W;
    }
    const int64_t sc = valid ? s : 0;
    const int dbase = g * VEC;
    const bool lane_data = dbase < Dp;
    const bool has[4] = {valid && y > 0, valid && y < lv.H - 1, valid && x > 0, valid && x < lv.W - 1};
    const int nbx[4] = {x, x, x - 1, x + 1};
    const int nby[4] = {y - 1, y + 1, y, y};
    const int opp[4] = {DIR_DOWN, DIR_UP, DIR_RIGHT, DIR_LEFT};
    const float *cost = reinterpret_cast<const float *>(colour ? lv.cost[1] : lv.cost[0]);
    const __half *msg_in = reinterpret_cast<const __half *>(colour ? lv.msg[1] : lv.msg[0]);
    __half *msg_out = reinterpret_cast<__half *>(colour ? lv.msg[0] : lv.msg[1]);
    unsigned *dirty_in = colour ? lv.dirty[1] : lv.dirty[0];
    unsigned *dirty_out = colour ? lv.dirty[0] : lv.dirty[1];

    float c[VEC];
    uint4 in[4][2], old[4][2];
    uint4 *dst[4];
    unsigned qsv[4];
    auto load_cost = [&]() {
        const float4 *cp = reinterpret_cast<const float4 *>(cost + (lane_data ? sc * Dp + dbase : 0));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float4 v = lane_data ? __ldg(cp + k) : make_float4(0.f, 0.f, 0.f, 0.f);
            c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
        }
    };
    auto load_messages = [&](bool send) {
        const uint4 *mp = reinterpret_cast<const uint4 *>(msg_in + sc * 4 * Dp + dbase);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool hq = lane_data && has[q];
            const uint4 *src = mp + (hq ? q * Dp / 8 : 0);
            in[q][0] = hq ? load_u4<RW>(src) : make_uint4(0u, 0u, 0u, 0u);
            in[q][1] = hq ? load_u4<RW>(src + 1) : make_uint4(0u, 0u, 0u, 0u);
            const int64_t qs = (send && has[q]) ? slot_of(nbx[q], nby[q], lv.Wh) : 0;
            qsv[q] = (unsigned)qs;
            dst[q] = reinterpret_cast<uint4 *>(msg_out + (qs * 4 + opp[q]) * Dp + dbase);
            const bool oq = skip && send && has[q] && lane_data;
            old[q][0] = oq ? dst[q][0] : make_uint4(0u, 0u, 0u, 0u);
            old[q][1] = oq ? dst[q][1] : make_uint4(0u, 0u, 0u, 0u);
        }
    };
    if constexpr (EAGER) {
        load_cost();
        load_messages(valid);
    }
    const bool active = valid && (LISTED || !skip || dirty_in[s] == 1u);
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) return;
    trace.add(act, Gp);
    if constexpr (!EAGER) {
        load_cost();
        load_messages(active);
    }
    // belief, costs normalised by their minimum over the pixel's labels
    float cmin = INFINITY;
#pragma unroll
    for (int k = 0; k < VEC; ++k)
        if (!PADDED || dbase + k < D) cmin = fminf(cmin, lane_data ? c[k] : INFINITY);
    for (int o = 1; o < Gp; o <<= 1) cmin = fminf(cmin, __shfl_xor_sync(FULL, cmin, o, Gp));
    __half2 b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool lo_pad = !lane_data || (PADDED && dbase + 2 * j >= D);
        const bool hi_pad = !lane_data || (PADDED && dbase + 2 * j + 1 >= D);
        b[j] = __floats2half2_rn(lo_pad ? INFINITY : c[2 * j] - cmin, hi_pad ? INFINITY : c[2 * j + 1] - cmin);
#pragma unroll
        for (int q = 0; q < 4; ++q) b[j] = __hadd2(b[j], u2h(word(in[q], j)));
    }
    if (lv.disp) {
        // the read-out of a recomputed pixel of the finest scale: the belief in FP32 from the cost
        // and the existing incoming messages in the order the standalone read-out adds them (the
        // same label, the lowest on ties)
        float best = __int_as_float(0x7f800000);
        int arg = 0x7fffffff;
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            float f = c[k];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (!has[q]) continue;
                const __half2 hv = u2h(word(in[q], k >> 1));
                f += (k & 1) ? __high2float(hv) : __low2float(hv);
            }
            const int lab = dbase + k;
            if (lane_data && lab < D && f < best) {
                best = f;
                arg = lab;
            }
        }
        for (int o = Gp >> 1; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(FULL, best, o, Gp);
            const int oa = __shfl_xor_sync(FULL, arg, o, Gp);
            if (ob < best || (ob == best && oa < arg)) {
                best = ob;
                arg = oa;
            }
        }
        if (active && g == 0) lv.disp[(int64_t)y * lv.W + x] = arg;
    }
    const __half2 L2 = __float2half2_rn(lam), LT2 = __float2half2_rn(lamT);
    const int gshift = lane & ~(Gp - 1);
    unsigned mark[4] = {0u, 0u, 0u, 0u};  // slot + 1 of each neighbour to mark (APPEND)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        __half2 h[8], m[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = __hsub2(b[j], u2h(word(in[q], j)));
        __half2 mm = __hmin2(h[0], h[1]);
#pragma unroll
        for (int j = 2; j < 8; ++j) mm = __hmin2(mm, h[j]);
        float hm = fminf(__low2float(mm), __high2float(mm));
        for (int o = 1; o < Gp; o <<= 1) hm = fminf(hm, __shfl_xor_sync(FULL, hm, o, Gp));
        const __half2 HM2 = __float2half2_rn(hm);  // exact: hm is a half value
        const __half2 CAP2 = __hadd2(HM2, LT2);
        if constexpr (TS == 1) {
#pragma unroll
            for (int j = 0; j < 8; ++j) m[j] = __hsub2(__hmin2(h[j], CAP2), HM2);
        } else {
            // labels dbase - 1 (the previous lane's 15) and dbase + 16 (the next lane's 0)
            uint32_t left = __shfl_up_sync(FULL, h2u(h[7]), 1, Gp);   // its high half
            uint32_t right = __shfl_down_sync(FULL, h2u(h[0]), 1, Gp); // its low half
            const uint32_t INF_H = 0x7c00u;
            const uint32_t lft0 = __byte_perm(g == 0 ? (INF_H << 16) : left, h2u(h[0]), 0x5432);
            const uint32_t rgt7 = __byte_perm(h2u(h[7]), g == Gp - 1 ? INF_H : right, 0x5432);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                // labels (2j-1, 2j) and (2j+1, 2j+2): halves of neighbouring registers
                const __half2 lft = u2h(j > 0 ? __byte_perm(h2u(h[j - 1]), h2u(h[j]), 0x5432) : lft0);
                const __half2 rgt = u2h(j < 7 ? __byte_perm(h2u(h[j]), h2u(h[j + 1]), 0x5432) : rgt7);
                m[j] = __hsub2(__hmin2(__hmin2(h[j], __hadd2(lft, L2)), __hmin2(__hadd2(rgt, L2), CAP2)), HM2);
            }
        }
        uint32_t w[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            w[j] = h2u(m[j]);
            if constexpr (PADDED) {  // the label padding always holds 0
                if (dbase + 2 * j >= D) w[j] &= 0xffff0000u;
                if (dbase + 2 * j + 1 >= D) w[j] &= 0x0000ffffu;
            }
        }
        const uint4 o0 = make_uint4(w[0], w[1], w[2], w[3]), o1 = make_uint4(w[4], w[5], w[6], w[7]);
        const bool send = active && has[q];
        const bool mine = send && lane_data;
        if (skip) {
            const bool diff = mine && ((old[q][0].x ^ o0.x) | (old[q][0].y ^ o0.y) | (old[q][0].z ^ o0.z) |
                                       (old[q][0].w ^ o0.w) | (old[q][1].x ^ o1.x) | (old[q][1].y ^ o1.y) |
                                       (old[q][1].z ^ o1.z) | (old[q][1].w ^ o1.w)) != 0u;
            const unsigned dm = __ballot_sync(FULL, diff);
            const bool changed = ((dm >> gshift) & group_bits(Gp)) != 0u;
            st_v4_if(dst[q], o0, mine && changed);
            st_v4_if(dst[q] + 1, o1, mine && changed);
            const bool lead = send && changed && g == 0;
            if constexpr (APPEND) mark[q] = lead ? qsv[q] + 1u : 0u;
            else st_u32_if(dirty_out + qsv[q], 1u, lead);
        } else {
            st_v4_if(dst[q], o0, mine);
            st_v4_if(dst[q] + 1, o1, mine);
        }
    }
    if constexpr (APPEND) {
        // the marked neighbours' flags flip together, then the warp appends the ones that were
        // clean with a single reservation
        unsigned was[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) was[q] = mark[q] ? atomicOr(dirty_out + (mark[q] - 1u), 1u) : 1u;
        unsigned am[4];
        unsigned total = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            am[q] = __ballot_sync(FULL, was[q] == 0u);
            total += __popc(am[q]);
        }
        if (total) {
            const unsigned below = (1u << lane) - 1u;
            if (trace.abuf) {  // gathered in the warp's buffer (see Tally)
                if (trace.an + total > LIST_BUF_CAP) trace.flush_appends(al.out, al.n_out, (unsigned)nslot, lv.err);
                unsigned base = trace.an;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (was[q] == 0u) trace.abuf[base + __popc(am[q] & below)] = mark[q] - 1u;
                    base += __popc(am[q]);
                }
                trace.an += total;
                __syncwarp();
            } else {
                unsigned base = 0u;
                if (lane == 0) base = atomicAdd(al.n_out, total);
                base = __shfl_sync(FULL, base, 0);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    if (was[q] == 0u) al.out[base + __popc(am[q] & below)] = mark[q] - 1u;
                    base += __popc(am[q]);
                }
            }
        }
    }
    if (skip && active && g == 0) dirty_in[s] = 0u;
}

}  // namespace bps
