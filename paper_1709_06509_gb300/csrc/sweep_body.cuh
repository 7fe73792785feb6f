// sweep_body.cuh -- the per-pixel work of the BP kernels, shared by the one-launch-per-
// half-sweep kernels (bp.cu) and the persistent batched kernel (persist.cu).
//
// sweep_group / sweep_group_u8: one red-black half-sweep for the pixels of block `block`
// of the active colour (256 / Gp pixels, Gp lanes each, 16 labels per lane).  A group
// forms the belief b = cost + sum of the existing incoming messages, and for each existing
// neighbour q the message
//     m(d) = min(F(d), B(d), min h + lambda*trunc) - min h,   h = b - (message from q),
// where F / B are the forward / backward passes of the distance transform for the linear
// cost lambda*|d - d'| (F(d) = min(h(d), F(d-1) + lambda), B mirrored).  Within a lane the
// passes run over its 16 labels; across the lanes of the group they are completed by a
// Kogge-Stone scan of the segment ends (warp shuffles), and min h by a butterfly.  The
// result is written straight into q's incoming slot (the other colour's arrays, so the
// update is race-free in place).
//
// Fast-converging skip, exact form: dirty[c][s] = 1 while some incoming message of the
// pixel changed since its last update.  A clean pixel would resend exactly what it sent
// last time, so the group skips it; a warp whose pixels are all clean returns at once.
// With the skip on, a sender compares each new message with the stored one and writes
// (and marks the receiver dirty) only on a change.
#pragma once

#include "bps_internal.cuh"

namespace bps {

constexpr unsigned FULL = 0xffffffffu;

__device__ inline unsigned group_bits(int Gp) { return Gp >= 32 ? FULL : ((1u << Gp) - 1u); }
__device__ inline unsigned leader_bits(int Gp) {
    unsigned m = 0;
    for (int l = 0; l < 32; l += Gp) m |= 1u << l;
    return m;
}

// The recomputed-pixel count of a launch (the skip trace): a warp counts its pixels in a register
// over all the blocks it computes and adds them to the counter once, when the launch ends (flush).
// The counter is one address for the whole grid, and atomics on one address serialise in L2: one
// a warp and block cost as much time as a dense half-sweep of the finest scale itself.
//
// The same holds for the active lists' length counter: a warp that appends newly dirty pixels
// can gather them in a buffer of its own in shared memory (abuf, LIST_BUF_CAP entries) and
// reserve room in the list once per LIST_BUF_CAP entries instead of once per pixel block
// (flush_appends; the launch's kernel calls it before it ends).  Without a buffer (abuf null:
// kernels that read a list they append to in the same launch) the warp reserves at once.  The
// order of the entries in a list is free: it only decides which pixel a later launch takes
// first, never a message.
constexpr unsigned LIST_BUF_CAP = 256;  // >= 4 appends a pixel x 32 pixels of a warp (Gp = 1)
// The append buffers of a 256-thread CTA's eight warps (a static shared array of the kernel).
#define BPS_LIST_BUFFER(name) __shared__ unsigned name[256 / 32][::bps::LIST_BUF_CAP]
//
// A list launch may also defer the append decision of a pixel block (`defer`): the flags of its
// marked neighbours are flipped with atomics whose results are consumed only once the next block's
// loads are in flight (settle), so the two round trips to memory overlap.
struct Tally {
    unsigned long long *ptr;  // the launch's counter (nullable: no trace)
    unsigned n;               // this warp's pixels so far (the same in every lane)
    unsigned *abuf;           // this warp's append buffer in shared memory (nullable: none)
    unsigned an;              // entries in it (the same in every lane)
    bool defer;               // settle a block's appends during the next block (the same in every lane)
    bool pend;                // appends of a block await settling (the same in every lane)
    unsigned pwas[4], pqs[4]; // per neighbour: the flag before the atomic (1: not marked) and the slot
    __device__ explicit Tally(unsigned long long *p, unsigned *append_buf = nullptr, bool defer_appends = false)
        : ptr(p), n(0u), abuf(append_buf), an(0u), defer(defer_appends), pend(false) {}
    __device__ __forceinline__ void add(unsigned act, int lanes_a_pixel) { n += __popc(act & leader_bits(lanes_a_pixel)); }
    __device__ __forceinline__ void flush() {
        if (ptr && n && (threadIdx.x & 31) == 0) atomicAdd(ptr, (unsigned long long)n);
        n = 0u;
    }
    // Move the buffered entries into the list `out` (length counter n_out, capacity cap): one
    // reservation, then coalesced stores.  Called by every lane of the warp together.
    __device__ __forceinline__ void flush_appends(unsigned *out, unsigned *n_out, unsigned cap, unsigned *err) {
        if (!abuf || an == 0u) return;
        __syncwarp();
        const unsigned lane = threadIdx.x & 31u;
        unsigned base = 0u;
        if (lane == 0u) base = atomicAdd(n_out, an);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (unsigned i = lane; i < an; i += 32u)
            if (BPS_CHECK(base + i < cap, err, 3u)) out[base + i] = abuf[i];
        an = 0u;
        __syncwarp();
    }
    // Append the neighbours whose flag this lane's atomics flipped from 0 (pwas, pqs): the warp's
    // ballots, then one reservation (or the warp's buffer).  Called by every lane of the warp together.
    __device__ __forceinline__ void settle(unsigned *out, unsigned *n_out, unsigned cap, unsigned *err) {
        if (!pend) return;
        pend = false;
        const unsigned lane = threadIdx.x & 31u;
        unsigned am[4];
        unsigned total = 0u;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            am[q] = __ballot_sync(0xffffffffu, pwas[q] == 0u);
            total += (unsigned)__popc(am[q]);
        }
        if (!total) return;
        const unsigned below = (1u << lane) - 1u;
        if (abuf) {
            if (an + total > LIST_BUF_CAP) flush_appends(out, n_out, cap, err);
            unsigned base = an;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (pwas[q] == 0u) abuf[base + __popc(am[q] & below)] = pqs[q];
                base += (unsigned)__popc(am[q]);
            }
            an += total;
            __syncwarp();
        } else {
            unsigned base = 0u;
            if (lane == 0u) base = atomicAdd(n_out, total);
            base = __shfl_sync(0xffffffffu, base, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const unsigned at = base + (unsigned)__popc(am[q] & below);
                if (pwas[q] == 0u && BPS_CHECK(at < cap, err, 3u)) out[at] = pqs[q];
                base += (unsigned)__popc(am[q]);
            }
        }
    }
    // Append the entries that lanes with `pred` hold in `v` (the ballot of pred is `am`, taken by
    // the caller), at positions `base` + (the rank of the lane among them).  Buffered when the warp
    // has a buffer, else reserved at once.
    __device__ __forceinline__ void append(unsigned am, bool pred, unsigned v, unsigned *out, unsigned *n_out,
                                           unsigned cap, unsigned *err) {
        if (am == 0u) return;
        const unsigned lane = threadIdx.x & 31u;
        const unsigned cnt = (unsigned)__popc(am);
        const unsigned rank = (unsigned)__popc(am & ((1u << lane) - 1u));
        if (abuf) {
            if (an + cnt > LIST_BUF_CAP) flush_appends(out, n_out, cap, err);
            if (pred) abuf[an + rank] = v;
            an += cnt;
            __syncwarp();
        } else {
            unsigned base = 0u;
            if (lane == 0u) base = atomicAdd(n_out, cnt);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (pred && BPS_CHECK(base + rank < cap, err, 3u)) out[base + rank] = v;
        }
    }
};

template <typename Acc>
__device__ inline void min_convolve(const Acc (&h)[VEC], Acc lam, Acc lamT, int g, int Gp, Acc (&m)[VEC]) {
    using A = Arith<Acc>;
    Acc F[VEC], B[VEC];
    F[0] = h[0];
#pragma unroll
    for (int k = 1; k < VEC; ++k) F[k] = A::mn(h[k], F[k - 1] + lam);
    B[VEC - 1] = h[VEC - 1];
#pragma unroll
    for (int k = VEC - 2; k >= 0; --k) B[k] = A::mn(h[k], B[k + 1] + lam);
    Acc hm = h[0];
#pragma unroll
    for (int k = 1; k < VEC; ++k) hm = A::mn(hm, h[k]);
    if (Gp > 1) {
        const Acc span = lam * (Acc)VEC;
        Acc fe = F[VEC - 1], bs = B[0];
        for (int o = 1; o < Gp; o <<= 1) {
            const Acc tf = __shfl_up_sync(FULL, fe, o, Gp);
            const Acc tb = __shfl_down_sync(FULL, bs, o, Gp);
            const Acc th = __shfl_xor_sync(FULL, hm, o, Gp);
            if (g >= o) fe = A::mn(fe, tf + span * (Acc)o);
            if (g + o < Gp) bs = A::mn(bs, tb + span * (Acc)o);
            hm = A::mn(hm, th);
        }
        Acc cf = __shfl_up_sync(FULL, fe, 1, Gp);
        Acc cb = __shfl_down_sync(FULL, bs, 1, Gp);
        if (g == 0) cf = A::big();
        if (g == Gp - 1) cb = A::big();
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            F[k] = A::mn(F[k], cf + lam * (Acc)(k + 1));
            B[k] = A::mn(B[k], cb + lam * (Acc)(VEC - k));
        }
    }
    const Acc cap = hm + lamT;
#pragma unroll
    for (int k = 0; k < VEC; ++k) m[k] = A::mn(A::mn(F[k], B[k]), cap) - hm;
}

template <typename CostT, typename MsgT, bool RW = false>
__device__ __forceinline__ void sweep_group(const LevelView &lv, int colour, int D, int Dp, int Gp,
                                            typename AccOf<MsgT>::type lam, typename AccOf<MsgT>::type lamT,
                                            int skip, Tally &trace, int64_t block) {
    using Acc = typename AccOf<MsgT>::type;
    using A = Arith<Acc>;
    const int lane = threadIdx.x & 31;
    const int g = threadIdx.x & (Gp - 1);
    const int64_t s = block * (blockDim.x / Gp) + threadIdx.x / Gp;
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    int x = 0, y = 0;
    bool valid = false;
    if (s < nslot) {
        const unsigned su = (unsigned)s, wh = (unsigned)lv.Wh;  // slots stay below 2^31: 32-bit division
        y = (int)(su / wh);
        x = 2 * (int)(su - (unsigned)y * wh) + ((y + colour) & 1);
        valid = x < lv.W;
    }
    const bool active = valid && (!skip || (colour ? lv.dirty[1] : lv.dirty[0])[s] != 0u);
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) return;
    trace.add(act, Gp);
    const int64_t sc = valid ? s : 0;
    const int dbase = g * VEC;
    const bool lane_data = dbase < Dp;
    const bool has[4] = {valid && y > 0, valid && y < lv.H - 1, valid && x > 0, valid && x < lv.W - 1};

    Acc b[VEC], in[4][VEC];
    if (lane_data) {
        load16(reinterpret_cast<const CostT *>(colour ? lv.cost[1] : lv.cost[0]) + sc * Dp + dbase, b);
        const MsgT *mp = reinterpret_cast<const MsgT *>(colour ? lv.msg[1] : lv.msg[0]) + sc * 4 * Dp + dbase;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (has[q]) {
                load16_msg<RW>(mp + q * Dp, in[q]);
            } else {
#pragma unroll
                for (int k = 0; k < VEC; ++k) in[q][k] = Acc(0);
            }
        }
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            b[k] = A::big();
            in[0][k] = in[1][k] = in[2][k] = in[3][k] = Acc(0);
        }
    }
#pragma unroll
    for (int k = 0; k < VEC; ++k) b[k] = b[k] + in[0][k] + in[1][k] + in[2][k] + in[3][k];

    const int nbx[4] = {x, x, x - 1, x + 1};
    const int nby[4] = {y - 1, y + 1, y, y};
    const int opp[4] = {DIR_DOWN, DIR_UP, DIR_RIGHT, DIR_LEFT};
    MsgT *out = reinterpret_cast<MsgT *>(colour ? lv.msg[0] : lv.msg[1]);
    const int gshift = lane & ~(Gp - 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        Acc h[VEC], m[VEC];
#pragma unroll
        for (int k = 0; k < VEC; ++k) h[k] = (dbase + k < D) ? b[k] - in[q][k] : A::big();
        min_convolve(h, lam, lamT, g, Gp, m);
#pragma unroll
        for (int k = 0; k < VEC; ++k)
            if (dbase + k >= D) m[k] = Acc(0);  // the label padding always holds 0
        const bool send = active && has[q];
        const int64_t qs = send ? slot_of(nbx[q], nby[q], lv.Wh) : 0;
        MsgT *dst = out + (qs * 4 + opp[q]) * Dp + dbase;
        if (skip) {
            bool diff = false;
            if (send && lane_data) {
                Acc old[VEC];
                load16_rw(dst, old);
#pragma unroll
                for (int k = 0; k < VEC; ++k) diff |= (old[k] != stored_value<MsgT>(m[k]));
            }
            const unsigned dm = __ballot_sync(FULL, diff);
            const bool changed = ((dm >> gshift) & group_bits(Gp)) != 0u;
            if (send && changed) {
                if (lane_data) store16(dst, m);
                if (g == 0) (colour ? lv.dirty[0] : lv.dirty[1])[qs] = 1u;
            }
        } else if (send && lane_data) {
            store16(dst, m);
        }
    }
    if (skip && active && g == 0) (colour ? lv.dirty[1] : lv.dirty[0])[s] = 0u;
}

// ------------------------------------------------------------------ u8 form, packed 16-bit arithmetic
// int16 costs and uint8 messages in the interleaved label order (see label_pos): register j
// of a lane holds labels (j, j + 8) of its 16 as two unsigned 16-bit halves.  Every value
// the update forms is a non-negative integer below 2^15 (beliefs <= 27000 + 4*255 by the
// host checks, padding labels are BIG16), so 32-bit adds and subtracts never carry between
// halves and the fused add-min / 3-way min on u16x2 are exact.  The two halves run the
// distance-transform chains of labels 0..7 and 8..15 side by side; a fix-up then carries
// the low chain's end into the high chain (forward) and back (backward), together with
// the carries from the neighbouring lanes.
constexpr uint32_t BIG16 = 0x7000u;

__device__ inline uint32_t pk(uint32_t lo, uint32_t hi) { return lo | (hi << 16); }

__device__ inline void unpack_msg(const uint4 r, uint32_t (&v)[8]) {
    v[0] = __byte_perm(r.x, 0u, 0x4140); v[1] = __byte_perm(r.x, 0u, 0x4342);
    v[2] = __byte_perm(r.y, 0u, 0x4140); v[3] = __byte_perm(r.y, 0u, 0x4342);
    v[4] = __byte_perm(r.z, 0u, 0x4140); v[5] = __byte_perm(r.z, 0u, 0x4342);
    v[6] = __byte_perm(r.w, 0u, 0x4140); v[7] = __byte_perm(r.w, 0u, 0x4342);
}

__device__ inline uint4 pack_msg(const uint32_t (&v)[8]) {
    return make_uint4(__byte_perm(v[0], v[1], 0x6420), __byte_perm(v[2], v[3], 0x6420),
                      __byte_perm(v[4], v[5], 0x6420), __byte_perm(v[6], v[7], 0x6420));
}

// The outgoing message of one direction from h = b - (message from that direction), for the
// Gp lanes (segment of Gp lanes, 16 labels each in the u8 storage order) of one pixel: the
// minimisation form TS (see sweep_group_u8), min h subtracted, padded labels zeroed.
template <bool PADDED, int TS>
__device__ __forceinline__ void u8_message(const uint32_t (&h)[8], int lam, int lamT, int g, int Gp, int D, int dbase,
                                           uint32_t (&m)[8]) {
    const uint32_t LAM2 = pk((uint32_t)lam, (uint32_t)lam);
    uint32_t mm = __vimin3_u16x2(h[0], h[1], h[2]);
    mm = __vimin3_u16x2(mm, h[3], h[4]);
    mm = __vimin3_u16x2(mm, h[5], h[6]);
    mm = __vimin3_u16x2(mm, h[7], h[7]);
    int hm = (int)min(mm & 0xffffu, mm >> 16);
    if constexpr (TS != 0) {
        for (int o = 1; o < Gp; o <<= 1) hm = min(hm, __shfl_xor_sync(FULL, hm, o, Gp));
        const uint32_t CAP2 = (uint32_t)(hm + lamT) * 0x10001u;
        const uint32_t HM2 = (uint32_t)hm * 0x10001u;
        if constexpr (TS == 1) {
#pragma unroll
            for (int j = 0; j < 8; ++j) m[j] = __vimin3_u16x2(h[j], CAP2, CAP2) - HM2;
        } else {
            // labels dbase - 1 (the previous lane's label 15) and dbase + 16 (the next lane's 0)
            int left = __shfl_up_sync(FULL, (int)(h[7] >> 16), 1, Gp);
            int right = __shfl_down_sync(FULL, (int)(h[0] & 0xffffu), 1, Gp);
            if (g == 0) left = (int)BIG16;
            if (g == Gp - 1) right = (int)BIG16;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                // register j holds labels (j, j+8): its neighbours sit in registers j-1 and j+1,
                // except across the lane edge and across the middle (labels 7 | 8)
                const uint32_t lft = j > 0 ? h[j - 1] : pk((uint32_t)left, h[7] & 0xffffu);
                const uint32_t rgt = j < 7 ? h[j + 1] : pk(h[0] >> 16, (uint32_t)right);
                // rgt + LAM2 cannot carry between the halves (both stay below 2^15 + 255)
                m[j] = __vimin3_u16x2(__viaddmin_u16x2(lft, LAM2, h[j]), rgt + LAM2, CAP2) - HM2;
            }
        }
    } else {
    uint32_t F[8], B[8];
    F[0] = h[0];
#pragma unroll
    for (int j = 1; j < 8; ++j) F[j] = __viaddmin_u16x2(F[j - 1], LAM2, h[j]);
    B[7] = h[7];
#pragma unroll
    for (int j = 6; j >= 0; --j) B[j] = __viaddmin_u16x2(B[j + 1], LAM2, h[j]);
    const int fl = (int)(F[7] & 0xffffu), fh = (int)(F[7] >> 16);  // local forward at labels 7, 15
    const int bl = (int)(B[0] & 0xffffu), bh = (int)(B[0] >> 16);  // local backward at labels 0, 8
    int cf = (int)BIG16, cb = (int)BIG16;
    if (Gp > 1) {
        int fe = min(fh, fl + 8 * lam);  // forward value at this lane's last label
        int bs = min(bl, bh + 8 * lam);  // backward value at this lane's first label
        for (int o = 1; o < Gp; o <<= 1) {
            const int tf = __shfl_up_sync(FULL, fe, o, Gp);
            const int tb = __shfl_down_sync(FULL, bs, o, Gp);
            const int th = __shfl_xor_sync(FULL, hm, o, Gp);
            if (g >= o) fe = min(fe, tf + 16 * lam * o);
            if (g + o < Gp) bs = min(bs, tb + 16 * lam * o);
            hm = min(hm, th);
        }
        cf = __shfl_up_sync(FULL, fe, 1, Gp);
        cb = __shfl_down_sync(FULL, bs, 1, Gp);
        if (g == 0) cf = (int)BIG16;
        if (g == Gp - 1) cb = (int)BIG16;
        cf = min(cf, (int)BIG16);
        cb = min(cb, (int)BIG16);
    }
    // forward: label j gets cf + lam*(j+1); label 8+j gets F(7) + lam*(j+1)
    const int f7 = min(min(fl, cf + 8 * lam), (int)BIG16);
    const uint32_t xF = pk((uint32_t)cf, (uint32_t)f7);
    // backward: label 8+j gets cb + lam*(8-j); label j gets B(8) + lam*(8-j)
    const int b8 = min(min(bh, cb + 8 * lam), (int)BIG16);
    const uint32_t xB = pk((uint32_t)b8, (uint32_t)cb);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        F[j] = __viaddmin_u16x2(xF, (uint32_t)(lam * (j + 1)) * 0x10001u, F[j]);
        B[j] = __viaddmin_u16x2(xB, (uint32_t)(lam * (8 - j)) * 0x10001u, B[j]);
    }
    const uint32_t CAP2 = (uint32_t)(hm + lamT) * 0x10001u;
    const uint32_t HM2 = (uint32_t)hm * 0x10001u;
#pragma unroll
    for (int j = 0; j < 8; ++j) m[j] = __vimin3_u16x2(F[j], B[j], CAP2) - HM2;
    }
    if constexpr (PADDED) {
#pragma unroll
        for (int j = 0; j < 8; ++j)
            m[j] &= (dbase + j < D ? 0xffffu : 0u) | (dbase + 8 + j < D ? 0xffff0000u : 0u);
    }
}

// The label of least belief of one pixel from its packed u8-form belief b (register j: labels
// dbase + j and dbase + 8 + j as 16-bit halves; padding labels hold BIG16, above every real belief),
// the lowest label on ties: the minimum over the group of (belief << 10 | label).  Every lane of
// the warp takes part (the butterfly spans the Gp lanes of each pixel).
__device__ __forceinline__ int u8_argmin(const uint32_t (&b)[8], int dbase, int Gp) {
    unsigned key = 0xffffffffu;
#pragma unroll
    for (int j = 0; j < 8; ++j) key = min(key, ((b[j] & 0xffffu) << 10) | (unsigned)(dbase + j));
#pragma unroll
    for (int j = 0; j < 8; ++j) key = min(key, ((b[j] >> 16) << 10) | (unsigned)(dbase + 8 + j));
    for (int o = 1; o < Gp; o <<= 1) key = min(key, __shfl_xor_sync(FULL, key, o, Gp));
    return (int)(key & 1023u);
}

// Stores under a predicate, without a branch around them.
__device__ __forceinline__ void st_v4_if(uint4 *p, const uint4 &v, bool pred) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %5, 0;\n\t@p st.global.v4.u32 [%0], {%1, %2, %3, %4};\n\t}" ::"l"(p),
                 "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w), "r"((unsigned)pred)
                 : "memory");
}
__device__ __forceinline__ void st_u32_if(unsigned *p, unsigned v, bool pred) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %2, 0;\n\t@p st.global.u32 [%0], %1;\n\t}" ::"l"(p), "r"(v),
                 "r"((unsigned)pred)
                 : "memory");
}

// Active lists (fast-converging skip).  After the first two half-sweeps of a scale, a
// half-sweep processes only the pixels listed for it, packed densely: a sender that flips a
// neighbour's skip flag from 0 to 1 appends the neighbour to the other colour's list (one
// atomic per warp and direction).  A pixel enters a list only on that 0 -> 1 flip and leaves
// the flag at 0 when it is processed, so no list holds a pixel twice.
struct ActiveList {
    const unsigned *in;   // slots to process (nullable: every slot of the colour)
    const unsigned *n_in; // number of entries of `in`
    unsigned *out;        // where newly dirty pixels of the other colour go (nullable: no list)
    unsigned *n_out;
};

// ------------------------------------------------------------------ staged inputs (cp.async)
// A staged sweep keeps every input of a pixel block in a per-thread shared-memory stage, filled
// by asynchronous 16-byte copies one block ahead, so the loads of the next block are in flight
// while the current one computes and memory parallelism does not cost registers.  Stage chunk k
// of thread t is stage[k * blockDim.x + t]: 0-1 cost, 2-5 incoming, 6-9 old outgoing, 10 flag.
// Chunks of absent inputs are zero-filled by the copy (source size 0, an in-bounds address).
constexpr int STAGE_CHUNKS = 11;
constexpr int BULK_CONSUMERS = 256;  // computing threads of a bulk-copy sweep CTA (one more warp copies)

__device__ __forceinline__ void cp_async16(uint4 *smem, const void *gmem, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(pred ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async4(uint4 *smem, const void *gmem, bool pred) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(pred ? 4 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// every committed group but the newest `n` has landed in shared memory
template <int n> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(n) : "memory");
}

// The start message of receiver (x, y) from direction `dir` in a scale's first iteration: its
// parent's incoming message from that direction (the fused coarse-to-fine start).  `use`
// false gives an in-bounds address that is not read.
__device__ __forceinline__ const uint8_t *start_slot_u8(const LevelView &lv, int x, int y, int dir, int Dp, int dbase,
                                                        bool use) {
    if (!use) return reinterpret_cast<const uint8_t *>(lv.pmsg[0]);
    const int px = x >> 1, py = y >> 1;
    return reinterpret_cast<const uint8_t *>(colour_of(px, py) ? lv.pmsg[1] : lv.pmsg[0]) +
           (slot_of(px, py, lv.pWh) * 4 + dir) * Dp + dbase;
}

// Issue the copies of block `block`'s inputs (eager: old messages of every valid pixel) into
// `stage` (this thread's chunks).  LISTED: the slot is the caller's list entry s_listed (nslot
// for none), and no flag is copied (a listed pixel is dirty by construction).
template <bool LISTED = false>
__device__ __forceinline__ void stage_u8(const LevelView &lv, int colour, int Dp, int Gp, int skip, int64_t block,
                                         uint4 *stage, int64_t s_listed = 0) {
    const int T = blockDim.x, t = threadIdx.x;
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
    const int16_t *cost = reinterpret_cast<const int16_t *>(colour ? lv.cost[1] : lv.cost[0]);
    const uint8_t *msg_in = reinterpret_cast<const uint8_t *>(colour ? lv.msg[1] : lv.msg[0]);
    const uint8_t *msg_out = reinterpret_cast<const uint8_t *>(colour ? lv.msg[0] : lv.msg[1]);
    const unsigned *dirty_in = colour ? lv.dirty[1] : lv.dirty[0];
    const int nbx[4] = {x, x, x - 1, x + 1};
    const int nby[4] = {y - 1, y + 1, y, y};
    const int opp[4] = {DIR_DOWN, DIR_UP, DIR_RIGHT, DIR_LEFT};
    const uint4 *cp = reinterpret_cast<const uint4 *>(cost + (lane_data ? sc * Dp + dbase : 0));
    cp_async16(stage + 0 * T + t, cp, lane_data);
    cp_async16(stage + 1 * T + t, cp + (lane_data ? 1 : 0), lane_data);
    const uint8_t *mp = msg_in + (lane_data ? sc * 4 * Dp + dbase : 0);
    if (lv.start == 1) {  // a scale's first half-sweep: the parent's record holds the start messages
        const int px = x >> 1, py = y >> 1;
        mp = reinterpret_cast<const uint8_t *>(colour_of(px, py) ? lv.pmsg[1] : lv.pmsg[0]) +
             (lane_data ? slot_of(px, py, lv.pWh) * 4 * Dp + dbase : 0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const bool hq = lane_data && has[q];
        cp_async16(stage + (2 + q) * T + t, mp + (hq ? q * Dp : 0), hq);
        // the change test's old message: none in a scale's first half-sweep (start 1), the
        // receiver's start message in its parent's record in the second (start 2)
        const bool oq = skip && hq && lv.start != 1;
        const uint8_t *op = lv.start == 2 ? start_slot_u8(lv, nbx[q], nby[q], opp[q], Dp, dbase, oq)
                                          : msg_out + (oq ? (slot_of(nbx[q], nby[q], lv.Wh) * 4 + opp[q]) * Dp + dbase : 0);
        cp_async16(stage + (6 + q) * T + t, op, oq);
    }
    if constexpr (!LISTED) cp_async4(stage + 10 * T + t, dirty_in + sc, valid);
}

// PADDED: D is not a multiple of 16, so the last lane holds labels >= D that must stay out
// of every minimum and be stored as 0.
// APPEND: newly dirty neighbours are appended to the other colour's active list.
// TS: how the truncated-linear minimisation is formed.
//   TS = 0, any trunc: the forward/backward distance transform described above.
//   TS = 1, trunc <= 1: m(d) = min(h(d), min h + lambda*trunc) - min h.
//   TS = 2, trunc == 2: m(d) = min(h(d), h(d-1) + lambda, h(d+1) + lambda, min h + 2 lambda) - min h,
//           the same function (a label two or more away costs the cap at least), needing only
//           each label's immediate neighbours: no chains, no scan across the lanes.
// EAGER: 0, the dirty flag is read first and only pixels that need it load their inputs;
//        1, every load of the half-sweep (cost, messages in, old messages out, flag) is issued at
//           once, so a pixel waits for one round trip to memory instead of two (clean pixels load
//           for nothing: for small, latency-bound scales);
//        2, as 1, and the cost loads also precede the wait on the predecessor kernel (no BP
//           kernel writes the cost volume); the caller then must not have called pdl_enter().
//        3, the inputs were staged by the caller (stage_u8, waited for): read from `stage`;
//        4, the inputs landed in a bulk-copy stage of the caller (sweep_u8_bulk_kernel; with LISTED).
// LISTED: the caller gives the slot (s_listed; nslot for none), an entry of the active list:
//         a listed pixel is dirty by construction (it was appended when its flag flipped from
//         0 to 1, and only its own update clears the flag), so its flag is not read.
template <bool PADDED, bool APPEND = false, int TS = 0, bool RW = false, int EAGER = 0, bool LISTED = false>
__device__ __forceinline__ void sweep_group_u8(const LevelView &lv, int colour, int D, int Dp, int Gp, int lam,
                                               int lamT, int skip, Tally &trace, int64_t block,
                                               const ActiveList &al = ActiveList{nullptr, nullptr, nullptr, nullptr},
                                               int64_t n_in = 0, int64_t s_listed = 0, const uint4 *stage = nullptr) {
    const int lane = threadIdx.x & 31;
    const int g = threadIdx.x & (Gp - 1);
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    int64_t s = block * (blockDim.x / Gp) + threadIdx.x / Gp;
    if constexpr (LISTED) s = s_listed;
    else if (al.in) s = s < n_in ? (int64_t)al.in[s] : nslot;
    int x = 0, y = 0;
    bool valid = false;
    // a list entry (or the caller's) names a slot of the scale, or nslot for none
    if (BPS_CHECK(!(LISTED || al.in) || s <= nslot, lv.err, 2u) && s < nslot) {
        const unsigned su = (unsigned)s, wh = (unsigned)lv.Wh;  // slots stay below 2^31: 32-bit division
        y = (int)(su / wh);
        x = 2 * (int)(su - (unsigned)y * wh) + ((y + colour) & 1);
        valid = x < lv.W;
    }
    const unsigned *dirty_in = colour ? lv.dirty[1] : lv.dirty[0];
    const int64_t sc = valid ? s : 0;
    const int dbase = g * VEC;
    const bool lane_data = dbase < Dp;
    const bool has[4] = {valid && y > 0, valid && y < lv.H - 1, valid && x > 0, valid && x < lv.W - 1};
    const int16_t *cost = reinterpret_cast<const int16_t *>(colour ? lv.cost[1] : lv.cost[0]);
    const uint8_t *msg_in = reinterpret_cast<const uint8_t *>(colour ? lv.msg[1] : lv.msg[0]);
    uint8_t *msg_out = reinterpret_cast<uint8_t *>(colour ? lv.msg[0] : lv.msg[1]);
    unsigned *dirty_out = colour ? lv.dirty[0] : lv.dirty[1];
    const int nbx[4] = {x, x, x - 1, x + 1};
    const int nby[4] = {y - 1, y + 1, y, y};
    const int opp[4] = {DIR_DOWN, DIR_UP, DIR_RIGHT, DIR_LEFT};

    uint32_t b[8];
    uint4 in[4];
    // the old outgoing messages (the skip's change test) are loaded together with the inputs,
    // so a recomputed pixel waits for one round trip to memory, not two
    uint4 old[4];
    unsigned qsv[4];  // the neighbours' slots (0 where there is none)
    // the slot a message to neighbour q goes to (recomputed where it is stored: fewer live registers)
    auto dst = [&](int q) {
        return reinterpret_cast<uint4 *>(msg_out + ((int64_t)qsv[q] * 4 + opp[q]) * Dp + dbase);
    };
    auto load_cost = [&]() {
        if (lane_data) {
            const uint4 *cp = reinterpret_cast<const uint4 *>(cost + sc * Dp + dbase);
            const uint4 c0 = __ldg(cp), c1 = __ldg(cp + 1);
            b[0] = c0.x; b[1] = c0.y; b[2] = c0.z; b[3] = c0.w;
            b[4] = c1.x; b[5] = c1.y; b[6] = c1.z; b[7] = c1.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = pk(BIG16, BIG16);
        }
    };
    // `send`: whether this lane's pixel sends (the active pixels; all valid ones when eager)
    auto load_messages = [&](bool send) {
        const uint8_t *mp = msg_in + sc * 4 * Dp + dbase;
        if (lv.start == 1) {  // a scale's first half-sweep: the parent's record holds the start messages
            const int px = x >> 1, py = y >> 1;
            mp = reinterpret_cast<const uint8_t *>(colour_of(px, py) ? lv.pmsg[1] : lv.pmsg[0]) +
                 slot_of(px, py, lv.pWh) * 4 * Dp + dbase;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            in[q] = (lane_data && has[q]) ? load_u4<RW>(reinterpret_cast<const uint4 *>(mp + q * Dp))
                                          : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int64_t qs = (send && has[q]) ? slot_of(nbx[q], nby[q], lv.Wh) : 0;
            qsv[q] = (unsigned)qs;
            // the change test's old message: none in a scale's first half-sweep (start 1), the
            // receiver's start message in its parent's record in the second (start 2)
            const bool oq = skip && send && has[q] && lane_data && lv.start != 1;
            old[q] = !oq ? make_uint4(0u, 0u, 0u, 0u)
                         : lv.start == 2 ? load_u4<RW>(reinterpret_cast<const uint4 *>(
                                               start_slot_u8(lv, nbx[q], nby[q], opp[q], Dp, dbase, true)))
                                         : *dst(q);
        }
    };
    unsigned flag_staged = 0u;
    if constexpr (EAGER == 3) {
        const int T = blockDim.x, t = threadIdx.x;
        const uint4 c0 = stage[0 * T + t], c1 = stage[1 * T + t];
        b[0] = c0.x; b[1] = c0.y; b[2] = c0.z; b[3] = c0.w;
        b[4] = c1.x; b[5] = c1.y; b[6] = c1.z; b[7] = c1.w;
        if (!lane_data) {
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = pk(BIG16, BIG16);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            in[q] = stage[(2 + q) * T + t];
            old[q] = stage[(6 + q) * T + t];
            const int64_t qs = (valid && has[q]) ? slot_of(nbx[q], nby[q], lv.Wh) : 0;
            qsv[q] = (unsigned)qs;
        }
        flag_staged = stage[10 * T + t].x;
    } else if constexpr (EAGER == 4) {
        // inputs landed in a bulk-copy stage (see sweep_u8_bulk_kernel): per pixel of the block its
        // cost record [P][2 Dp], its incoming record [P][4 Dp] and the four old outgoing slots
        // [P][4][Dp] (absent neighbours' chunks are not copied and are not read)
        const int pix = threadIdx.x / Gp, P = BULK_CONSUMERS / Gp;
        const uint8_t *base = reinterpret_cast<const uint8_t *>(stage);
        if (lane_data) {
            const uint4 *cp = reinterpret_cast<const uint4 *>(base + (size_t)pix * 2 * Dp + 2 * dbase);
            const uint4 c0 = cp[0], c1 = cp[1];
            b[0] = c0.x; b[1] = c0.y; b[2] = c0.z; b[3] = c0.w;
            b[4] = c1.x; b[5] = c1.y; b[6] = c1.z; b[7] = c1.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = pk(BIG16, BIG16);
        }
        const uint8_t *ip = base + (size_t)P * 2 * Dp + (size_t)pix * 4 * Dp + dbase;
        const uint8_t *op = base + (size_t)P * 6 * Dp + (size_t)pix * 4 * Dp + dbase;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const bool hq = lane_data && has[q];
            in[q] = hq ? *reinterpret_cast<const uint4 *>(ip + q * Dp) : make_uint4(0u, 0u, 0u, 0u);
            old[q] = (hq && skip && lv.start != 1) ? *reinterpret_cast<const uint4 *>(op + q * Dp)
                                                   : make_uint4(0u, 0u, 0u, 0u);
            const int64_t qs = (valid && has[q]) ? slot_of(nbx[q], nby[q], lv.Wh) : 0;
            qsv[q] = (unsigned)qs;
        }
    } else if constexpr (EAGER != 0) {
        load_cost();
        if constexpr (EAGER == 2) pdl_enter();
        load_messages(valid);
    }
    // dirty and not frozen (flags are 0 / 1 under the exact skip rule)
    const bool active =
        valid && (LISTED || !skip || lv.start != 0 || (EAGER == 3 ? flag_staged : dirty_in[s]) == 1u);
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) return;
    trace.add(act, Gp);
    if constexpr (EAGER == 0) {
        load_cost();
        load_messages(active);
    }
    // the previous block's appends, now that this block's loads are in flight
    if constexpr (APPEND) trace.settle(al.out, al.n_out, (unsigned)nslot, lv.err);
    if (lv.bsum8) {
        // every incoming message is at most 63: the four add up bytewise without a carry, and the
        // sum is unpacked once
        const uint4 sum = make_uint4(in[0].x + in[1].x + in[2].x + in[3].x, in[0].y + in[1].y + in[2].y + in[3].y,
                                     in[0].z + in[1].z + in[2].z + in[3].z, in[0].w + in[1].w + in[2].w + in[3].w);
        uint32_t t[8];
        unpack_msg(sum, t);
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] += t[j];
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t t[8];
            unpack_msg(in[q], t);
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] += t[j];
        }
    }
    if constexpr (PADDED) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool plo = dbase + j >= D, phi = dbase + 8 + j >= D;
            b[j] = __vimax3_u16x2(b[j], pk(plo ? BIG16 : 0u, phi ? BIG16 : 0u), 0u);
        }
    }

    if (lv.disp) {  // the read-out of a recomputed pixel of the finest scale, from the belief just formed
        const int d = u8_argmin(b, dbase, Gp);
        if (active && g == 0) lv.disp[(int64_t)y * lv.W + x] = d;
    }
    const int gshift = lane & ~(Gp - 1);
    unsigned marks = 0u;  // bit q: this group marks neighbour q dirty (APPEND)
    const uint32_t EPS4 = (uint32_t)lv.eps * 0x01010101u;
    bool marked = false;                  // this pixel marked some receiver (skip rule freeze)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t t[8], h[8], m[8];
        unpack_msg(in[q], t);
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = b[j] - t[j];
        u8_message<PADDED, TS>(h, lam, lamT, g, Gp, D, dbase, m);
        const uint4 out = pack_msg(m);

        const bool send = active && has[q];
        const bool mine = send && lane_data;
        if (skip && lv.start == 1) {
            // a scale's first half-sweep: every receiver is recomputed next, so nothing is compared
            // or marked; the receivers' slots are written whole
            st_v4_if(dst(q), out, mine);
        } else if (skip) {
            const bool diff =
                mine && ((old[q].x ^ out.x) | (old[q].y ^ out.y) | (old[q].z ^ out.z) | (old[q].w ^ out.w)) != 0u;
            bool big = false;
            if (lv.eps)  // uniform: the exact rule (eps = 0) marks exactly the changed messages
                big = mine && (__vcmpgtu4(__vabsdiffu4(old[q].x, out.x), EPS4) |
                               __vcmpgtu4(__vabsdiffu4(old[q].y, out.y), EPS4) |
                               __vcmpgtu4(__vabsdiffu4(old[q].z, out.z), EPS4) |
                               __vcmpgtu4(__vabsdiffu4(old[q].w, out.w), EPS4)) != 0u;
            const unsigned dm = __ballot_sync(FULL, diff);
            const unsigned bm = lv.eps ? __ballot_sync(FULL, big) : dm;
            const bool changed = ((dm >> gshift) & group_bits(Gp)) != 0u;
            const bool significant = ((bm >> gshift) & group_bits(Gp)) != 0u;  // = changed when eps = 0
            // the second half-sweep of a scale writes every slot: the receivers' own records do
            // not hold their start messages (those stay in the parent's records)
            st_v4_if(dst(q), out, mine && (changed || lv.start == 2));
            const bool mk = send && significant;
            marked = marked || mk;
            const bool lead = mk && g == 0;  // one mark per pixel group
            if constexpr (APPEND) {
                marks |= (lead ? 1u : 0u) << q;
            } else if (lv.freeze) {
                if (lead) atomicOr(dirty_out + qsv[q], 1u);  // keeps the frozen bit
            } else {
                st_u32_if(dirty_out + qsv[q], 1u, lead);
            }
        } else {
            st_v4_if(dst(q), out, mine);
        }
    }
    if constexpr (APPEND) {
        // the flags of the marked neighbours flip together (one round trip); the warp appends the
        // ones that were clean with a single reservation, now or (deferred) during its next block
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            trace.pwas[q] = ((marks >> q) & 1u) ? atomicOr(dirty_out + qsv[q], 1u) : 1u;
            trace.pqs[q] = qsv[q];
        }
        trace.pend = true;
        if (!trace.defer) trace.settle(al.out, al.n_out, (unsigned)nslot, lv.err);
    }
    if (skip && active && g == 0 && !lv.keep_flag)
        (colour ? lv.dirty[1] : lv.dirty[0])[s] = (lv.freeze && !marked) ? 2u : 0u;  // frozen: bit 1
}


// sweep_group_u8_dp: the same half-sweep with one group of Gp lanes per (pixel, direction),
// 4 Gp lanes a pixel (Gp <= 8): every group forms the pixel's belief (the four incoming
// message loads of a pixel are the same addresses across its groups, served once per warp)
// and computes, compares and stores the one message of its direction.  The four messages of a
// pixel are then computed side by side instead of one after another: a quarter of the
// dependent work per lane, for scales whose time is the latency of few pixels.  Template
// parameters as for sweep_group_u8; `block` counts blockDim / (4 Gp) pixels.
template <bool PADDED, bool APPEND = false, int TS = 0, int EAGER = 0, bool LISTED = false>
__device__ __forceinline__ void sweep_group_u8_dp(const LevelView &lv, int colour, int D, int Dp, int Gp, int lam,
                                                  int lamT, int skip, Tally &trace, int64_t block,
                                                  const ActiveList &al = ActiveList{nullptr, nullptr, nullptr, nullptr},
                                                  int64_t s_listed = 0) {
    const int lane = threadIdx.x & 31;
    const int LP = 4 * Gp;
    const int g = threadIdx.x & (Gp - 1);
    const int qo = (threadIdx.x / Gp) & 3;  // this group's direction
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    int64_t s = block * (blockDim.x / LP) + threadIdx.x / LP;
    if constexpr (LISTED) s = s_listed;
    int x = 0, y = 0;
    bool valid = false;
    if (s < nslot) {
        const unsigned su = (unsigned)s, wh = (unsigned)lv.Wh;  // slots stay below 2^31: 32-bit division
        y = (int)(su / wh);
        x = 2 * (int)(su - (unsigned)y * wh) + ((y + colour) & 1);
        valid = x < lv.W;
    }
    const unsigned *dirty_in = colour ? lv.dirty[1] : lv.dirty[0];
    const int64_t sc = valid ? s : 0;
    const int dbase = g * VEC;
    const bool lane_data = dbase < Dp;
    const bool has[4] = {valid && y > 0, valid && y < lv.H - 1, valid && x > 0, valid && x < lv.W - 1};
    const bool has_o = qo == 0 ? has[0] : (qo == 1 ? has[1] : (qo == 2 ? has[2] : has[3]));
    const int nbx = qo == 2 ? x - 1 : (qo == 3 ? x + 1 : x);
    const int nby = qo == 0 ? y - 1 : (qo == 1 ? y + 1 : y);
    const int16_t *cost = reinterpret_cast<const int16_t *>(colour ? lv.cost[1] : lv.cost[0]);
    const uint8_t *msg_in = reinterpret_cast<const uint8_t *>(colour ? lv.msg[1] : lv.msg[0]);
    uint8_t *msg_out = reinterpret_cast<uint8_t *>(colour ? lv.msg[0] : lv.msg[1]);
    unsigned *dirty_out = colour ? lv.dirty[0] : lv.dirty[1];

    uint32_t b[8];
    uint4 in[4];
    uint4 *dst;
    uint4 old;
    unsigned qs_o = 0u;  // the receiver's slot
    auto load_cost = [&]() {
        if (lane_data) {
            const uint4 *cp = reinterpret_cast<const uint4 *>(cost + sc * Dp + dbase);
            const uint4 c0 = __ldg(cp), c1 = __ldg(cp + 1);
            b[0] = c0.x; b[1] = c0.y; b[2] = c0.z; b[3] = c0.w;
            b[4] = c1.x; b[5] = c1.y; b[6] = c1.z; b[7] = c1.w;
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] = pk(BIG16, BIG16);
        }
    };
    auto load_messages = [&](bool send) {
        const uint8_t *mp = msg_in + sc * 4 * Dp + dbase;
        if (lv.start == 1) {  // a scale's first half-sweep: the parent's record holds the start messages
            const int px = x >> 1, py = y >> 1;
            mp = reinterpret_cast<const uint8_t *>(colour_of(px, py) ? lv.pmsg[1] : lv.pmsg[0]) +
                 slot_of(px, py, lv.pWh) * 4 * Dp + dbase;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            in[q] = (lane_data && has[q]) ? __ldg(reinterpret_cast<const uint4 *>(mp + q * Dp))
                                          : make_uint4(0u, 0u, 0u, 0u);
        const int64_t qs = (send && has_o) ? slot_of(nbx, nby, lv.Wh) : 0;
        qs_o = (unsigned)qs;
        dst = reinterpret_cast<uint4 *>(msg_out + (qs * 4 + (qo ^ 1)) * Dp + dbase);
        // the change test's old message: none at start 1, the receiver's parent record at start 2
        const bool oq = skip && send && has_o && lane_data && lv.start != 1;
        old = !oq ? make_uint4(0u, 0u, 0u, 0u)
                  : lv.start == 2 ? __ldg(reinterpret_cast<const uint4 *>(
                                        start_slot_u8(lv, nbx, nby, qo ^ 1, Dp, dbase, true)))
                                  : *dst;
    };
    if constexpr (EAGER != 0) {
        load_cost();
        if constexpr (EAGER == 2) pdl_enter();
        load_messages(valid);
    }
    const bool active = valid && (LISTED || !skip || lv.start != 0 || dirty_in[s] == 1u);
    const unsigned act = __ballot_sync(FULL, active);
    if (act == 0) return;
    trace.add(act, LP);
    if constexpr (EAGER == 0) {
        load_cost();
        load_messages(active);
    }
    if (lv.bsum8) {
        // every incoming message is at most 63: the four add up bytewise without a carry, and the
        // sum is unpacked once
        const uint4 sum = make_uint4(in[0].x + in[1].x + in[2].x + in[3].x, in[0].y + in[1].y + in[2].y + in[3].y,
                                     in[0].z + in[1].z + in[2].z + in[3].z, in[0].w + in[1].w + in[2].w + in[3].w);
        uint32_t t[8];
        unpack_msg(sum, t);
#pragma unroll
        for (int j = 0; j < 8; ++j) b[j] += t[j];
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint32_t t[8];
            unpack_msg(in[q], t);
#pragma unroll
            for (int j = 0; j < 8; ++j) b[j] += t[j];
        }
    }
    if constexpr (PADDED) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const bool plo = dbase + j >= D, phi = dbase + 8 + j >= D;
            b[j] = __vimax3_u16x2(b[j], pk(plo ? BIG16 : 0u, phi ? BIG16 : 0u), 0u);
        }
    }
    if (lv.disp) {  // the read-out of a recomputed pixel of the finest scale (the up-direction group writes)
        const int d = u8_argmin(b, dbase, Gp);
        if (active && g == 0 && qo == 0) lv.disp[(int64_t)y * lv.W + x] = d;
    }
    const uint4 in_o = qo == 0 ? in[0] : (qo == 1 ? in[1] : (qo == 2 ? in[2] : in[3]));
    uint32_t t[8], h[8], m[8];
    unpack_msg(in_o, t);
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = b[j] - t[j];
    u8_message<PADDED, TS>(h, lam, lamT, g, Gp, D, dbase, m);
    const uint4 out = pack_msg(m);

    const bool send = active && has_o;
    unsigned mark = 0u;  // slot + 1 of the neighbour to mark dirty (APPEND)
    bool marked = false;  // this group marked its receiver (skip rule freeze)
    const bool mine = send && lane_data;
    if (skip && lv.start == 1) {  // a scale's first half-sweep: nothing compared or marked
        st_v4_if(dst, out, mine);
    } else if (skip) {
        const bool diff = mine && ((old.x ^ out.x) | (old.y ^ out.y) | (old.z ^ out.z) | (old.w ^ out.w)) != 0u;
        bool big = false;
        if (lv.eps) {
            const uint32_t EPS4 = (uint32_t)lv.eps * 0x01010101u;
            big = mine && (__vcmpgtu4(__vabsdiffu4(old.x, out.x), EPS4) | __vcmpgtu4(__vabsdiffu4(old.y, out.y), EPS4) |
                           __vcmpgtu4(__vabsdiffu4(old.z, out.z), EPS4) | __vcmpgtu4(__vabsdiffu4(old.w, out.w), EPS4)) != 0u;
        }
        const unsigned dm = __ballot_sync(FULL, diff);
        const unsigned bm = lv.eps ? __ballot_sync(FULL, big) : dm;
        const bool changed = ((dm >> (lane & ~(Gp - 1))) & group_bits(Gp)) != 0u;
        const bool significant = ((bm >> (lane & ~(Gp - 1))) & group_bits(Gp)) != 0u;
        st_v4_if(dst, out, mine && (changed || lv.start == 2));  // start 2: every slot written
        marked = send && significant;
        const bool lead = marked && g == 0;
        if constexpr (APPEND) {
            mark = lead ? qs_o + 1u : 0u;
        } else if (lv.freeze) {
            if (lead) atomicOr(dirty_out + qs_o, 1u);  // keeps the frozen bit
        } else {
            st_u32_if(dirty_out + qs_o, 1u, lead);
        }
    } else {
        st_v4_if(dst, out, mine);
    }
    if constexpr (APPEND) {
        const bool app = mark != 0u && atomicOr(dirty_out + (mark - 1u), 1u) == 0u;
        const unsigned am = __ballot_sync(FULL, app);
        trace.append(am, app, mark - 1u, al.out, al.n_out, (unsigned)nslot, lv.err);
    }
    // the pixel's four direction groups: did any mark its receiver?
    const unsigned mk = __ballot_sync(FULL, marked && g == 0);
    const unsigned pix_dirs = (1u | (1u << Gp) | (1u << (2 * Gp)) | (1u << (3 * Gp))) << (lane & ~(LP - 1));
    if (skip && active && g == 0 && qo == 0)
        (colour ? lv.dirty[1] : lv.dirty[0])[s] = (lv.freeze && (mk & pix_dirs) == 0u) ? 2u : 0u;
}

// ------------------------------------------------------------------ coarse-to-fine start
// Element k of the copy of parent records into the fine pixels of `colour` (16-byte chunks).
__device__ __forceinline__ void upsample_chunk(const LevelView &coarse, const LevelView &fine, int colour,
                                               int rec_chunks, int64_t k) {
    const int chunk = (int)(k % rec_chunks);
    const int64_t s = k / rec_chunks;
    const int y = (int)(s / fine.Wh);
    const int x = 2 * (int)(s - (int64_t)y * fine.Wh) + ((y + colour) & 1);
    if (x >= fine.W) return;
    const int px = x >> 1, py = y >> 1;
    const uint4 *src = reinterpret_cast<const uint4 *>(colour_of(px, py) ? coarse.msg[1] : coarse.msg[0]) +
                       slot_of(px, py, coarse.Wh) * rec_chunks + chunk;
    uint4 *dst = reinterpret_cast<uint4 *>(colour ? fine.msg[1] : fine.msg[0]) + s * rec_chunks + chunk;
    *dst = *src;
}

// ------------------------------------------------------------------ winner-take-all
// Pixels of block `block` in raster order, Gp lanes each: argmin of the belief, the lowest
// label on ties (labels are compared through the storage order of the form).
// The read-out of pixel (x, y) by its group of Gp lanes (when `valid`); every lane of the warp
// takes part in the butterfly.
template <typename CostT, typename MsgT, bool RW = false>
__device__ __forceinline__ void wta_pixel(const LevelView &lv, int D, int Dp, int Gp, int32_t *disp, int x, int y,
                                          bool valid) {
    using Acc = typename AccOf<MsgT>::type;
    using A = Arith<Acc>;
    const int g = threadIdx.x & (Gp - 1);
    const int64_t p = (int64_t)y * lv.W + x;
    const int c = colour_of(x, y);
    const int64_t s = slot_of(x, y, lv.Wh);
    const int dbase = g * VEC;
    Acc best = A::big();
    int arg = 0x7fffffff;
    if (valid && dbase < Dp) {
        Acc b[VEC], t[VEC];
        load16(reinterpret_cast<const CostT *>(c ? lv.cost[1] : lv.cost[0]) + s * Dp + dbase, b);
        const MsgT *mp = reinterpret_cast<const MsgT *>(c ? lv.msg[1] : lv.msg[0]) + s * 4 * Dp + dbase;
        const bool has[4] = {y > 0, y < lv.H - 1, x > 0, x < lv.W - 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (!has[q]) continue;
            load16_msg<RW>(mp + q * Dp, t);
#pragma unroll
            for (int k = 0; k < VEC; ++k) b[k] += t[k];
        }
#pragma unroll
        for (int k = 0; k < VEC; ++k) {
            const int lab = dbase + pos_label<MsgT>(k);
            if (lab < D && (b[k] < best || (b[k] == best && lab < arg))) {
                best = b[k];
                arg = lab;
            }
        }
    }
    for (int o = Gp >> 1; o > 0; o >>= 1) {
        const Acc ob = __shfl_xor_sync(FULL, best, o, Gp);
        const int oa = __shfl_xor_sync(FULL, arg, o, Gp);
        if (ob < best || (ob == best && oa < arg)) {
            best = ob;
            arg = oa;
        }
    }
    if (valid && g == 0 && BPS_CHECK(p < (int64_t)lv.W * lv.H, lv.err, 5u)) disp[p] = arg;
}

template <typename CostT, typename MsgT, bool RW = false>
__device__ __forceinline__ void wta_group(const LevelView &lv, int D, int Dp, int Gp, int32_t *disp, int64_t block) {
    const int64_t p = block * (blockDim.x / Gp) + threadIdx.x / Gp;
    const bool valid = p < (int64_t)lv.W * lv.H;
    wta_pixel<CostT, MsgT, RW>(lv, D, Dp, Gp, disp, valid ? (int)(p % lv.W) : 0, valid ? (int)(p / lv.W) : 0, valid);
}

}  // namespace bps
