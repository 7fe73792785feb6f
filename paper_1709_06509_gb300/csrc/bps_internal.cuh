// bps_internal.cuh -- device-side layout and helpers shared by the stereo kernels.
//
// Layout in HBM (per scale l, W_l x H_l pixels, Dp = D rounded up to 16 labels):
//   Pixels are split by checkerboard colour c = (x + y) & 1 ("red-black").  Pixel (x, y)
//   lives in the colour-c arrays at slot s = y * Wh + (x >> 1), Wh = ceil(W_l / 2).  A
//   half-sweep of colour c then reads one dense block (the colour-c records) and writes
//   one dense block (the other colour's message slots): no half-used 32-byte sectors.
//   cost[c]   [H_l][Wh][Dp]      data cost            (int32 | int16 | float)
//   msg[c]    [H_l][Wh][4][Dp]   incoming messages    (int32 | uint8 | half)
//             direction = the neighbour the message comes from: 0 up, 1 down, 2 left, 3 right
//   dirty[c]  [H_l][Wh] uint32   1 = some incoming message changed since the last update
//   Labels d >= D inside the Dp padding are never winners: the sweep treats their belief
//   as +infinity.
//
// A pixel's Dp labels are handled by a group of Gp (a power of two <= 32) consecutive lanes,
// VEC = 16 labels per lane, so one lane moves 16 labels with 16-byte vector accesses.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace bps {

constexpr int VEC = 16;              // labels per lane
constexpr int DIR_UP = 0, DIR_DOWN = 1, DIR_LEFT = 2, DIR_RIGHT = 3;
constexpr int BIG_I = 1 << 29;       // "+infinity" of the integer forms

struct LevelView {
    int W, H, Wh;
    void *cost[2];
    void *msg[2];
    unsigned *dirty[2];  // 32-bit words so a sender can flip them atomically: bit 0 dirty, bit 1 frozen
    int eps;             // skip rule: a receiver is marked when its message moves by more than eps
    int freeze;          // skip rule: a recomputed pixel that marked no receiver is frozen
    // u8 form: 1 when every message a half-sweep reads is at most 63 (lambda * trunc <= 63 and no
    // caller-given start messages), so four of them add up bytewise without a carry
    int bsum8;
    // 1: a recomputed pixel leaves its own skip flag alone (the first half of a temporally blocked
    // first iteration, whose flags are cleared before the launch)
    int keep_flag;
    // A scale's first iteration without a separate coarse-to-fine copy (u8 sweeps): start = 1, the
    // first half-sweep reads each even pixel's start messages straight from its parent's record
    // (pmsg, pWh: the parent scale's message arrays and slots per row) and recomputes every
    // pixel; start = 2, the second half-sweep recomputes every pixel.  0 otherwise.
    int start;
    int pWh;
    const void *pmsg[2];
    // Read-out during the finest scale's half-sweeps (u8 form, exact skip rule): each recomputed
    // pixel writes the argmin of the belief it forms to disp[y * W + x] (nullable: no read-out).
    int32_t *disp;
    // Error word of the context's device-side checks: 1 when a bounded wait of a bulk-copy sweep gave
    // up, 2 and above from the debug build's bounds checks; read and cleared by bps_get_error.
    unsigned *err;
};

// Device-side consistency checks of the debug build (compiled with -DBPS_DEBUG_BOUNDS): a failed
// check records its code in the context's error word (the largest code wins) and the caller skips
// the access it guards; bps_get_error then reports BPS_ERR_INTERNAL.  In the normal build a check
// is the constant true and costs nothing.  Codes: 2 a list entry past the scale, 3 a list append
// past its capacity, 4 a data-cost store outside its scale, 5 a read-out pixel outside the image;
// the tensor-core NCC: 6 a data-cost store, 7 a scale-1 store, 8 an FP64 list entry, 9 an
// accumulator column or stage label, 10 a window record, 11 a slab row, 12 an FP64 pass store.
#ifdef BPS_DEBUG_BOUNDS
__device__ __forceinline__ bool bps_check(bool ok, unsigned *err, unsigned code) {
    if (!ok && err) atomicMax(err, code);
    return ok;
}
#define BPS_CHECK(cond, err, code) ::bps::bps_check((cond), (err), (code))
#else
#define BPS_CHECK(cond, err, code) true
#endif

// Programmatic dependent launch: every kernel of the stereo chain is launched so that it may
// start while its predecessor is still running; it waits here until the predecessor's grid
// has completed and its writes are visible, then lets its own successor start launching.
// Without a programmatic predecessor the wait returns at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__host__ __device__ inline int colour_of(int x, int y) { return (x + y) & 1; }
__host__ __device__ inline int64_t slot_of(int x, int y, int Wh) { return (int64_t)y * Wh + (x >> 1); }

// ------------------------------------------------------------------ arithmetic per form
template <typename T> struct Arith;
template <> struct Arith<int> {
    __device__ static inline int big() { return BIG_I; }
    __device__ static inline int mn(int a, int b) { return min(a, b); }
};
template <> struct Arith<float> {
    __device__ static inline float big() { return __int_as_float(0x7f800000); }
    __device__ static inline float mn(float a, float b) { return fminf(a, b); }
};

// ------------------------------------------------------------------ 16-label vector I/O
// load16: read labels [0, 16) starting at p (16-byte aligned) into A registers.
__device__ inline void load16(const uint8_t *p, int (&v)[VEC]) {
    const uint4 r = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = (w[k >> 2] >> (8 * (k & 3))) & 0xff;
}
__device__ inline void load16(const int16_t *p, int (&v)[VEC]) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint4 r = __ldg(q + h);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int k = 0; k < 8; ++k) v[8 * h + k] = (int)(int16_t)(w[k >> 1] >> (16 * (k & 1)));
    }
}
__device__ inline void load16(const int32_t *p, int (&v)[VEC]) {
    const int4 *q = reinterpret_cast<const int4 *>(p);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int4 r = __ldg(q + h);
        v[4 * h + 0] = r.x; v[4 * h + 1] = r.y; v[4 * h + 2] = r.z; v[4 * h + 3] = r.w;
    }
}
__device__ inline void load16(const float *p, float (&v)[VEC]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const float4 r = __ldg(q + h);
        v[4 * h + 0] = r.x; v[4 * h + 1] = r.y; v[4 * h + 2] = r.z; v[4 * h + 3] = r.w;
    }
}
__device__ inline void load16(const __half *p, float (&v)[VEC]) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint4 r = __ldg(q + h);
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const __half2 hv = *reinterpret_cast<const __half2 *>(&w[k]);
            const float2 f = __half22float2(hv);
            v[8 * h + 2 * k] = f.x;
            v[8 * h + 2 * k + 1] = f.y;
        }
    }
}

// Plain (coherent) loads, for message slots the same kernel may also write.
__device__ inline void load16_rw(const uint8_t *p, int (&v)[VEC]) {
    const uint4 r = *reinterpret_cast<const uint4 *>(p);
    const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
    for (int k = 0; k < VEC; ++k) v[k] = (w[k >> 2] >> (8 * (k & 3))) & 0xff;
}
__device__ inline void load16_rw(const int32_t *p, int (&v)[VEC]) {
    const int4 *q = reinterpret_cast<const int4 *>(p);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int4 r = q[h];
        v[4 * h + 0] = r.x; v[4 * h + 1] = r.y; v[4 * h + 2] = r.z; v[4 * h + 3] = r.w;
    }
}
__device__ inline void load16_rw(const __half *p, float (&v)[VEC]) {
    const uint4 *q = reinterpret_cast<const uint4 *>(p);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint4 r = q[h];
        const uint32_t w[4] = {r.x, r.y, r.z, r.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2 *>(&w[k]));
            v[8 * h + 2 * k] = f.x;
            v[8 * h + 2 * k + 1] = f.y;
        }
    }
}

// Message loads of a kernel that may also have written them earlier in the same launch (a
// cluster or persistent kernel, across its barriers) must take the coherent path.
template <bool RW, typename T, typename V> __device__ inline void load16_msg(const T *p, V (&v)[VEC]) {
    if constexpr (RW) load16_rw(p, v);
    else load16(p, v);
}
template <bool RW> __device__ inline uint4 load_u4(const uint4 *p) {
    if constexpr (RW) return *p;
    else return __ldg(p);
}

// The value a message takes once stored (fp16 rounds; the integer forms are exact).
template <typename MsgT> __device__ inline int stored_value(int v) { return v; }
template <typename MsgT> __device__ inline float stored_value(float v) { return __half2float(__float2half_rn(v)); }

__device__ inline void store16(uint8_t *p, const int (&v)[VEC]) {
    uint32_t w[4];
#pragma unroll
    for (int j = 0; j < 4; ++j)
        w[j] = (uint32_t)(v[4 * j] & 0xff) | ((uint32_t)(v[4 * j + 1] & 0xff) << 8) |
               ((uint32_t)(v[4 * j + 2] & 0xff) << 16) | ((uint32_t)(v[4 * j + 3] & 0xff) << 24);
    *reinterpret_cast<uint4 *>(p) = make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ inline void store16(int16_t *p, const int (&v)[VEC]) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
            w[j] = (uint32_t)(uint16_t)v[8 * h + 2 * j] | ((uint32_t)(uint16_t)v[8 * h + 2 * j + 1] << 16);
        q[h] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}
__device__ inline void store16(int32_t *p, const int (&v)[VEC]) {
    int4 *q = reinterpret_cast<int4 *>(p);
#pragma unroll
    for (int h = 0; h < 4; ++h) q[h] = make_int4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
}
__device__ inline void store16(float *p, const float (&v)[VEC]) {
    float4 *q = reinterpret_cast<float4 *>(p);
#pragma unroll
    for (int h = 0; h < 4; ++h) q[h] = make_float4(v[4 * h], v[4 * h + 1], v[4 * h + 2], v[4 * h + 3]);
}
__device__ inline void store16(__half *p, const float (&v)[VEC]) {
    uint4 *q = reinterpret_cast<uint4 *>(p);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint32_t w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __half2 hv = __floats2half2_rn(v[8 * h + 2 * j], v[8 * h + 2 * j + 1]);
            w[j] = *reinterpret_cast<const uint32_t *>(&hv);
        }
        q[h] = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Storage order of labels.  The u8 form (int16 costs, uint8 messages) interleaves each
// aligned group of 16 labels: position 2k holds label k and position 2k+1 holds label k+8
// (k < 8), so one 32-bit word of int16 costs, or one byte pair of messages, carries labels
// (k, k+8).  The other forms keep the natural order.
template <typename T> __host__ __device__ inline int label_pos(int d) { return d; }
template <> __host__ __device__ inline int label_pos<int16_t>(int d) {
    const int k = d & 15;
    return (d & ~15) | (k < 8 ? 2 * k : 2 * (k - 8) + 1);
}
template <> __host__ __device__ inline int label_pos<uint8_t>(int d) { return label_pos<int16_t>(d); }
template <typename T> __host__ __device__ inline int pos_label(int p) { return p; }
template <> __host__ __device__ inline int pos_label<int16_t>(int p) {
    const int k = p & 15;
    return (p & ~15) | ((k & 1) ? 8 + (k >> 1) : (k >> 1));
}
template <> __host__ __device__ inline int pos_label<uint8_t>(int p) { return pos_label<int16_t>(p); }

// Accumulator type of each storage form.
template <typename MsgT> struct AccOf { using type = int; };
template <> struct AccOf<__half> { using type = float; };

}  // namespace bps
