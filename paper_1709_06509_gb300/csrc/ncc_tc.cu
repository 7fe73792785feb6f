// ncc_tc.cu -- the integer data-cost volume (section "Correlation volume computation") with the
// window correlations on the fifth-generation tensor cores (tcgen05), and scale 1 of the cost
// pyramid (section "GPU Implementation") from the same pass.
//
// For one image row y, a tile of 128 consecutive pixels x = x0 + m and a block of labels
// d = d0 + t (t < DB <= 128), every window sum of products
//   S_ab(x, d) = sum_{|j|, |i| <= R} L(x + i, y + j) R(x - d + i, y + j)      (reads clamped)
// is an entry of one matrix product: with u0 = x0 - d0 - (DB - 1) and right positions
// u = u0 + n (n < NB = 127 + DB rounded up to 16),
//   P[m][n] = sum_j sum_i A_j[m][i] B_j[n][i],  A_j[m][i] = L(x0 + m + i - R, y + j),
//                                              B_j[n][i] = R(u0 + n + i - R, y + j),
// S_ab(x0 + m, d0 + t) = P[m][m + DB - 1 - t]: a band of the 128 x NB product.  Each image row
// is one K = 16 slab (its 2R + 1 taps i, zero-padded) of A and of B, written once into shared
// memory and used by the 2R + 1 output rows whose window holds it: the MMA of output row y adds
// up the 2R + 1 slabs of rows y - R .. y + R into a 128-lane x NB-column FP32 accumulator in
// tensor memory, after one more MMA that starts it at 2^23.  Image bytes are exact in BF16 and
// every partial sum is an integer in [2^23, 2^24) (S_ab < 81 * 255^2 < 2^23), exact in FP32, so
// the accumulator's bits are 0x4B000000 + S_ab.
//
// A CTA owns one tile, one label block and a strip of rows, one CTA an SM (its tensor memory is
// two accumulators of 256 columns).  Its warps split the work of a row and pipeline it across
// rows through mbarriers:
//   - 4 producer warps: stage the image row entering the window (left: 128 + 2R columns, right:
//     NB + 2R positions, clamped, fetched a row ahead) into a ring of 2R + 2 rows, as bytes and as
//     BF16; build its two slabs; keep the column sums and sums of squares of the window rows; form
//     the window records of the next row ({-S, T / sqrt(N S_xx - S_x^2)} per pixel,
//     {S, 1 / sqrt(N S_xx - S_x^2)} per right position, and the variance terms); issue its MMAs
//     (one thread); then take the previous row out of the CTA: the FP64 decisions it queued, and
//     its costs in the storage order of the form, with the 2x2 sums of scale 1 completing in
//     registers over each row pair;
//   - 12 epilogue warps: warp w reads lanes 32 (w % 4) .. + 31 (its pixels) and a third of the
//     columns their band spans (tcgen05.ld) and quantises each (pixel, label) with the fp32 step
//     of the row kernel into a byte stage (costs <= T <= 127); a value within the margin of a
//     level boundary is queued for the FP64 sequence.
// Two accumulators, two record buffers and two stages let the MMA of row y + 1, the epilogue of
// row y and the copy-out of row y - 1 run at the same time.  Every wait is bounded: one that gives
// up sets the context's error word, the waiting group leaves its loop (the others then give up in
// turn), and the tensor memory is still freed.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>

#include "bps_internal.cuh"
#include "bps_launch.h"
#include "ncc_quant.cuh"

namespace bps {

namespace {

constexpr int TCN_M = 128;          // pixels a tile (accumulator lanes)
constexpr int TCN_DB = 128;         // labels a block at most
constexpr int TCN_EPI_WARPS = 12;   // three per 32 lanes of tensor memory
constexpr int TCN_PROD = 128;       // producer threads (4 warps)
constexpr int TCN_THREADS = 32 * TCN_EPI_WARPS + TCN_PROD;
constexpr int TCN_QMAX = 256;       // queued FP64 decisions a row (more are decided in place)
constexpr int TCN_ACC_COLS = 256;   // columns an accumulator
constexpr unsigned TCN_WAIT_LIMIT = 1u << 26;  // polls of an mbarrier before giving up

// Shared-memory layout of a CTA (bytes), for label block size DB and window radius R.
struct TcnLayout {
    int DB, NB, NS, LWB, RWB, SSTB;
    unsigned slabA, slabB, magic, rowbf, rowu8, col, rec, stage, queue, misc, total;
};

__host__ __device__ inline TcnLayout tcn_layout(int Dp, int R) {
    TcnLayout t;
    t.DB = Dp < TCN_DB ? Dp : TCN_DB;
    t.NB = (127 + t.DB + 15) / 16 * 16;
    t.NS = 2 * R + 2;
    t.LWB = TCN_M + 2 * R;
    t.RWB = t.NB + 2 * R;
    t.SSTB = t.DB + 80;  // a pixel's staged costs: bytes in label order, 32 spare labels each side
    unsigned o = 0;
    t.slabA = o; o += (unsigned)t.NS * TCN_M * 32;
    t.slabB = o; o += (unsigned)t.NS * t.NB * 32;
    t.magic = o; o += (unsigned)(TCN_M + t.NB) * 32;
    t.rowbf = o; o += (unsigned)t.NS * (t.LWB + t.RWB) * 2; o = (o + 15u) & ~15u;
    t.rowu8 = o; o += (unsigned)t.NS * (t.LWB + t.RWB); o = (o + 15u) & ~15u;
    t.col = o; o += 2u * (t.LWB + t.RWB) * 4u;
    t.rec = o; o += 2u * 2u * (TCN_M + t.NB) * 8u;  // [buffer][hot, cold][pixels, positions] int2
    t.stage = o; o += 2u * TCN_M * (unsigned)t.SSTB;
    t.queue = o; o += 2u * TCN_QMAX * 16u;
    t.misc = o; o += 128u;
    t.total = o;
    return t;
}

__device__ __forceinline__ uint32_t s_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major shared-memory operand without swizzle: 8-row x 16-byte core matrices, 128 bytes
// between the two core matrices of a row group along K, 256 bytes between row groups.
__device__ __forceinline__ uint64_t slab_desc(uint32_t addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)(128u >> 4) << 16) | ((uint64_t)(256u >> 4) << 32) |
           (1ull << 46);
}

// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, N and M.
__device__ __forceinline__ uint32_t tcn_idesc(int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TCN_M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(s_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(s_addr(bar)) : "memory");
}
// Wait until the phase of `bar` with this parity has completed, bounded: false (and the error
// word set) when it gives up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned *err) {
    for (unsigned it = 0; it < TCN_WAIT_LIMIT; ++it) {
        unsigned ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(s_addr(bar)), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    if (err) atomicExch(err, 1u);
    return false;
}
// The producer warps' barrier (named barrier 1), and their vote on a condition; each first
// reconverges its warp (a bounded wait may have split it).
__device__ __forceinline__ void prod_sync() {
    __syncwarp();
    asm volatile("bar.sync 1, %0;" ::"n"(TCN_PROD) : "memory");
}
__device__ __forceinline__ bool prod_any(bool v) {
    __syncwarp();
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.or.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((unsigned)v), "n"(TCN_PROD)
        : "memory");
    return r != 0;
}

// tcgen05.ld of CW consecutive accumulator columns for the warp's 32 lanes (one lane a thread) and
// the wait for it, in one asm statement: the load writes its registers asynchronously, so nothing
// may read, move or reuse them before the wait.
template <int CW> __device__ __forceinline__ void tmem_load(uint32_t addr, uint32_t (&v)[CW]);
template <> __device__ __forceinline__ void tmem_load<16>(uint32_t addr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]), "=r"(v[8]),
          "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(addr)
        : "memory");
}
template <> __device__ __forceinline__ void tmem_load<8>(uint32_t addr, uint32_t (&v)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "r"(addr)
        : "memory");
}
template <> __device__ __forceinline__ void tmem_load<4>(uint32_t addr, uint32_t (&v)[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
        : "r"(addr)
        : "memory");
}

__device__ __forceinline__ int clampi_tc(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ uint16_t bf16_bits(unsigned v) {
    return __bfloat16_as_ushort(__float2bfloat16_rn((float)v));  // exact for v <= 256
}

// A queued FP64 decision of one row: pixel and label, numerator and the two variance terms.
struct __align__(16) TcnFix {
    int lt;  // pixel | label << 8
    int num;
    int va, vb;
};

// A value to decide again in FP64 after the kernel: x, y, label, the fp32 level; numerator and
// the two variance terms.  Each CTA owns a region of per_cta entries after a header entry
// (header.a.x = entries used), written in row order and read by ncc_tc_fix_kernel.
struct __align__(16) TcnEntry {
    int4 a;  // x, y, d, c32
    int4 b;  // num, va, vb, 0
};

// prmt.b32 in its default mode, where a selector nibble with bit 3 set fills its byte with the
// sign (bit 7) of the selected byte (the __byte_perm intrinsic uses only bits 0-2).
__device__ __forceinline__ uint32_t prmt_sign(uint32_t a, uint32_t b, uint32_t sel) {
    uint32_t d;
    asm("prmt.b32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(sel));
    return d;
}

// One pixel's 16 labels, staged as bytes in label order (w[0..3]), stored in the storage order of
// CostT.  Costs are at most 127, so the sign fill gives zero high bytes.
template <typename CostT>
__device__ __forceinline__ void put_group(CostT *dst, const uint32_t (&w)[4]);
template <>
__device__ __forceinline__ void put_group<int16_t>(int16_t *dst, const uint32_t (&w)[4]) {
    // position 2k holds label k, 2k + 1 label k + 8: word j = (label j, label j + 8)
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    d4[0] = make_uint4(prmt_sign(w[0], w[2], 0xC480), prmt_sign(w[0], w[2], 0xD591),
                       prmt_sign(w[0], w[2], 0xE6A2), prmt_sign(w[0], w[2], 0xF7B3));
    d4[1] = make_uint4(prmt_sign(w[1], w[3], 0xC480), prmt_sign(w[1], w[3], 0xD591),
                       prmt_sign(w[1], w[3], 0xE6A2), prmt_sign(w[1], w[3], 0xF7B3));
}
template <>
__device__ __forceinline__ void put_group<int32_t>(int32_t *dst, const uint32_t (&w)[4]) {
    int4 *d4 = reinterpret_cast<int4 *>(dst);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        d4[k] = make_int4((int)(w[k] & 0xffu), (int)((w[k] >> 8) & 0xffu), (int)((w[k] >> 16) & 0xffu),
                          (int)(w[k] >> 24));
}
// The scale-1 sum of a group (16 labels as int16 pairs in label order: s[k] = labels 2k, 2k + 1),
// stored in the storage order of CostT.
template <typename CostT>
__device__ __forceinline__ void put_sum(CostT *dst, const uint32_t (&s)[8]);
template <>
__device__ __forceinline__ void put_sum<int16_t>(int16_t *dst, const uint32_t (&s)[8]) {
    uint4 *d4 = reinterpret_cast<uint4 *>(dst);
    d4[0] = make_uint4(__byte_perm(s[0], s[4], 0x5410), __byte_perm(s[0], s[4], 0x7632),
                       __byte_perm(s[1], s[5], 0x5410), __byte_perm(s[1], s[5], 0x7632));
    d4[1] = make_uint4(__byte_perm(s[2], s[6], 0x5410), __byte_perm(s[2], s[6], 0x7632),
                       __byte_perm(s[3], s[7], 0x5410), __byte_perm(s[3], s[7], 0x7632));
}
template <>
__device__ __forceinline__ void put_sum<int32_t>(int32_t *dst, const uint32_t (&s)[8]) {
    int4 *d4 = reinterpret_cast<int4 *>(dst);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        d4[k] = make_int4((int)(s[2 * k] & 0xffffu), (int)(s[2 * k] >> 16), (int)(s[2 * k + 1] & 0xffffu),
                          (int)(s[2 * k + 1] >> 16));
}

template <typename CostT, int R>
__global__ void __launch_bounds__(TCN_THREADS, 1)
ncc_tc_kernel(const uint8_t *__restrict__ Limg, const uint8_t *__restrict__ Rimg, int pitch, int W, int H, int D,
              int Dp, int T, int rows, LevelView l0, LevelView l1, int write_l1, TcnEntry *fix, int per_cta) {
    static_assert(R <= 4, "windows up to 9: S_ab below 2^23, N S_ab below 2^31");
    constexpr int WIN = 2 * R + 1, N = WIN * WIN;
    extern __shared__ __align__(1024) unsigned char sm[];
    const TcnLayout lay = tcn_layout(Dp, R);
    const int DB = lay.DB, NB = lay.NB, NS = lay.NS, LWB = lay.LWB, RWB = lay.RWB, SSTB = lay.SSTB;
    unsigned char *slabA = sm + lay.slabA;
    unsigned char *slabB = sm + lay.slabB;
    unsigned char *magicA = sm + lay.magic;
    unsigned char *magicB = magicA + TCN_M * 32;
    uint16_t *rowbf = reinterpret_cast<uint16_t *>(sm + lay.rowbf);
    uint8_t *rowu8 = sm + lay.rowu8;
    int *colS = reinterpret_cast<int *>(sm + lay.col);
    int *colQ = colS + (LWB + RWB);
    int2 *rec = reinterpret_cast<int2 *>(sm + lay.rec);  // [buffer][hot | cold][TCN_M + NB]
    uint8_t *stage = sm + lay.stage;                     // [buffer][TCN_M][SSTB]
    TcnFix *queue = reinterpret_cast<TcnFix *>(sm + lay.queue);  // [buffer][TCN_QMAX]
    uint64_t *acc_full = reinterpret_cast<uint64_t *>(sm + lay.misc);  // [2] MMA done + records ready
    uint64_t *acc_empty = acc_full + 2;    // [2] the epilogue has read the accumulator and records
    uint64_t *stage_full = acc_full + 4;   // [2] the epilogue has written the stage
    uint64_t *stage_empty = acc_full + 6;  // [2] the copy-out has read the stage
    int *qcount = reinterpret_cast<int *>(sm + lay.misc + 64);  // [2]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + lay.misc + 72);
    int *fused = reinterpret_cast<int *>(sm + lay.misc + 76);  // entries of the CTA's region in use

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int x0 = blockIdx.x * TCN_M, d0 = blockIdx.y * TCN_DB;
    const int ys = blockIdx.z * rows, ye = min(H, ys + rows);
    const int nrows = max(0, ye - ys);
    const int u0 = x0 - d0 - (DB - 1);
    const int RS = TCN_M + NB;  // records of a row (pixels, then right positions)
    const int64_t cta = blockIdx.x + (int64_t)gridDim.x * (blockIdx.y + (int64_t)gridDim.y * blockIdx.z);

    pdl_enter();
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s_addr(tmem_slot)),
                     "r"(2 * TCN_ACC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(&acc_full[i], 2);  // the MMAs' commit and the producers' records
            mbar_init(&acc_empty[i], 32 * TCN_EPI_WARPS);  // every epilogue thread (its own writes released)
            mbar_init(&stage_full[i], 32 * TCN_EPI_WARPS);
            mbar_init(&stage_empty[i], 1);
            qcount[i] = 0;
        }
        *fused = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // the offset slabs: A holds 2^23 in tap 0 of every row, B holds 1 there
    for (int row = tid; row < TCN_M + NB; row += TCN_THREADS) {
        const bool a = row < TCN_M;
        const int rr = a ? row : row - TCN_M;
        unsigned char *base = (a ? magicA : magicB) + (rr >> 3) * 256 + (rr & 7) * 16;
        *reinterpret_cast<uint4 *>(base) = make_uint4(a ? 0x4B00u : 0x3F80u, 0u, 0u, 0u);
        *reinterpret_cast<uint4 *>(base + 128) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tmem_slot;
    unsigned *err = l0.err;

    if (warp >= TCN_EPI_WARPS) {
        // ------------------------------------------------------------- producers and copy-out
        const int pt = tid - 32 * TCN_EPI_WARPS;
        auto slot_of_row = [&](int r) { return (r - (ys - R)) % NS; };
        // staged positions of a row (LWB + RWB <= 4 * TCN_PROD): up to four a thread, fetched a row ahead
        unsigned pf[4] = {0u, 0u, 0u, 0u};
        auto fetch_row = [&](int r) {
            const int64_t off = (int64_t)clampi_tc(r, 0, H - 1) * pitch;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = pt + j * TCN_PROD;
                if (p < LWB + RWB) {
                    const bool left = p < LWB;
                    const int c = left ? clampi_tc(x0 - R + p, 0, W - 1) : clampi_tc(u0 - R + (p - LWB), 0, W - 1);
                    pf[j] = __ldg((left ? Limg : Rimg) + off + c);
                }
            }
        };
        auto store_row = [&](int r) {
            const int s = slot_of_row(r);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int p = pt + j * TCN_PROD;
                if (p < LWB + RWB) {
                    rowu8[s * (LWB + RWB) + p] = (uint8_t)pf[j];
                    rowbf[s * (LWB + RWB) + p] = bf16_bits(pf[j]);
                }
            }
        };
        // the two K = 16 slabs of the row in slot s: row m of A holds the left taps of pixel
        // x0 + m, row n of B the right taps of position u0 + n; taps past 2R are zero
        auto build_slabs = [&](int s) {
            const uint16_t *src = rowbf + s * (LWB + RWB);
            for (int row = pt; row < TCN_M + NB; row += TCN_PROD) {
                const bool a = row < TCN_M;
                const int rr = a ? row : row - TCN_M;
                const uint16_t *t = src + (a ? rr : LWB + rr);
                uint32_t w[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) {
                    const uint32_t lo = 2 * k < WIN ? (uint32_t)t[2 * k] : 0u;
                    const uint32_t hi = 2 * k + 1 < WIN ? (uint32_t)t[2 * k + 1] : 0u;
                    w[k] = lo | (hi << 16);
                }
                unsigned char *base =
                    (a ? slabA + s * (TCN_M * 32) : slabB + s * (NB * 32)) + (rr >> 3) * 256 + (rr & 7) * 16;
                *reinterpret_cast<uint4 *>(base) = make_uint4(w[0], w[1], w[2], w[3]);
                *reinterpret_cast<uint4 *>(base + 128) = make_uint4(w[4], w[5], w[6], w[7]);
            }
        };
        auto records = [&](int b) {
            int2 *hot = rec + (2 * b) * RS, *cold = rec + (2 * b + 1) * RS;
            for (int k = pt; k < RS; k += TCN_PROD) {
                const bool left = k < TCN_M;
                const int c = left ? k : LWB + (k - TCN_M);
                int s = 0, ss = 0;
#pragma unroll
                for (int q = 0; q < WIN; ++q) {
                    s += colS[c + q];
                    ss += colQ[c + q];
                }
                const unsigned v = (unsigned)N * (unsigned)ss - (unsigned)s * (unsigned)s;
                const float r = v ? rsqrtf((float)v) : 0.f;
                hot[k] = make_int2(left ? -s : s, __float_as_int(left ? __fmul_rn((float)T, r) : r));
                cold[k] = make_int2((int)v, __float_as_int(r));
            }
        };
        // the MMAs of row y into accumulator b: the offset, then the 2R + 1 slabs of its window;
        // one producer thread issues them and commits, and also arrives (records ready)
        auto issue_mma = [&](int y, int b) {
            if (pt == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t idesc = tcn_idesc(NB);
                const uint32_t acc = tmem + (uint32_t)(b * TCN_ACC_COLS);
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 0, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                    "l"(slab_desc(s_addr(magicA))), "l"(slab_desc(s_addr(magicB))), "r"(idesc)
                    : "memory");
#pragma unroll 1
                for (int j = 0; j < WIN; ++j) {
                    const int s = slot_of_row(y - R + j);
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, 1, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(acc),
                        "l"(slab_desc(s_addr(slabA + s * (TCN_M * 32)))),
                        "l"(slab_desc(s_addr(slabB + s * (NB * 32)))), "r"(idesc)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 s_addr(&acc_full[b]))
                             : "memory");
                mbar_arrive(&acc_full[b]);
            }
        };
        // copy-out items: (pixel pair p, label group g); consecutive threads take consecutive
        // groups of a pixel pair; the same items in every row (scale-1 sums in registers)
        constexpr int NIT = (TCN_M / 2) * (TCN_DB / 16) / TCN_PROD;  // 4
        const int ngroups = min(DB, Dp - d0) / 16;
        uint32_t part[NIT][8];
#pragma unroll
        for (int it = 0; it < NIT; ++it)
#pragma unroll
            for (int k = 0; k < 8; ++k) part[it][k] = 0u;
        // the queued decisions of row j and its copy-out
        auto copyout = [&](int j) -> bool {
            const int bj = j & 1, y = ys + j;
            if (prod_any(!mbar_wait_bounded(&stage_full[bj], (unsigned)((j >> 1) & 1), err))) return false;
            uint8_t *stg = stage + bj * (TCN_M * SSTB);
            const int qn = qcount[bj];
            if (qn) {
                const int used = *fused;
                const TcnFix *qb = queue + bj * TCN_QMAX;
                const int qm = min(qn, TCN_QMAX);  // (the epilogue decided the rest in place)
                if (used + qm <= per_cta) {
                    TcnEntry *dst = fix + cta * (int64_t)(per_cta + 1) + 1 + used;
                    for (int i = pt; i < qm; i += TCN_PROD) {
                        const TcnFix f = qb[i];
                        const int pl = f.lt & 255, pl_t = f.lt >> 8;
                        if (!(pl < TCN_M && pl_t >= 0 && pl_t < DB) || !BPS_CHECK(used + i < per_cta, err, 8u)) continue;
                        TcnEntry e;
                        e.a = make_int4(x0 + pl, y, d0 + pl_t, (int)stg[pl * SSTB + 32 + pl_t]);
                        e.b = make_int4(f.num, f.va, f.vb, 0);
                        dst[i] = e;
                    }
                } else {
                    for (int i = pt; i < qm; i += TCN_PROD) {
                        const TcnFix f = qb[i];
                        const int pl = f.lt & 255, pl_t = f.lt >> 8;
                        if (!(pl < TCN_M && pl_t >= 0 && pl_t < DB)) continue;
                        int cc = quantise_fp64<int>(f.num, (unsigned)f.va, (unsigned)f.vb, T);
                        cc = cc < 0 ? 0 : (cc > T ? T : cc);
                        stg[pl * SSTB + 32 + pl_t] = (uint8_t)cc;
                    }
                }
                prod_sync();  // the stage is final; every producer has read qcount and fused
                if (pt == 0) {
                    if (used + qm <= per_cta) *fused = used + qm;
                    qcount[bj] = 0;
                }
            }
            const bool last_of_pair = (y & 1) || y == H - 1;
#pragma unroll
            for (int it = 0; it < NIT; ++it) {
                const int item = pt + it * TCN_PROD;
                const int g = item & 7, p = item >> 3;
                const int xe = x0 + 2 * p;
                if (g >= ngroups || xe >= W) continue;
                const bool odd_ok = xe + 1 < W;
                const uint4 e4 = *reinterpret_cast<const uint4 *>(stg + (2 * p) * SSTB + 32 + 16 * g);
                uint4 o4 = make_uint4(0u, 0u, 0u, 0u);
                if (odd_ok) o4 = *reinterpret_cast<const uint4 *>(stg + (2 * p + 1) * SSTB + 32 + 16 * g);
                uint32_t we[4] = {e4.x, e4.y, e4.z, e4.w}, wo[4] = {o4.x, o4.y, o4.z, o4.w};
                const int dpos = d0 + 16 * g;  // the group's first storage position (aligned groups)
                if (dpos + 16 > D) {           // padding labels (D and above) cost 0
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) {
                        unsigned keep = 0u;
#pragma unroll
                        for (int bb = 0; bb < 4; ++bb) keep |= (dpos + 4 * k2 + bb < D ? 0xffu : 0u) << (8 * bb);
                        we[k2] &= keep;
                        wo[k2] &= keep;
                    }
                }
                const int64_t slot = (int64_t)y * l0.Wh + (xe >> 1);
                if (!BPS_CHECK(slot < (int64_t)l0.H * l0.Wh && dpos + 16 <= Dp, err, 6u)) continue;
                put_group<CostT>(reinterpret_cast<CostT *>(l0.cost[(xe + y) & 1]) + slot * Dp + dpos, we);
                if (odd_ok)
                    put_group<CostT>(reinterpret_cast<CostT *>(l0.cost[(xe + 1 + y) & 1]) + slot * Dp + dpos, wo);
                if (write_l1) {
                    // int16 pairs in label order: labels (2k, 2k + 1) of both children, no carry
#pragma unroll
                    for (int k2 = 0; k2 < 4; ++k2) {
                        part[it][2 * k2] += __byte_perm(we[k2], 0u, 0x4140) + __byte_perm(wo[k2], 0u, 0x4140);
                        part[it][2 * k2 + 1] += __byte_perm(we[k2], 0u, 0x4342) + __byte_perm(wo[k2], 0u, 0x4342);
                    }
                    if (last_of_pair) {
                        const int X = xe >> 1, Y = y >> 1;
                        if (BPS_CHECK(slot_of(X, Y, l1.Wh) < (int64_t)l1.H * l1.Wh, err, 7u))
                            put_sum<CostT>(
                                reinterpret_cast<CostT *>(l1.cost[(X + Y) & 1]) + slot_of(X, Y, l1.Wh) * Dp + dpos,
                                part[it]);
#pragma unroll
                        for (int k2 = 0; k2 < 8; ++k2) part[it][k2] = 0u;
                    }
                }
            }
            prod_sync();  // every producer has read the stage
            if (pt == 0) mbar_arrive(&stage_empty[bj]);
            return true;
        };

        bool ok = nrows > 0;
        if (ok) {
            // the window of the strip's first row: rows ys - R .. ys + R
            for (int r = ys - R; r <= ys + R; ++r) {
                fetch_row(r);
                store_row(r);
            }
            prod_sync();
            for (int r = ys - R; r <= ys + R; ++r) build_slabs(slot_of_row(r));
            for (int p = pt; p < LWB + RWB; p += TCN_PROD) {
                int s = 0, ss = 0;
                for (int r = ys - R; r <= ys + R; ++r) {
                    const int v = rowu8[slot_of_row(r) * (LWB + RWB) + p];
                    s += v;
                    ss += v * v;
                }
                colS[p] = s;
                colQ[p] = ss;
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            prod_sync();
            records(0);
            prod_sync();
            issue_mma(ys, 0);
            if (nrows > 1) fetch_row(ys + 1 + R);
        }
        for (int k = 0; ok && k < nrows; ++k) {
            const int y = ys + k;
            if (k + 1 < nrows) {
                // the entering row goes into the slot of row y - R - 1, read last by MMA(y - 1)
                if (k >= 1 &&
                    prod_any(!mbar_wait_bounded(&acc_full[(k - 1) & 1], (unsigned)(((k - 1) >> 1) & 1), err))) {
                    ok = false;
                    break;
                }
                store_row(y + 1 + R);
                prod_sync();
                const int sin = slot_of_row(y + 1 + R), sout = slot_of_row(y - R);
                build_slabs(sin);
                for (int p = pt; p < LWB + RWB; p += TCN_PROD) {
                    const int vi = rowu8[sin * (LWB + RWB) + p], vo = rowu8[sout * (LWB + RWB) + p];
                    colS[p] += vi - vo;
                    colQ[p] += vi * vi - vo * vo;
                }
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                prod_sync();
                // the records and the accumulator of row y + 1 replace those of row y - 1
                const int b1 = (k + 1) & 1;
                if (prod_any(!mbar_wait_bounded(&acc_empty[b1], (unsigned)((((k + 1) >> 1) + 1) & 1), err))) {
                    ok = false;
                    break;
                }
                records(b1);
                prod_sync();
                issue_mma(y + 1, b1);
                if (k + 2 < nrows) fetch_row(y + 2 + R);  // in flight during the copy-out
            }
            if (k >= 1 && !copyout(k - 1)) {
                ok = false;
                break;
            }
        }
        if (ok && nrows > 0) copyout(nrows - 1);
    } else {
        // ------------------------------------------------------------- epilogue warps
        const int q4 = warp & 3, share = warp >> 2;  // share 0..2 of the quarter's columns
        const int l = 32 * q4 + lane;
        const bool px_ok = x0 + l < W;
        // the 32 + DB columns the band of the quarter's 32 lanes spans, in pieces of 4 split in
        // three shares (the larger first)
        const int P4 = (32 + DB) / 4;
        const int s0 = (P4 + 2) / 3, s1 = (P4 + 1) / 3;
        const int cs = 32 * q4 + 4 * (share == 0 ? 0 : (share == 1 ? s0 : s0 + s1));
        const int ce = 32 * q4 + 4 * (share == 0 ? s0 : (share == 1 ? s0 + s1 : P4));
        const int tmax = min(DB, D - d0);  // labels of the block below D
        const float T_half = (float)T + 0.5f, half_m = 0.5f - (float)(T + 1) * (1.f / 131072.f);
        // N S_ab - S_a S_b = N bits - N bits(2^23) - S_a S_b, in 32-bit wrap-around arithmetic
        // (the result fits a signed int)
        const unsigned KOFF = 0u - (unsigned)N * 0x4B000000u;
        auto numer = [&](uint32_t bits, int negSa, int Sb) -> int {
            return (int)(bits * (unsigned)N + ((unsigned)(negSa * Sb) + KOFF));
        };
        for (int k = 0; k < nrows; ++k) {
            const int b = k & 1;
            bool got = mbar_wait_bounded(&acc_full[b], (unsigned)((k >> 1) & 1), err);
            got = got && mbar_wait_bounded(&stage_empty[b], (unsigned)(((k >> 1) + 1) & 1), err);
            if (!__all_sync(0xffffffffu, got)) break;
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const int2 *hot = rec + (2 * b) * RS, *cold = rec + (2 * b + 1) * RS;
            const int negSa = hot[l].x;
            const float tra = __int_as_float(hot[l].y);
            const int va = cold[l].x;
            // the stage row of pixel l has 32 spare labels on each side: every column of the
            // quarter's pieces lands inside the row, in the band or in a margin nobody reads
            uint8_t *srow = stage + b * (TCN_M * SSTB) + l * SSTB + 32;
            TcnFix *qb = queue + b * TCN_QMAX;
            const uint32_t lane_base = tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)(b * TCN_ACC_COLS);
            // one piece of CW columns from c0: right positions u0 + c0 + r, labels t = tb - r
            auto piece = [&](auto cw_tag, int c0) {
                constexpr int CW = decltype(cw_tag)::value;
                uint32_t v[CW];
                __syncwarp();  // the previous piece's queue loop may have split the warp
                BPS_CHECK(c0 >= 0 && c0 + CW <= NB && l + DB - 1 - c0 - (CW - 1) >= -32 && l + DB - 1 - c0 <= DB + 30,
                          err, 9u);
                tmem_load<CW>(lane_base + (uint32_t)c0, v);
                const int tb = l + DB - 1 - c0;
                uint8_t *sdst = srow + tb;
                const int4 *rb4 = reinterpret_cast<const int4 *>(hot + TCN_M + c0);
                unsigned near_mask = 0u;
#pragma unroll
                for (int h2 = 0; h2 < CW / 2; ++h2) {
                    const int4 pb = rb4[h2];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int r = 2 * h2 + e;
                        const int num = numer(v[r], negSa, e ? pb.z : pb.x);
                        bool near;
                        const int c = quantise_fp32((float)num, tra, __int_as_float(e ? pb.w : pb.y), T_half, half_m,
                                                    T, &near);
                        near_mask |= (near ? 1u : 0u) << r;
                        if (px_ok) sdst[-r] = (uint8_t)c;
                    }
                }
                // only the real labels of the band: registers tb - tmax < r <= tb
                const int rlo = max(0, tb - tmax + 1), rhi = min(CW - 1, tb);
                near_mask &= (rlo <= rhi && px_ok) ? ((2u << rhi) - (1u << rlo)) : 0u;
                while (near_mask) {  // rare: queued for the FP64 decision
                    const int r = __ffs(near_mask) - 1;
                    near_mask &= near_mask - 1;
                    uint32_t bits = v[0];
#pragma unroll
                    for (int rr = 1; rr < CW; ++rr) bits = rr == r ? v[rr] : bits;
                    const int n = c0 + r;
                    const int num = numer(bits, negSa, hot[TCN_M + n].x);
                    const int vb = cold[TCN_M + n].x;
                    const int qi = atomicAdd(&qcount[b], 1);
                    if (qi < TCN_QMAX) {
                        TcnFix f;
                        f.lt = l | ((tb - r) << 8);
                        f.num = num;
                        f.va = va;
                        f.vb = vb;
                        qb[qi] = f;
                    } else {  // a full queue: decided here
                        int cc = quantise_fp64<int>(num, (unsigned)va, (unsigned)vb, T);
                        cc = cc < 0 ? 0 : (cc > T ? T : cc);
                        sdst[-r] = (uint8_t)cc;
                    }
                }
            };
            // pieces aligned to their width: 16 where the column is a multiple of 16, else 8, else 4
            for (int c0 = cs; c0 < ce;) {
                if (!(c0 & 15) && c0 + 16 <= ce) {
                    piece(std::integral_constant<int, 16>(), c0);
                    c0 += 16;
                } else if (!(c0 & 7) && c0 + 8 <= ce) {
                    piece(std::integral_constant<int, 8>(), c0);
                    c0 += 8;
                } else {
                    piece(std::integral_constant<int, 4>(), c0);
                    c0 += 4;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            mbar_arrive(&acc_empty[b]);
            mbar_arrive(&stage_full[b]);
        }
    }
    // release the tensor memory (every MMA has completed, or a wait gave up)
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) fix[cta * (int64_t)(per_cta + 1)].a.x = *fused;
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * TCN_ACC_COLS)
                     : "memory");
    }
}

// The FP64 decisions of the values the kernel listed: one block a CTA region.  A value whose
// level changes is stored again, and the change is added to its scale-1 sum (atomically: the
// four children of a coarse cost may change in different blocks; every partial sum stays
// non-negative, so a 16-bit half never borrows from its neighbour).  The block empties its
// region for the next launch.
template <typename CostT>
__global__ void __launch_bounds__(128)
ncc_tc_fix_kernel(TcnEntry *fix, int per_cta, LevelView l0, LevelView l1, int write_l1, int Dp, int T) {
    pdl_enter();
    TcnEntry *reg = fix + (int64_t)blockIdx.x * (per_cta + 1);
    const int n = min(reg[0].a.x, per_cta);
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const TcnEntry e = reg[1 + i];
        const int x = e.a.x, y = e.a.y, d = e.a.z, c32 = e.a.w;
        int c = quantise_fp64<int>(e.b.x, (unsigned)e.b.y, (unsigned)e.b.z, T);
        c = c < 0 ? 0 : (c > T ? T : c);
        if (c == c32) continue;
        const int pos = label_pos<CostT>(d);
        if (!BPS_CHECK(x >= 0 && x < l0.W && y >= 0 && y < l0.H && d >= 0 && d < Dp, l0.err, 12u)) continue;
        reinterpret_cast<CostT *>(l0.cost[(x + y) & 1])[slot_of(x, y, l0.Wh) * Dp + pos] = (CostT)c;
        if (write_l1) {
            const int X = x >> 1, Y = y >> 1;
            CostT *pc = reinterpret_cast<CostT *>(l1.cost[(X + Y) & 1]) + slot_of(X, Y, l1.Wh) * Dp + pos;
            if constexpr (sizeof(CostT) == 4) {
                atomicAdd(reinterpret_cast<int *>(pc), c - c32);
            } else {
                unsigned *word = reinterpret_cast<unsigned *>(reinterpret_cast<uintptr_t>(pc) & ~(uintptr_t)3);
                atomicAdd(word, (unsigned)(c - c32) << ((pos & 1) ? 16 : 0));
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) reg[0].a.x = 0;
}

int g_optin_tc = 0;
int smem_optin_tc() {
    if (!g_optin_tc) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        g_optin_tc = v;
    }
    return g_optin_tc;
}

template <typename CostT, int R> void *tc_kernel_ptr() { return (void *)ncc_tc_kernel<CostT, R>; }

template <typename CostT> void *tc_kernel(int R) {
    switch (R) {
    case 0: return tc_kernel_ptr<CostT, 0>();
    case 1: return tc_kernel_ptr<CostT, 1>();
    case 2: return tc_kernel_ptr<CostT, 2>();
    case 3: return tc_kernel_ptr<CostT, 3>();
    default: return tc_kernel_ptr<CostT, 4>();
    }
}

}  // namespace

// At least 120 KB, so that two CTAs never share an SM's shared memory and with it its tensor
// memory (each allocates all 512 columns).
size_t ncc_tc_smem_bytes(int Dp, int window) {
    return std::max<size_t>(tcn_layout(Dp, window / 2).total, 120u * 1024u);
}

bool ncc_tc_supported(int cost_kind, int Dp, int window, int T) {
    // the stage holds costs as bytes, their high bytes filled from bit 7 (T <= 127)
    if (cost_kind == COST_F32 || window < 1 || window > NCC_TC_MAX_WINDOW || !(window & 1) || T < 0 || T > 127)
        return false;
    return (int)ncc_tc_smem_bytes(Dp, window) <= smem_optin_tc();
}

// The limit is a property of the kernel function, shared by every context of the process (and
// their label counts), so it is raised once to the device's opt-in maximum; each launch still
// requests only what its shape needs.
cudaError_t ncc_tc_prepare(int cost_kind, int Dp) {
    (void)Dp;
    if (cost_kind == COST_F32) return cudaSuccess;
    for (int R = 0; R <= NCC_TC_MAX_WINDOW / 2; ++R) {
        void *k = cost_kind == COST_I16 ? tc_kernel<int16_t>(R) : tc_kernel<int32_t>(R);
        const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin_tc());
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Rows per strip (even) so that tiles x label blocks x strips cover the SMs about once.
static int tc_default_rows(int W, int H, int Dp) {
    int sms = 152, dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int tiles = ((W + TCN_M - 1) / TCN_M) * ((Dp + TCN_DB - 1) / TCN_DB);
    const int strips = std::max(1, sms / std::max(1, tiles));
    int rows = (H + strips - 1) / strips;
    return std::max(2, (rows + 1) & ~1);
}

template <typename CostT, int R>
static cudaError_t launch_tc_t(const uint8_t *L, const uint8_t *Rim, int pitch, int W, int H, int D, int Dp, int T,
                               const LevelView &l0, const LevelView *l1, cudaStream_t st, int rows, TcnEntry *fix,
                               size_t fix_entries) {
    const dim3 grid((W + TCN_M - 1) / TCN_M, (Dp + TCN_DB - 1) / TCN_DB, (H + rows - 1) / rows);
    const int64_t nctas = (int64_t)grid.x * grid.y * grid.z;
    const int per_cta = (int)std::min<int64_t>(1 << 30, std::max<int64_t>(0, (int64_t)fix_entries / nctas - 1));
    if (!fix || per_cta < 1) return cudaErrorInvalidValue;  // the kernel writes each region's header
    const size_t smem = ncc_tc_smem_bytes(Dp, 2 * R + 1);
    const LevelView l1v = l1 ? *l1 : l0;
    cudaError_t e = launch_k(ncc_tc_kernel<CostT, R>, grid, dim3(TCN_THREADS), smem, st, L, Rim, pitch, W, H, D, Dp,
                             T, rows, l0, l1v, l1 ? 1 : 0, fix, per_cta);
    if (e == cudaSuccess)
        e = launch_k(ncc_tc_fix_kernel<CostT>, dim3((unsigned)nctas), dim3(128), 0, st, fix, per_cta, l0, l1v,
                     l1 ? 1 : 0, Dp, T);
    return e;
}

template <typename CostT>
static cudaError_t launch_tc(int R, const uint8_t *L, const uint8_t *Rim, int pitch, int W, int H, int D, int Dp,
                             int T, const LevelView &l0, const LevelView *l1, cudaStream_t st, int rows, TcnEntry *fix,
                             size_t n) {
    switch (R) {
    case 0: return launch_tc_t<CostT, 0>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, st, rows, fix, n);
    case 1: return launch_tc_t<CostT, 1>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, st, rows, fix, n);
    case 2: return launch_tc_t<CostT, 2>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, st, rows, fix, n);
    case 3: return launch_tc_t<CostT, 3>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, st, rows, fix, n);
    default: return launch_tc_t<CostT, 4>(L, Rim, pitch, W, H, D, Dp, T, l0, l1, st, rows, fix, n);
    }
}

size_t ncc_tc_fix_bytes(int W, int H, int Dp) {
    // about 6 times the expected share of values near a level boundary (2 (T + 1) 2^-17 <= 3e-4)
    const size_t entries = std::max<size_t>(16384, (size_t)W * H * Dp / 512);
    return entries * sizeof(TcnEntry);
}

cudaError_t launch_ncc_tc(int cost_kind, const uint8_t *L, const uint8_t *Rim, int pitch, int W, int H, int D, int Dp,
                          int window, int T, const LevelView &l0, const LevelView *l1, cudaStream_t st, int rows,
                          void *fix, size_t fix_bytes) {
    if (!ncc_tc_supported(cost_kind, Dp, window, T)) return cudaErrorInvalidValue;
    if (rows <= 0) rows = tc_default_rows(W, H, Dp);
    const int R = window / 2;
    TcnEntry *f = reinterpret_cast<TcnEntry *>(fix);
    const size_t n = fix ? fix_bytes / sizeof(TcnEntry) : 0;
    // strips few enough that every CTA's region holds its header and at least one entry
    const int64_t tiles = (int64_t)((W + TCN_M - 1) / TCN_M) * ((Dp + TCN_DB - 1) / TCN_DB);
    const int64_t max_strips = std::max<int64_t>(1, (int64_t)(n / 2) / tiles);
    rows = std::max<int64_t>(rows, (H + max_strips - 1) / max_strips);
    rows = std::max(2, (rows + 1) & ~1);
    if (cost_kind == COST_I16) return launch_tc<int16_t>(R, L, Rim, pitch, W, H, D, Dp, T, l0, l1, st, rows, f, n);
    return launch_tc<int32_t>(R, L, Rim, pitch, W, H, D, Dp, T, l0, l1, st, rows, f, n);
}

}  // namespace bps
