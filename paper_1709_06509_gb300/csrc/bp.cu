// bp.cu -- hierarchical min-sum loopy BP on the 4-connected grid (sections "Fast
// Converging BP" and "GPU Implementation"): one kernel launch per red-black half-sweep,
// the coarse-to-fine start, and import / export of messages and costs in the natural
// layout.  The per-pixel work lives in sweep_body.cuh.
#include <cooperative_groups.h>

#include <algorithm>
#include <type_traits>

#include "bps_launch.h"
#include "sweep_body.cuh"

namespace bps {

// Grid-stride over the pixel blocks: the grid is capped at the CTAs resident at once, so a
// large scale does not pay for scheduling tens of thousands of CTAs that mostly find clean
// pixels.
template <typename CostT, typename MsgT>
__global__ void __launch_bounds__(256)
sweep_kernel(LevelView lv, int colour, int D, int Dp, int Gp, typename AccOf<MsgT>::type lam,
             typename AccOf<MsgT>::type lamT, int skip, unsigned long long *trace, int nblocks) {
    pdl_enter();
    Tally tally(trace);
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x)
        sweep_group<CostT, MsgT>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b);
    tally.flush();
}

// Grid-stride over the colour's pixel blocks: the grid is capped at what is resident at
// once, so a launch pays for block scheduling once, not once per wave.
#ifndef BPS_SWEEP_MIN_BLOCKS
#define BPS_SWEEP_MIN_BLOCKS 3  // resident CTAs per SM the u8 sweep is compiled for (distance transform)
#endif
#ifndef BPS_SWEEP_STENCIL_MIN_BLOCKS
// ... and with the stencil minimisation (T <= 2) and D a multiple of 16: 64 registers a thread,
// 32 warps an SM, which hides more of the dependent round trips to memory than 24 (spills of at
// most 8 bytes a thread)
#define BPS_SWEEP_STENCIL_MIN_BLOCKS 4
#endif
#define BPS_SWEEP_BLOCKS(PADDED, TS) (((TS) == 0 || (PADDED)) ? BPS_SWEEP_MIN_BLOCKS : BPS_SWEEP_STENCIL_MIN_BLOCKS)

template <bool PADDED, bool APPEND, int TS, bool DP>
__global__ void __launch_bounds__(256, BPS_SWEEP_BLOCKS(PADDED, TS))
sweep_u8_kernel(LevelView lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                unsigned long long *trace, int nblocks, ActiveList al) {
    unsigned *abuf = nullptr;
    if constexpr (APPEND) {
        BPS_LIST_BUFFER(list_buf);
        abuf = list_buf[threadIdx.x >> 5];
    }
    pdl_enter();
    Tally tally(trace, abuf);
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x) {
        if constexpr (DP) sweep_group_u8_dp<PADDED, APPEND, TS>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b, al);
        else sweep_group_u8<PADDED, APPEND, TS>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b, al);
    }
    if constexpr (APPEND) tally.flush_appends(al.out, al.n_out, (unsigned)lv.H * (unsigned)lv.Wh, lv.err);
    tally.flush();
}

// The same half-sweep with every load issued at once (see EAGER in sweep_group_u8): the first
// block of each CTA loads its costs before waiting for the predecessor kernel.
template <bool PADDED, int TS, bool DP>
__global__ void __launch_bounds__(256, BPS_SWEEP_BLOCKS(PADDED, TS))
sweep_u8_eager_kernel(LevelView lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                      unsigned long long *trace, int nblocks) {
    Tally tally(trace);
    if constexpr (DP) {
        sweep_group_u8_dp<PADDED, false, TS, 2>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, blockIdx.x);
        for (int b = blockIdx.x + gridDim.x; b < nblocks; b += gridDim.x)
            sweep_group_u8_dp<PADDED, false, TS, 1>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b);
    } else {
        sweep_group_u8<PADDED, false, TS, false, 2>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, blockIdx.x);
        for (int b = blockIdx.x + gridDim.x; b < nblocks; b += gridDim.x)
            sweep_group_u8<PADDED, false, TS, false, 1>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b);
    }
    tally.flush();
}

// The same half-sweep with staged inputs (see stage_u8): each thread copies the next block's
// inputs into its shared-memory stage while it computes the current block (two stages, so a
// stage is refilled only after the block that read it has been computed).
#ifndef BPS_SWEEP_STAGED_MIN_BLOCKS
#define BPS_SWEEP_STAGED_MIN_BLOCKS 2  // 2 x 256 threads x 2 stages x 11 chunks x 16 B = 180 KB a SM
#endif
template <bool PADDED, bool APPEND, int TS>
__global__ void __launch_bounds__(256, BPS_SWEEP_STAGED_MIN_BLOCKS)
sweep_u8_staged_kernel(LevelView lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                       unsigned long long *trace, int nblocks, ActiveList al) {
    extern __shared__ uint4 stage_mem[];  // [2][STAGE_CHUNKS][blockDim.x]
    pdl_enter();
    const int stage_len = STAGE_CHUNKS * blockDim.x;
    int buf = 0;
    unsigned *abuf = nullptr;
    if constexpr (APPEND) {
        BPS_LIST_BUFFER(list_buf);
        abuf = list_buf[threadIdx.x >> 5];
    }
    Tally tally(trace, abuf);
    if (blockIdx.x < (unsigned)nblocks) stage_u8(lv, colour, Dp, Gp, skip, blockIdx.x, stage_mem);
    cp_async_commit();
    for (int b = blockIdx.x; b < nblocks; b += gridDim.x, buf ^= 1) {
        if (b + (int)gridDim.x < nblocks)
            stage_u8(lv, colour, Dp, Gp, skip, b + gridDim.x, stage_mem + (buf ^ 1) * stage_len);
        cp_async_commit();
        cp_async_wait<1>();  // block b's copies have landed; the next block's may be in flight
        sweep_group_u8<PADDED, APPEND, TS, false, 3>(lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b, al, 0, 0,
                                                     stage_mem + buf * stage_len);
    }
    if constexpr (APPEND) tally.flush_appends(al.out, al.n_out, (unsigned)lv.H * (unsigned)lv.Wh, lv.err);
    tally.flush();
    cp_async_wait<0>();
}

// The staged half-sweep over the pixels of an active list: the entries of a thread's current
// and next block are read one block ahead of their copies, the copies one block ahead of the
// computation.
template <bool PADDED, int TS>
__global__ void __launch_bounds__(256, BPS_SWEEP_STAGED_MIN_BLOCKS)
sweep_u8_staged_list_kernel(LevelView lv, int colour, int D, int Dp, int Gp, int lam, int lamT,
                            unsigned long long *trace, ActiveList al) {
    extern __shared__ uint4 stage_mem[];  // [2][STAGE_CHUNKS][blockDim.x]
    pdl_enter();
    const int stage_len = STAGE_CHUNKS * blockDim.x;
    const int groups = blockDim.x / Gp;
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    const int64_t stride = (int64_t)gridDim.x * groups;
    int64_t idx = (int64_t)blockIdx.x * groups + threadIdx.x / Gp;
    // the length and the first two entries are read together: an entry past the length is
    // stale but inside the buffer, which holds a slot of every pixel of a colour
    const unsigned e0 = idx < nslot ? al.in[idx] : 0u;
    const unsigned e1 = idx + stride < nslot ? al.in[idx + stride] : 0u;
    const int64_t n = *al.n_in;
    int64_t cur = idx < n ? (int64_t)e0 : nslot;
    int64_t nxt = idx + stride < n ? (int64_t)e1 : nslot;
    int buf = 0;
    BPS_LIST_BUFFER(list_buf);
    Tally tally(trace, list_buf[threadIdx.x >> 5]);
    if ((int64_t)blockIdx.x * groups < n) stage_u8<true>(lv, colour, Dp, Gp, 1, blockIdx.x, stage_mem, cur);
    cp_async_commit();
    for (int64_t b = blockIdx.x; b * groups < n; b += gridDim.x, idx += stride, buf ^= 1) {
        if ((b + gridDim.x) * groups < n)
            stage_u8<true>(lv, colour, Dp, Gp, 1, b + gridDim.x, stage_mem + (buf ^ 1) * stage_len, nxt);
        cp_async_commit();
        const int64_t after = idx + 2 * stride < n ? (int64_t)al.in[idx + 2 * stride] : nslot;
        cp_async_wait<1>();  // block b's copies have landed; the next block's may be in flight
        sweep_group_u8<PADDED, true, TS, false, 3, true>(lv, colour, D, Dp, Gp, lam, lamT, 1, tally, b, al, n, cur,
                                                         stage_mem + buf * stage_len);
        cur = nxt;
        nxt = after;
    }
    tally.flush_appends(al.out, al.n_out, (unsigned)nslot, lv.err);
    tally.flush();
    cp_async_wait<0>();
}

static size_t staged_smem_bytes() { return (size_t)2 * STAGE_CHUNKS * 256 * sizeof(uint4); }

// ------------------------------------------------------------------ bulk-copy pipeline
// sweep_u8_bulk_kernel: one warp of the CTA copies, eight compute.  The copy warp walks the CTA's
// pixel blocks (grid-stride; consecutive slots, or the entries of an active list) and, for every
// pixel that needs it, issues 1-D bulk copies (cp.async.bulk, completion counted in bytes on an
// mbarrier) of its whole records into a stage of shared memory: the cost record (2 Dp bytes), the
// incoming record (4 Dp; the parent's record in a scale's first half-sweep) and, for the skip's
// change test, the receivers' four slots (Dp each; the parents' slots in a scale's second
// half-sweep).  The compute warps wait for a stage, run the u8 body on it and release it.  Memory
// parallelism then costs shared memory only, and the copies of the next block are in flight while
// the current one computes, stores its messages and flips the skip flags.  Every wait is bounded:
// a wait that gives up sets lv.err and the CTA returns (the copy warp first waits, again bounded,
// for the stages it filled).
constexpr int BULK_THREADS = BULK_CONSUMERS + 32, BULK_STAGES = 2;
constexpr unsigned BULK_WAIT_LIMIT = 1u << 22;  // try_wait attempts before a wait gives up (seconds)

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(ok)
                 : "r"(smem_u32(bar)), "r"(parity)
                 : "memory");
    return ok != 0;
}
// Wait for phase `parity` of `bar` to complete, at most BULK_WAIT_LIMIT attempts; false (and the
// error word set) when it gives up or another warp already has.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, unsigned parity, unsigned *err) {
    for (unsigned it = 0; it < BULK_WAIT_LIMIT; ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 255u) == 255u && err && *reinterpret_cast<volatile unsigned *>(err)) return false;
    }
    if (err) atomicExch(err, 1u);
    return false;
}
__device__ __forceinline__ void bulk_copy(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

__host__ __device__ inline size_t bulk_stage_bytes(int Dp, int Gp) {
    return ((size_t)(BULK_CONSUMERS / Gp) * 10 * Dp + 127) / 128 * 128;
}
static size_t bulk_smem_bytes(int Dp, int Gp) {
    return BULK_STAGES * bulk_stage_bytes(Dp, Gp) + 2 * BULK_STAGES * sizeof(uint64_t) +
           (size_t)BULK_STAGES * (BULK_CONSUMERS / Gp) * sizeof(unsigned);
}
constexpr size_t BULK_SMEM_MAX = BULK_STAGES * (size_t)BULK_CONSUMERS * 10 * VEC + 2 * BULK_STAGES * 8 +
                                 BULK_STAGES * BULK_CONSUMERS * 4;

// LISTED: the pixels are the entries of al.in (count *al.n_in); otherwise consecutive slots, and a
// pixel is copied and computed only when it needs it (scale start, skip off, or its flag set).
template <bool PADDED, int TS, bool LISTED, bool APPEND>
__global__ void __launch_bounds__(BULK_THREADS, 2)
sweep_u8_bulk_kernel(LevelView lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                     unsigned long long *trace, int nblocks, ActiveList al) {
    extern __shared__ __align__(128) unsigned char bulk_mem[];
    const int P = BULK_CONSUMERS / Gp;  // pixels a block
    const size_t stage_bytes = bulk_stage_bytes(Dp, Gp);
    uint64_t *full = reinterpret_cast<uint64_t *>(bulk_mem + BULK_STAGES * stage_bytes);
    uint64_t *empty = full + BULK_STAGES;
    unsigned *slots = reinterpret_cast<unsigned *>(empty + BULK_STAGES);  // [BULK_STAGES][P]
    if (threadIdx.x == 0) {
        for (int k = 0; k < BULK_STAGES; ++k) {
            mbar_init(&full[k], 1);                      // the copy warp's arrival (and the bytes)
            mbar_init(&empty[k], BULK_CONSUMERS / 32);  // one arrival per compute warp
        }
    }
    __syncthreads();
    pdl_enter();
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    const int64_t n = LISTED ? (int64_t)*al.n_in : nslot;
    const int64_t nb = LISTED ? (n + P - 1) / P : nblocks;
    const int16_t *cost = reinterpret_cast<const int16_t *>(colour ? lv.cost[1] : lv.cost[0]);
    const uint8_t *msg_in = reinterpret_cast<const uint8_t *>(colour ? lv.msg[1] : lv.msg[0]);
    const uint8_t *msg_out = reinterpret_cast<const uint8_t *>(colour ? lv.msg[0] : lv.msg[1]);
    const unsigned *dirty_in = colour ? lv.dirty[1] : lv.dirty[0];
    const bool old_copies = skip && lv.start != 1;  // a scale's first half-sweep compares nothing

    if (threadIdx.x >= BULK_CONSUMERS) {  // the copy warp
        const int lane = threadIdx.x & 31;
        int64_t k = 0;
        bool ok = true;
        for (int64_t b = blockIdx.x; b < nb; b += gridDim.x, ++k) {
            const int st = (int)(k % BULK_STAGES);
            if (k >= BULK_STAGES && !mbar_wait(&empty[st], (unsigned)((k / BULK_STAGES - 1) & 1), lv.err)) {
                ok = false;
                break;
            }
            unsigned char *base = bulk_mem + st * stage_bytes;
            unsigned *sl = slots + st * P;
            unsigned bytes = 0;
            for (int i = lane; i < P; i += 32) {  // which pixels, and how many bytes they bring
                int64_t s = b * P + i;
                if (LISTED) s = s < n ? (int64_t)al.in[s] : nslot;
                bool act = false;
                if (s < nslot) {
                    const int y = (int)(s / lv.Wh);
                    const int x = 2 * (int)(s - (int64_t)y * lv.Wh) + ((y + colour) & 1);
                    act = x < lv.W && (LISTED || !skip || lv.start != 0 || dirty_in[s] == 1u);
                    if (act && old_copies) {
                        const int nq = (y > 0) + (y < lv.H - 1) + (x > 0) + (x < lv.W - 1);
                        bytes += (unsigned)(nq * Dp);
                    }
                }
                sl[i] = act ? (unsigned)s : 0xffffffffu;
                if (act) bytes += (unsigned)(6 * Dp);
            }
            for (int o = 16; o > 0; o >>= 1) bytes += __shfl_xor_sync(FULL, bytes, o);
            __syncwarp();
            if (lane == 0) mbar_arrive_expect_tx(&full[st], bytes);
            __syncwarp();
            for (int i = lane; i < P; i += 32) {
                const unsigned s = sl[i];
                if (s == 0xffffffffu) continue;
                const int y = (int)(s / (unsigned)lv.Wh);
                const int x = 2 * (int)(s - (unsigned)y * (unsigned)lv.Wh) + ((y + colour) & 1);
                bulk_copy(base + (size_t)i * 2 * Dp, cost + (int64_t)s * Dp, 2 * Dp, &full[st]);
                const uint8_t *src = msg_in + (int64_t)s * 4 * Dp;
                if (lv.start == 1) {  // a scale's first half-sweep: the parent's record
                    const int px = x >> 1, py = y >> 1;
                    src = reinterpret_cast<const uint8_t *>(colour_of(px, py) ? lv.pmsg[1] : lv.pmsg[0]) +
                          slot_of(px, py, lv.pWh) * 4 * Dp;
                }
                bulk_copy(base + (size_t)P * 2 * Dp + (size_t)i * 4 * Dp, src, 4 * Dp, &full[st]);
                if (old_copies) {
                    const bool has[4] = {y > 0, y < lv.H - 1, x > 0, x < lv.W - 1};
                    const int nbx[4] = {x, x, x - 1, x + 1};
                    const int nby[4] = {y - 1, y + 1, y, y};
                    const int opp[4] = {DIR_DOWN, DIR_UP, DIR_RIGHT, DIR_LEFT};
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        if (!has[q]) continue;
                        const uint8_t *o = lv.start == 2 ? start_slot_u8(lv, nbx[q], nby[q], opp[q], Dp, 0, true)
                                                         : msg_out + (slot_of(nbx[q], nby[q], lv.Wh) * 4 + opp[q]) * Dp;
                        bulk_copy(base + (size_t)P * 6 * Dp + (size_t)i * 4 * Dp + q * Dp, o, Dp, &full[st]);
                    }
                }
            }
        }
        if (!ok) {
            // a wait gave up: let the stages this warp filled land before the CTA returns
            for (int64_t j = (k > BULK_STAGES ? k - BULK_STAGES : 0); j < k; ++j)
                mbar_wait(&full[j % BULK_STAGES], (unsigned)((j / BULK_STAGES) & 1), nullptr);
        }
        return;
    }
    // the compute warps
    Tally tally(trace);
    int64_t k = 0;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x, ++k) {
        const int st = (int)(k % BULK_STAGES);
        if (!mbar_wait(&full[st], (unsigned)((k / BULK_STAGES) & 1), lv.err)) break;
        const unsigned s = slots[st * P + threadIdx.x / Gp];
        sweep_group_u8<PADDED, APPEND, TS, false, 4, true>(
            lv, colour, D, Dp, Gp, lam, lamT, skip, tally, b, al, n, s == 0xffffffffu ? nslot : (int64_t)s,
            reinterpret_cast<const uint4 *>(bulk_mem + st * stage_bytes));
        __syncwarp();
        if ((threadIdx.x & 31) == 0) mbar_arrive(&empty[st]);
    }
    tally.flush();
}

// CTAs of the bulk-copy sweep resident at once for this shared-memory size.
static int resident_bulk_blocks(size_t smem) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_u8_bulk_kernel<false, 2, true, true>, BULK_THREADS,
                                                  smem);
    return std::max(1, sms * std::max(1, per_sm));
}

template <bool PADDED, int TS>
static cudaError_t launch_u8_bulk(const LevelView &lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                                  unsigned long long *trace, const ActiveList &al, cudaStream_t st) {
    static int cached_smem = -1, cached_grid = 0;  // the resident CTAs depend on the stage size only
    const size_t smem = bulk_smem_bytes(Dp, Gp);
    if ((int)smem != cached_smem) {
        cached_grid = resident_bulk_blocks(smem);
        cached_smem = (int)smem;
    }
    const int P = BULK_CONSUMERS / Gp;
    const int64_t blocks = ((int64_t)lv.H * lv.Wh + P - 1) / P;
    if (blocks == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>(blocks, cached_grid);
    if (skip && al.in)
        return launch_k(sweep_u8_bulk_kernel<PADDED, TS, true, true>, dim3(grid), dim3(BULK_THREADS), smem, st, lv,
                        colour, D, Dp, Gp, lam, lamT, skip, trace, (int)blocks, al);
    const ActiveList dense{nullptr, nullptr, al.out, al.n_out};
    if (al.out)
        return launch_k(sweep_u8_bulk_kernel<PADDED, TS, false, true>, dim3(grid), dim3(BULK_THREADS), smem, st, lv,
                        colour, D, Dp, Gp, lam, lamT, skip, trace, (int)blocks, dense);
    return launch_k(sweep_u8_bulk_kernel<PADDED, TS, false, false>, dim3(grid), dim3(BULK_THREADS), smem, st, lv,
                    colour, D, Dp, Gp, lam, lamT, skip, trace, (int)blocks, dense);
}

// A list launch's loop over the entries with one group of Gp lanes a pixel, or with 4 Gp lanes
// a pixel (DP: one group per direction); `e` is this thread's first entry, read by the caller
// together with the list length n.  Indexes are 32-bit: a colour has at most 2^30 pixels
// (bps_create admits at most 2^31 pixels), so n, idx + stride and b * groups stay below 2^31.
template <bool PADDED, int TS, bool DP>
__device__ __forceinline__ void list_loop(const LevelView &lv, int colour, int D, int Dp, int Gp, int lam, int lamT,
                                          Tally &trace, const ActiveList &al, unsigned n, unsigned e) {
    const unsigned lpp = DP ? 4 * Gp : Gp;  // lanes a pixel
    const unsigned groups = blockDim.x / lpp;
    const unsigned nslot = (unsigned)lv.H * (unsigned)lv.Wh;
    const unsigned stride = gridDim.x * groups;
    unsigned idx = blockIdx.x * groups + threadIdx.x / lpp;
    for (unsigned b = blockIdx.x; b * groups < n; b += gridDim.x, idx += stride) {
        const unsigned s = idx < n ? e : nslot;
        if (idx + stride < n) e = al.in[idx + stride];
        if constexpr (DP) sweep_group_u8_dp<PADDED, true, TS, 0, true>(lv, colour, D, Dp, Gp, lam, lamT, 1, trace, b, al, s);
        else sweep_group_u8<PADDED, true, TS, false, 0, true>(lv, colour, D, Dp, Gp, lam, lamT, 1, trace, b, al, n, s);
    }
}

// The same half-sweep over the pixels of an active list; its length is read on the device
// (a recorded graph keeps the launch shape, the list decides the work).  DP: direction-parallel
// lanes while the list has at most dp_max entries (short lists: a quarter of the dependent work
// per lane), one group a pixel on longer ones (fewer passes of the resident CTAs).
template <bool PADDED, int TS, bool DP>
__global__ void __launch_bounds__(256, BPS_SWEEP_BLOCKS(PADDED, TS))
sweep_u8_list_kernel(LevelView lv, int colour, int D, int Dp, int Gp, int lam, int lamT,
                     unsigned long long *trace, ActiveList al, int64_t dp_max) {
    pdl_enter();
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    // the list length and this thread's first entry (of either lane mapping) are read together:
    // an entry past the length is stale but inside the buffer, which holds a slot of every
    // pixel of a colour
    const int64_t i_pix = (int64_t)blockIdx.x * (blockDim.x / Gp) + threadIdx.x / Gp;
    const unsigned e_pix = i_pix < nslot ? al.in[i_pix] : 0u;
    unsigned e_dp = 0u;
    if constexpr (DP) {
        const int64_t i_dp = (int64_t)blockIdx.x * (blockDim.x / (4 * Gp)) + threadIdx.x / (4 * Gp);
        e_dp = i_dp < nslot ? al.in[i_dp] : 0u;
    }
    const unsigned n = *al.n_in;
    BPS_LIST_BUFFER(list_buf);
    Tally tally(trace, list_buf[threadIdx.x >> 5], true);
    if (DP && n <= dp_max) list_loop<PADDED, TS, DP>(lv, colour, D, Dp, Gp, lam, lamT, tally, al, n, e_dp);
    else list_loop<PADDED, TS, false>(lv, colour, D, Dp, Gp, lam, lamT, tally, al, n, e_pix);
    tally.settle(al.out, al.n_out, (unsigned)nslot, lv.err);  // the last block's deferred appends
    tally.flush_appends(al.out, al.n_out, (unsigned)nslot, lv.err);
    tally.flush();
}

// ------------------------------------------------------------------ temporal blocking, depth 2
// A scale's first iteration with the fused coarse-to-fine start in ONE launch, tile by tile: a CTA
// takes a tile of BLK_TW x BLK_TH pixels and computes first every even pixel of the tile, then the
// even pixels just outside it that send to its odd pixels (the rows above and below, the columns
// to the left and right), all from their parents' start messages (start 1), and, after a CTA
// barrier, every odd pixel of the tile (start 2) from the messages just written, which it reads
// back from L2 instead of HBM.  An even pixel is computed by its own tile and by every tile it
// borders: each writes the same bytes (its inputs are its cost and its parent's record, which no
// pixel of this launch writes), and only its own tile counts it in the trace.  The first half
// changes no skip flag (the even flags are cleared before the launch), so the marks that a
// neighbouring tile's second half sets are never lost; the second half marks and lists exactly as
// the unblocked second half-sweep.  Results are those of the two separate half-sweeps.
constexpr int BLK_TW = 32, BLK_TH = 16;  // tile width (even) and height (even)

template <bool PADDED, bool APPEND, int TS>
__global__ void __launch_bounds__(256, BPS_SWEEP_BLOCKS(PADDED, TS))
sweep_u8_block2_kernel(LevelView first, LevelView second, int D, int Dp, int Gp, int lam, int lamT,
                       unsigned long long *trace0, unsigned long long *trace1, ActiveList al, int tiles_x, int tiles) {
    unsigned *abuf = nullptr;
    if constexpr (APPEND) {
        BPS_LIST_BUFFER(list_buf);
        abuf = list_buf[threadIdx.x >> 5];
    }
    pdl_enter();
    Tally t0(trace0), t1(trace1, abuf), ring(nullptr);
    const int W = first.W, H = first.H, Wh = first.Wh;
    const int64_t nslot = (int64_t)H * Wh;
    const int groups = blockDim.x / Gp, gi = threadIdx.x / Gp;
    constexpr int HALF = BLK_TW / 2;                  // pixels of one colour in a tile row
    constexpr int OWN = BLK_TH * HALF;                // entries of one colour in a tile
    constexpr int RING = 2 * HALF + BLK_TH;           // even pixels around it (rows, then columns)
    const ActiveList none{nullptr, nullptr, nullptr, nullptr};
    // the slot of the k-th pixel of colour c in the tile's rows y0 .. y0 + th - 1, columns x0 .. x0 + tw - 1
    auto own_slot = [&](int c, int k, int x0, int y0, int tw, int th) -> int64_t {
        const int row = k / HALF, i = k % HALF, y = y0 + row, x = x0 + ((c + y) & 1) + 2 * i;
        return (row < th && x < x0 + tw) ? (int64_t)y * Wh + (x >> 1) : nslot;
    };
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int x0 = (tile % tiles_x) * BLK_TW, y0 = (tile / tiles_x) * BLK_TH;
        const int tw = min(BLK_TW, W - x0), th = min(BLK_TH, H - y0);
        for (int k0 = 0; k0 < OWN; k0 += groups)
            sweep_group_u8<PADDED, false, TS, false, 0, true>(first, 0, D, Dp, Gp, lam, lamT, 1, t0, 0, none, 0,
                                                              own_slot(0, k0 + gi, x0, y0, tw, th));
        for (int r0 = 0; r0 < RING; r0 += groups) {
            const int r = r0 + gi;
            int x = -1, y = -1;
            if (r < 2 * HALF) {  // the rows above and below: their even pixels over the tile's columns
                y = r < HALF ? y0 - 1 : y0 + th;
                x = x0 + (y & 1) + 2 * (r % HALF);
                if (x >= x0 + tw) x = -1;
            } else if (r < 2 * HALF + BLK_TH / 2) {  // the column to the left: even where y is odd
                x = x0 - 1;
                y = y0 + 1 + 2 * (r - 2 * HALF);
            } else if (r < RING) {  // the column to the right
                x = x0 + tw;
                y = y0 + (x & 1) + 2 * (r - 2 * HALF - BLK_TH / 2);
            }
            // a column pixel must border a tile row; a row pixel is one row outside the tile
            const bool in = x >= 0 && x < W && y >= 0 && y < H && (r < 2 * HALF || y < y0 + th);
            sweep_group_u8<PADDED, false, TS, false, 0, true>(first, 0, D, Dp, Gp, lam, lamT, 1, ring, 0, none, 0,
                                                              in ? (int64_t)y * Wh + (x >> 1) : nslot);
        }
        __syncthreads();  // the tile's odd pixels' incoming messages are written
        for (int k0 = 0; k0 < OWN; k0 += groups)
            sweep_group_u8<PADDED, APPEND, TS, true, 0, true>(second, 1, D, Dp, Gp, lam, lamT, 1, t1, 0, al, 0,
                                                              own_slot(1, k0 + gi, x0, y0, tw, th));
    }
    if constexpr (APPEND) t1.flush_appends(al.out, al.n_out, (unsigned)nslot, second.err);
    t0.flush();
    t1.flush();
}

__global__ void clear_flags_kernel(unsigned *flags, int64_t n) {
    pdl_enter();
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x)
        flags[k] = 0u;
}

template <bool PADDED, int TS>
static cudaError_t launch_block2_t(const LevelView &first, const LevelView &second, int D, int Dp, int Gp, int lam,
                                   int lamT, unsigned long long *trace0, unsigned long long *trace1,
                                   const ActiveList &al, int grid, int tiles_x, int tiles, cudaStream_t st) {
    if (al.out)
        return launch_k(sweep_u8_block2_kernel<PADDED, true, TS>, dim3(grid), dim3(256), 0, st, first, second, D, Dp,
                        Gp, lam, lamT, trace0, trace1, al, tiles_x, tiles);
    return launch_k(sweep_u8_block2_kernel<PADDED, false, TS>, dim3(grid), dim3(256), 0, st, first, second, D, Dp, Gp,
                    lam, lamT, trace0, trace1, al, tiles_x, tiles);
}

static int resident_blocks(int ts, bool padded);

cudaError_t launch_sweep_block2(const LevelView &first, const LevelView &second, int D, int Dp, int Gp, int lambda,
                                int trunc, unsigned long long *trace0, unsigned long long *trace1,
                                const SweepLists &lists, cudaStream_t st) {
    const int64_t nslot = (int64_t)first.H * first.Wh;
    if (nslot == 0) return cudaSuccess;
    cudaError_t e = launch_k(clear_flags_kernel, dim3((unsigned)std::min<int64_t>((nslot + 255) / 256, 4096)),
                             dim3(256), 0, st, first.dirty[0], nslot);
    if (e != cudaSuccess) return e;
    const int tiles_x = (first.W + BLK_TW - 1) / BLK_TW, tiles_y = (first.H + BLK_TH - 1) / BLK_TH;
    const int tiles = tiles_x * tiles_y;
    const int lam = trunc == 0 ? 0 : lambda;
    const int ts = trunc <= 1 ? 1 : (trunc == 2 ? 2 : 0);
    const bool padded = (D & 15) != 0;
    const int grid = (int)std::min<int64_t>(tiles, resident_blocks(ts, padded));
    const ActiveList al{nullptr, nullptr, lists.out, lists.n_out};
    switch (ts) {
    case 1: return padded ? launch_block2_t<true, 1>(first, second, D, Dp, Gp, lam, lam * trunc, trace0, trace1, al, grid, tiles_x, tiles, st)
                          : launch_block2_t<false, 1>(first, second, D, Dp, Gp, lam, lam * trunc, trace0, trace1, al, grid, tiles_x, tiles, st);
    case 2: return padded ? launch_block2_t<true, 2>(first, second, D, Dp, Gp, lam, lam * trunc, trace0, trace1, al, grid, tiles_x, tiles, st)
                          : launch_block2_t<false, 2>(first, second, D, Dp, Gp, lam, lam * trunc, trace0, trace1, al, grid, tiles_x, tiles, st);
    default: return padded ? launch_block2_t<true, 0>(first, second, D, Dp, Gp, lam, lam * trunc, trace0, trace1, al, grid, tiles_x, tiles, st)
                           : launch_block2_t<false, 0>(first, second, D, Dp, Gp, lam, lam * trunc, trace0, trace1, al, grid, tiles_x, tiles, st);
    }
}

// Every iteration of one small scale in ONE launch of ONE thread-block cluster.  The CTAs of
// a cluster are co-scheduled, so the hardware cluster barrier (release / acquire at cluster
// scope, covering global memory) separates the half-sweeps: no software spin, no launch per
// half-sweep.  Used where the whole scale is a few passes of the cluster's threads.
constexpr int CLUSTER_CTAS = 16, CLUSTER_THREADS = 512;

template <bool PADDED, int TS, int EAGER>
__global__ void __launch_bounds__(CLUSTER_THREADS, 1)
sweep_u8_cluster_kernel(LevelView lv, int D, int Dp, int Gp, int lam, int lamT, int skip, unsigned long long *trace,
                        int iters, int nblocks) {
    pdl_enter();
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    const int ncta = (int)cl.num_blocks(), rank = (int)cl.block_rank();
    for (int it = 0; it < iters; ++it)
        for (int colour = 0; colour < 2; ++colour) {
            Tally tr(trace ? trace + 2 * it + colour : nullptr);
            for (int b = rank; b < nblocks; b += ncta)
                sweep_group_u8<PADDED, false, TS, true, EAGER>(lv, colour, D, Dp, Gp, lam, lamT, skip, tr, b);
            tr.flush();
            cl.sync();
        }
}

template <bool PADDED, int TS, int EAGER>
static cudaError_t launch_cluster_ts(const LevelView &lv, int D, int Dp, int Gp, int lam, int lamT, int skip,
                                     unsigned long long *trace, int iters, cudaStream_t st) {
    const int groups = CLUSTER_THREADS / Gp;
    const int nblocks = (int)(((int64_t)lv.H * lv.Wh + groups - 1) / groups);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CLUSTER_CTAS);
    cfg.blockDim = dim3(CLUSTER_THREADS);
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CLUSTER_CTAS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[1].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, sweep_u8_cluster_kernel<PADDED, TS, EAGER>, lv, D, Dp, Gp, lam, lamT, skip, trace,
                              iters, nblocks);
}

template <int EAGER>
static cudaError_t launch_cluster_form(bool padded, int ts, const LevelView &lv, int D, int Dp, int Gp, int lam,
                                       int lt, int skip, unsigned long long *trace, int iters, cudaStream_t st) {
    if (padded) {
        if (ts == 1) return launch_cluster_ts<true, 1, EAGER>(lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
        if (ts == 2) return launch_cluster_ts<true, 2, EAGER>(lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
        return launch_cluster_ts<true, 0, EAGER>(lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
    }
    if (ts == 1) return launch_cluster_ts<false, 1, EAGER>(lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
    if (ts == 2) return launch_cluster_ts<false, 2, EAGER>(lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
    return launch_cluster_ts<false, 0, EAGER>(lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
}

cudaError_t launch_sweep_level_cluster(const LevelView &lv, int D, int Dp, int Gp, int lambda, int trunc, int skip,
                                       unsigned long long *trace, int iters, int variant, cudaStream_t st) {
    const int lam = trunc == 0 ? 0 : lambda;
    const int ts = (variant & VARIANT_GENERAL_DT) ? 0 : (trunc <= 1 ? 1 : (trunc == 2 ? 2 : 0));
    const int lt = lam * trunc;
    const bool eager = (variant & VARIANT_EAGER) != 0;
    if (eager) return launch_cluster_form<1>(D & 15, ts, lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
    return launch_cluster_form<0>(D & 15, ts, lv, D, Dp, Gp, lam, lt, skip, trace, iters, st);
}

template <bool PADDED, int TS, int EAGER> static cudaError_t prepare_cluster1() {
    cudaError_t e = cudaFuncSetAttribute(sweep_u8_cluster_kernel<PADDED, TS, EAGER>,
                                         cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    cudaFuncAttributes a;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, sweep_u8_cluster_kernel<PADDED, TS, EAGER>);
    return e;
}
template <bool PADDED, int TS> static cudaError_t prepare_cluster() {
    const cudaError_t e = prepare_cluster1<PADDED, TS, 0>();
    return e == cudaSuccess ? prepare_cluster1<PADDED, TS, 1>() : e;
}

// Whether a 16-CTA cluster of the u8 sweep fits on this GPU (looked up once per process).
bool cluster_sweep_available() {
    static int state = -1;
    if (state < 0) {
        state = 0;
        if (prepare_cluster<false, 0>() == cudaSuccess && prepare_cluster<false, 1>() == cudaSuccess &&
            prepare_cluster<false, 2>() == cudaSuccess && prepare_cluster<true, 0>() == cudaSuccess &&
            prepare_cluster<true, 1>() == cudaSuccess && prepare_cluster<true, 2>() == cudaSuccess) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(CLUSTER_CTAS);
            cfg.blockDim = dim3(CLUSTER_THREADS);
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = CLUSTER_CTAS;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            int clusters = 0;
            if (cudaOccupancyMaxActiveClusters(&clusters, sweep_u8_cluster_kernel<false, 0, 0>, &cfg) == cudaSuccess &&
                clusters >= 1)
                state = 1;
        }
        cudaGetLastError();
    }
    return state == 1;
}

// Kernel of one u8 half-sweep: padding variant x list / append mode x minimisation form.
// CTAs of the staged sweep that fit on the GPU at once (looked up once per process).
static int resident_staged_blocks() {
    static int cached = 0;
    if (!cached) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_u8_staged_kernel<false, false, 0>, 256,
                                                      staged_smem_bytes());
        cached = std::max(1, sms * std::max(1, per_sm));
    }
    return cached;
}

template <bool PADDED, int TS, bool DP>
static cudaError_t launch_u8_dp(const LevelView &lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                                unsigned long long *trace, int64_t blocks, unsigned grid, const ActiveList &al,
                                bool eager, cudaStream_t st, bool staged = false, bool bulk = false) {
    if constexpr (!DP) {
        if (bulk) return launch_u8_bulk<PADDED, TS>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, al, st);
        if (staged && skip && al.in)
            return launch_k(sweep_u8_staged_list_kernel<PADDED, TS>,
                            dim3((unsigned)std::min<int64_t>(blocks, resident_staged_blocks())), dim3(256),
                            staged_smem_bytes(), st, lv, colour, D, Dp, Gp, lam, lamT, trace, al);
        if (staged && !al.in) {
            const unsigned g = (unsigned)std::min<int64_t>(blocks, resident_staged_blocks());
            const ActiveList dense{nullptr, nullptr, al.out, al.n_out};
            if (al.out)
                return launch_k(sweep_u8_staged_kernel<PADDED, true, TS>, dim3(g), dim3(256), staged_smem_bytes(), st,
                                lv, colour, D, Dp, Gp, lam, lamT, skip, trace, (int)blocks, dense);
            return launch_k(sweep_u8_staged_kernel<PADDED, false, TS>, dim3(g), dim3(256), staged_smem_bytes(), st, lv,
                            colour, D, Dp, Gp, lam, lamT, skip, trace, (int)blocks, dense);
        }
    }
    if (eager && !al.in && !al.out)  // grid <= blocks: every CTA has a first block
        return launch_k(sweep_u8_eager_kernel<PADDED, TS, DP>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp,
                        lam, lamT, skip, trace, (int)blocks);
    if (skip && al.in) {
        // direction-parallel lanes up to about one and a half passes of the launch's CTAs
        const int64_t dp_max = DP ? (int64_t)grid * (256 / (4 * Gp)) * 3 / 2 : 0;
        return launch_k(sweep_u8_list_kernel<PADDED, TS, DP>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp, lam,
                        lamT, trace, al, dp_max);
    }
    const ActiveList dense{nullptr, nullptr, al.out, al.n_out};
    if (al.out)
        return launch_k(sweep_u8_kernel<PADDED, true, TS, DP>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp,
                        lam, lamT, skip, trace, (int)blocks, dense);
    return launch_k(sweep_u8_kernel<PADDED, false, TS, DP>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp, lam,
                    lamT, skip, trace, (int)blocks, dense);
}

template <bool PADDED, int TS>
static cudaError_t launch_u8_ts(const LevelView &lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                                unsigned long long *trace, int64_t blocks, unsigned grid, const ActiveList &al,
                                bool eager, bool dp, bool staged, bool bulk, cudaStream_t st) {
    if (dp) return launch_u8_dp<PADDED, TS, true>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, blocks, grid, al, eager, st);
    return launch_u8_dp<PADDED, TS, false>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, blocks, grid, al, eager, st,
                                           staged, bulk);
}

template <bool PADDED>
static cudaError_t launch_u8(int ts, const LevelView &lv, int colour, int D, int Dp, int Gp, int lam, int lamT, int skip,
                             unsigned long long *trace, int64_t blocks, unsigned grid, const ActiveList &al,
                             bool eager, bool dp, bool staged, bool bulk, cudaStream_t st) {
    switch (ts) {
    case 1:
        return launch_u8_ts<PADDED, 1>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, blocks, grid, al, eager, dp,
                                       staged, bulk, st);
    case 2:
        return launch_u8_ts<PADDED, 2>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, blocks, grid, al, eager, dp,
                                       staged, bulk, st);
    default:
        return launch_u8_ts<PADDED, 0>(lv, colour, D, Dp, Gp, lam, lamT, skip, trace, blocks, grid, al, eager, dp,
                                       staged, bulk, st);
    }
}

template <typename CostT, typename MsgT>
static cudaError_t sweep_t(const LevelView &lv, int colour, int D, int Dp, int Gp, int lambda, int trunc, int skip,
                           unsigned long long *trace, cudaStream_t st) {
    using Acc = typename AccOf<MsgT>::type;
    static int resident = 0;  // CTAs of this kernel resident at once (looked up once per process)
    if (!resident) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_kernel<CostT, MsgT>, 256, 0);
        resident = std::max(1, sms * std::max(1, per_sm));
    }
    const int groups = 256 / Gp;
    const int64_t nslot = (int64_t)lv.H * lv.Wh;
    const int64_t blocks = (nslot + groups - 1) / groups;
    if (blocks == 0) return cudaSuccess;
    const unsigned grid = (unsigned)std::min<int64_t>(blocks, resident);
    return launch_k(sweep_kernel<CostT, MsgT>, dim3(grid), dim3(256), 0, st, lv, colour, D, Dp, Gp, (Acc)lambda,
                    (Acc)lambda * (Acc)trunc, skip, trace, (int)blocks);
}

// CTAs of the u8 sweep that fit on the GPU at once: the distance-transform or padded kernels, or
// the stencil kernels of D a multiple of 16 (looked up once per process).
static int resident_blocks(int ts, bool padded) {
    static int cached[2] = {0, 0};
    const int k = (ts == 0 || padded) ? 0 : 1;
    if (!cached[k]) {
        int dev = 0, sms = 0, per_sm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (k == 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_u8_kernel<false, false, 0, false>, 256, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, sweep_u8_kernel<false, false, 2, false>, 256, 0);
        cached[k] = std::max(1, sms * std::max(1, per_sm));
    }
    return cached[k];
}

cudaError_t launch_sweep(int msg_kind, const LevelView &lv, int colour, int D, int Dp, int Gp, int lambda, int trunc,
                         int skip, unsigned long long *trace, cudaStream_t st, const SweepLists &lists, int variant) {
    switch (msg_kind) {
    case MSG_I32: return sweep_t<int32_t, int32_t>(lv, colour, D, Dp, Gp, lambda, trunc, skip, trace, st);
    case MSG_U8: {
        // direction-parallel lanes (4 Gp a pixel) fit a warp up to Gp = 8: on every launch of
        // the scale, or on its list launches only (few pixels each)
        const bool list_launch = skip && lists.in;
        const bool dp = Gp <= 8 && ((variant & VARIANT_DPAR) || (list_launch && (variant & VARIANT_DPAR_LISTS)));
        const int groups = 256 / (dp ? 4 * Gp : Gp);
        const int64_t blocks = ((int64_t)lv.H * lv.Wh + groups - 1) / groups;
        if (blocks == 0) return cudaSuccess;
        const int lam = trunc == 0 ? 0 : lambda;  // with trunc 0 every message is 0 whatever lambda is
        const int ts = (variant & VARIANT_GENERAL_DT) ? 0 : (trunc <= 1 ? 1 : (trunc == 2 ? 2 : 0));
        const unsigned grid = (unsigned)std::min<int64_t>(blocks, resident_blocks(ts, (D & 15) != 0));
        const ActiveList al{lists.in, lists.n_in, skip ? lists.out : nullptr, lists.n_out};
        const bool eager = (variant & VARIANT_EAGER) != 0;
        const bool staged = (variant & (list_launch ? VARIANT_STAGED_LISTS : VARIANT_STAGED)) != 0 && !dp;
        const bool bulk = (variant & (list_launch ? VARIANT_BULK_LISTS : VARIANT_BULK)) != 0 && !dp;
        if (D & 15)
            return launch_u8<true>(ts, lv, colour, D, Dp, Gp, lam, lam * trunc, skip, trace, blocks, grid, al, eager, dp,
                                   staged, bulk, st);
        return launch_u8<false>(ts, lv, colour, D, Dp, Gp, lam, lam * trunc, skip, trace, blocks, grid, al, eager, dp,
                                staged, bulk, st);
    }
    default:
        // packed half2 arithmetic where the stencil forms apply (the GENERAL_DT variant keeps the
        // generic kernel)
        if (sweep_f16_applies(trunc) && !(variant & VARIANT_GENERAL_DT))
            return launch_sweep_f16(lv, colour, D, Dp, Gp, lambda, trunc, skip, trace, (variant & VARIANT_EAGER) != 0,
                                    lists, st);
        return sweep_t<float, __half>(lv, colour, D, Dp, Gp, lambda, trunc, skip, trace, st);
    }
}

// ------------------------------------------------------------------ coarse-to-fine start
// Fine pixel (x, y) of `colour` copies the whole message record of its parent
// (x >> 1, y >> 1) in 16-byte chunks.
__global__ void upsample_kernel(LevelView coarse, LevelView fine, int both_colours, int rec_chunks, int set_dirty) {
    pdl_enter();
    const int64_t n = (int64_t)fine.H * fine.Wh * rec_chunks;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int colour = 0; colour <= both_colours; ++colour)
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += stride)
            upsample_chunk(coarse, fine, colour, rec_chunks, k);
    if (set_dirty) {
        const int64_t m = (int64_t)fine.H * fine.Wh;
        for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < m; k += stride)
            fine.dirty[0][k] = fine.dirty[1][k] = 1;
    }
}

__global__ void solve_start_kernel(LevelView top, int rec_words, int zero_msgs, int set_dirty,
                                   unsigned long long *trace, unsigned *list_counts, int ntrace) {
    pdl_enter();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t slots = (int64_t)top.H * top.Wh;
    if (zero_msgs) {
        const int64_t n = slots * rec_words;  // 16-byte words of one colour's message array
        for (int64_t k = t0; k < n; k += stride) {
            reinterpret_cast<uint4 *>(top.msg[0])[k] = make_uint4(0u, 0u, 0u, 0u);
            reinterpret_cast<uint4 *>(top.msg[1])[k] = make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (set_dirty)
        for (int64_t k = t0; k < slots; k += stride) top.dirty[0][k] = top.dirty[1][k] = 1;
    for (int64_t k = t0; k < ntrace; k += stride) {
        trace[k] = 0ull;
        if (list_counts) list_counts[k] = 0u;
    }
}

static int msg_bytes(int msg_kind) { return msg_kind == MSG_I32 ? 4 : (msg_kind == MSG_U8 ? 1 : 2); }

static unsigned grid_for(int64_t n) { return (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 152 * 32)); }

cudaError_t launch_upsample(int msg_kind, const LevelView &coarse, const LevelView &fine, int both_colours, int Dp,
                            int set_dirty, cudaStream_t st) {
    const int rec_chunks = 4 * Dp * msg_bytes(msg_kind) / 16;
    const int64_t n = (int64_t)fine.H * fine.Wh * rec_chunks;
    return launch_k(upsample_kernel, dim3(grid_for(n)), dim3(256), 0, st, coarse, fine, both_colours, rec_chunks,
                    set_dirty);
}

cudaError_t launch_solve_start(int msg_kind, const LevelView &top, int Dp, int zero_msgs, int set_dirty,
                               unsigned long long *trace, unsigned *list_counts, int ntrace, cudaStream_t st) {
    const int rec_words = 4 * Dp * msg_bytes(msg_kind) / 16;
    const int64_t n = std::max<int64_t>((int64_t)top.H * top.Wh * (zero_msgs ? rec_words : 1), ntrace);
    return launch_k(solve_start_kernel, dim3(grid_for(n)), dim3(256), 0, st, top, rec_words, zero_msgs, set_dirty,
                    trace, list_counts, ntrace);
}

// ------------------------------------------------------------------ natural-layout import / export
template <typename MsgT> __device__ inline MsgT to_msg(int v);
template <> __device__ inline int32_t to_msg<int32_t>(int v) { return v; }
template <> __device__ inline uint8_t to_msg<uint8_t>(int v) { return (uint8_t)min(max(v, 0), 255); }
template <typename MsgT> __device__ inline MsgT to_msg_f(float v);
template <> __device__ inline __half to_msg_f<__half>(float v) { return __float2half_rn(v); }

template <typename MsgT, typename SrcT>
__global__ void import_kernel(LevelView lv, int D, int Dp, const SrcT *src) {
    pdl_enter();
    const int64_t n = 4LL * lv.H * lv.W * Dp;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(k % Dp);
        int64_t r = k / Dp;
        const int x = (int)(r % lv.W);
        r /= lv.W;
        const int y = (int)(r % lv.H);
        const int q = (int)(r / lv.H);
        const SrcT v = d < D ? src[(((int64_t)q * lv.H + y) * lv.W + x) * D + d] : SrcT(0);
        MsgT *dst = reinterpret_cast<MsgT *>(lv.msg[colour_of(x, y)]) + (slot_of(x, y, lv.Wh) * 4 + q) * Dp +
                    label_pos<MsgT>(d);
        if constexpr (sizeof(SrcT) == 4 && std::is_same<SrcT, float>::value)
            *dst = to_msg_f<MsgT>(v);
        else
            *dst = to_msg<MsgT>(v);
    }
}

template <typename MsgT, typename DstT>
__global__ void export_msgs_kernel(LevelView lv, int D, int Dp, DstT *out) {
    pdl_enter();
    const int64_t n = 4LL * lv.H * lv.W * D;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(k % D);
        int64_t r = k / D;
        const int x = (int)(r % lv.W);
        r /= lv.W;
        const int y = (int)(r % lv.H);
        const int q = (int)(r / lv.H);
        const bool has = q == DIR_UP ? y > 0 : q == DIR_DOWN ? y < lv.H - 1 : q == DIR_LEFT ? x > 0 : x < lv.W - 1;
        const MsgT *src = reinterpret_cast<const MsgT *>(lv.msg[colour_of(x, y)]) +
                          (slot_of(x, y, lv.Wh) * 4 + q) * Dp + label_pos<MsgT>(d);
        DstT v = DstT(0);
        if (has) {
            if constexpr (std::is_same<MsgT, __half>::value)
                v = (DstT)__half2float(*src);
            else
                v = (DstT)*src;
        }
        out[k] = v;
    }
}

template <typename CostT, typename DstT>
__global__ void export_cost_kernel(LevelView lv, int D, int Dp, DstT *out) {
    pdl_enter();
    const int64_t n = (int64_t)lv.H * lv.W * D;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const int d = (int)(k % D);
        const int64_t p = k / D;
        const int x = (int)(p % lv.W), y = (int)(p / lv.W);
        out[k] = (DstT) reinterpret_cast<const CostT *>(lv.cost[colour_of(x, y)])[slot_of(x, y, lv.Wh) * Dp +
                                                                                  label_pos<CostT>(d)];
    }
}

// The one-launch-per-half-sweep kernels need little shared memory (the list buffers, 8 KB a CTA):
// they ask for a carveout that leaves most of the SM's 256 KB to the L1 cache (spilled words,
// parent records read by two children), whatever the kernel before them needed (the tensor-core
// NCC takes 224 KB).  29 % of the 228 KB maximum is 66 KB: room for four CTAs' list buffers.
constexpr int SWEEP_CARVEOUT_PCT = 29;
template <typename K> static cudaError_t prefer_l1(K kernel) {
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, SWEEP_CARVEOUT_PCT);
}
template <bool PADDED, int TS, bool DP> static cudaError_t preload_u8_dp() {
    cudaError_t e = prefer_l1(sweep_u8_kernel<PADDED, false, TS, DP>);
    if (e == cudaSuccess) e = prefer_l1(sweep_u8_kernel<PADDED, true, TS, DP>);
    if (e == cudaSuccess) e = prefer_l1(sweep_u8_list_kernel<PADDED, TS, DP>);
    if (e == cudaSuccess) e = prefer_l1(sweep_u8_eager_kernel<PADDED, TS, DP>);
    return e;
}
template <bool PADDED, int TS> static cudaError_t preload_u8() {
    cudaError_t e = preload_u8_dp<PADDED, TS, false>();
    if (e == cudaSuccess) e = preload_u8_dp<PADDED, TS, true>();
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_u8_staged_kernel<PADDED, false, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)staged_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_u8_staged_kernel<PADDED, true, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)staged_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_u8_staged_list_kernel<PADDED, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)staged_smem_bytes());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_u8_bulk_kernel<PADDED, TS, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)BULK_SMEM_MAX);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_u8_bulk_kernel<PADDED, TS, false, true>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BULK_SMEM_MAX);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(sweep_u8_bulk_kernel<PADDED, TS, false, false>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BULK_SMEM_MAX);
    return e;
}

cudaError_t preload_bp_kernels(int msg_kind) {
    cudaFuncAttributes a;
    cudaError_t e = cudaFuncGetAttributes(&a, upsample_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, solve_start_kernel);
    if (e != cudaSuccess) return e;
    switch (msg_kind) {
    case MSG_I32:
        e = cudaFuncGetAttributes(&a, sweep_kernel<int32_t, int32_t>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, import_kernel<int32_t, int32_t>);
        break;
    case MSG_U8:
        e = preload_u8<false, 0>();
        if (e == cudaSuccess) e = preload_u8<false, 1>();
        if (e == cudaSuccess) e = preload_u8<false, 2>();
        if (e == cudaSuccess) e = preload_u8<true, 0>();
        if (e == cudaSuccess) e = preload_u8<true, 1>();
        if (e == cudaSuccess) e = preload_u8<true, 2>();
        if (e == cudaSuccess) resident_blocks(0, false);
        if (e == cudaSuccess) resident_blocks(2, false);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, import_kernel<uint8_t, int32_t>);
        break;
    default:
        e = cudaFuncGetAttributes(&a, sweep_kernel<float, __half>);
        if (e == cudaSuccess) e = cudaFuncGetAttributes(&a, import_kernel<__half, float>);
        break;
    }
    return e;
}

cudaError_t launch_import_msgs(int msg_kind, const LevelView &lv, int D, int Dp, const void *src, cudaStream_t st) {
    const unsigned g = grid_for(4LL * lv.H * lv.W * Dp);
    switch (msg_kind) {
    case MSG_I32: return launch_k(import_kernel<int32_t, int32_t>, dim3(g), dim3(256), 0, st, lv, D, Dp, (const int32_t *)src);
    case MSG_U8: return launch_k(import_kernel<uint8_t, int32_t>, dim3(g), dim3(256), 0, st, lv, D, Dp, (const int32_t *)src);
    default: return launch_k(import_kernel<__half, float>, dim3(g), dim3(256), 0, st, lv, D, Dp, (const float *)src);
    }
}

cudaError_t launch_export_msgs(int msg_kind, const LevelView &lv, int D, int Dp, void *dst, cudaStream_t st) {
    const unsigned g = grid_for(4LL * lv.H * lv.W * D);
    switch (msg_kind) {
    case MSG_I32: export_msgs_kernel<int32_t, int32_t><<<g, 256, 0, st>>>(lv, D, Dp, (int32_t *)dst); break;
    case MSG_U8: export_msgs_kernel<uint8_t, int32_t><<<g, 256, 0, st>>>(lv, D, Dp, (int32_t *)dst); break;
    default: export_msgs_kernel<__half, float><<<g, 256, 0, st>>>(lv, D, Dp, (float *)dst); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_export_cost(int cost_kind, const LevelView &lv, int D, int Dp, void *dst, cudaStream_t st) {
    const unsigned g = grid_for((int64_t)lv.H * lv.W * D);
    switch (cost_kind) {
    case COST_I32: export_cost_kernel<int32_t, int32_t><<<g, 256, 0, st>>>(lv, D, Dp, (int32_t *)dst); break;
    case COST_I16: export_cost_kernel<int16_t, int32_t><<<g, 256, 0, st>>>(lv, D, Dp, (int32_t *)dst); break;
    default: export_cost_kernel<float, float><<<g, 256, 0, st>>>(lv, D, Dp, (float *)dst); break;
    }
    return cudaGetLastError();
}

}  // namespace bps
