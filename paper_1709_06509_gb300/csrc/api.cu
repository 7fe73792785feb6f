// api.cu -- the C ABI (include/bpstereo.h): context, workspace plan, argument checks and
// the launch sequence of the hot path.  No exception crosses the boundary; every CUDA
// error becomes BPS_ERR_CUDA.
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/bpstereo.h"
#include "bps_launch.h"

using namespace bps;

namespace {

// Failure injection on the host (bps_test_fail_resources): the number of resource acquisitions
// of bps_create / bps_batch_create still allowed to succeed, -1 when no failure is planned.
std::atomic<int> g_fail_after{-1};

// Whether this acquisition is the one planned to fail (the plan is used up by it).
bool injected_failure() {
    int v = g_fail_after.load();
    while (v >= 0)
        if (g_fail_after.compare_exchange_weak(v, v - 1)) return v == 0;
    return false;
}
cudaError_t acquire_memory(void **p, size_t bytes) {
    return injected_failure() ? cudaErrorMemoryAllocation : cudaMalloc(p, bytes);
}
cudaError_t acquire_stream(cudaStream_t *s) {
    return injected_failure() ? cudaErrorMemoryAllocation : cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
}
cudaError_t acquire_event(cudaEvent_t *e) {
    return injected_failure() ? cudaErrorMemoryAllocation : cudaEventCreateWithFlags(e, cudaEventDisableTiming);
}

// Host-side ranges (NVTX) around the enqueued stages: visible in a timeline profiler, free otherwise.
struct Range {
    explicit Range(const char *name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

constexpr size_t ALIGN = 256;
inline size_t up(size_t v, size_t a = ALIGN) { return (v + a - 1) / a * a; }

struct Plan {
    int levels = 0;
    int Ws[BPS_MAX_LEVELS], Hs[BPS_MAX_LEVELS], Whs[BPS_MAX_LEVELS];
    size_t cost[BPS_MAX_LEVELS][2], msg[BPS_MAX_LEVELS][2], dirty[BPS_MAX_LEVELS][2];
    size_t trace, partials, img[2], disp, energy, desc, prefix, barrier, lists[2], list_counts, sparse[2], ncc_fix,
        ncc_fix_bytes, total;
};

int cost_kind_of(int msg_type) { return msg_type == BPS_MSG_INT32 ? COST_I32 : msg_type == BPS_MSG_U8 ? COST_I16 : COST_F32; }
int msg_kind_of(int msg_type) { return msg_type == BPS_MSG_INT32 ? MSG_I32 : msg_type == BPS_MSG_U8 ? MSG_U8 : MSG_F16; }
size_t cost_size(int msg_type) { return msg_type == BPS_MSG_U8 ? 2 : 4; }
size_t msg_size(int msg_type) { return msg_type == BPS_MSG_INT32 ? 4 : msg_type == BPS_MSG_U8 ? 1 : 2; }
int pad_labels(int D) { return (D + VEC - 1) / VEC * VEC; }

bool shape_ok(int W, int H, int D, int levels, int msg_type) {
    return W >= 1 && H >= 1 && D >= 1 && D <= BPS_MAX_D && levels >= 1 && levels <= BPS_MAX_LEVELS &&
           (msg_type == BPS_MSG_INT32 || msg_type == BPS_MSG_U8 || msg_type == BPS_MSG_FP16) &&
           (int64_t)W * H <= (int64_t)1 << 31;
}

bool make_plan(int W, int H, int D, int levels, int msg_type, Plan &p) {
    if (!shape_ok(W, H, D, levels, msg_type)) return false;
    const size_t Dp = (size_t)pad_labels(D);
    size_t off = 0;
    p.levels = levels;
    for (int l = 0; l < levels; ++l) {
        p.Ws[l] = l ? (p.Ws[l - 1] + 1) / 2 : W;
        p.Hs[l] = l ? (p.Hs[l - 1] + 1) / 2 : H;
        p.Whs[l] = (p.Ws[l] + 1) / 2;
        const size_t nslot = (size_t)p.Hs[l] * p.Whs[l];
        for (int c = 0; c < 2; ++c) {
            p.cost[l][c] = off;
            off += up(nslot * Dp * cost_size(msg_type));
            p.msg[l][c] = off;
            off += up(nslot * 4 * Dp * msg_size(msg_type));
            p.dirty[l][c] = off;
            off += up(nslot * sizeof(unsigned));
        }
    }
    p.trace = off;
    off += up((size_t)levels * BPS_MAX_ITERS * 2 * sizeof(unsigned long long));
    p.partials = off;
    off += up(1024 * 8);
    p.img[0] = off;
    off += up((size_t)W * H);
    p.img[1] = off;
    off += up((size_t)W * H);
    p.disp = off;
    off += up((size_t)W * H * 4);
    p.energy = off;
    off += up(16);
    p.desc = off;
    off += up(sizeof(PairDesc));
    p.prefix = off;
    off += up(sizeof(int) * 2 * (levels + 1));
    p.barrier = off;
    off += up(16);
    // active lists of the two colours (sized for the finest scale, reused at every scale) and
    // one entry count per half-sweep
    for (int c = 0; c < 2; ++c) {
        p.lists[c] = off;
        off += up((size_t)p.Hs[0] * p.Whs[0] * sizeof(unsigned));
    }
    p.list_counts = off;
    off += up((size_t)levels * BPS_MAX_ITERS * 2 * sizeof(unsigned));
    // sparse candidates of the finest scale (u8 form): labels then costs, BPS_MAX_CANDIDATES a slot
    for (int c = 0; c < 2; ++c) {
        p.sparse[c] = off;
        if (msg_type == BPS_MSG_U8) off += up((size_t)p.Hs[0] * p.Whs[0] * BPS_MAX_CANDIDATES * 4);
    }
    // values the tensor-core NCC leaves to its FP64 pass (integer forms)
    p.ncc_fix = off;
    p.ncc_fix_bytes = msg_type == BPS_MSG_FP16 ? 0 : ncc_tc_fix_bytes(W, H, (int)Dp);
    off += up(p.ncc_fix_bytes);
    p.total = off;
    return true;
}

// Iterations per scale of a solve (0 = the finest scale).
struct Iters {
    int n[BPS_MAX_LEVELS] = {};
    static Iters uniform(int levels, int iters) {
        Iters it;
        for (int l = 0; l < levels; ++l) it.n[l] = iters;
        return it;
    }
    int trace_len(int levels) const {  // half-sweeps of the solve
        int t = 0;
        for (int l = 0; l < levels; ++l) t += 2 * n[l];
        return t;
    }
    bool uniform_over(int levels) const {
        for (int l = 1; l < levels; ++l)
            if (n[l] != n[0]) return false;
        return true;
    }
};

struct GraphKey {
    const void *L, *R;
    int32_t *disp;
    int pitch, window, trunc_data, iters, lambda, trunc, flags;
    bool operator==(const GraphKey &o) const { return std::memcmp(this, &o, sizeof(GraphKey)) == 0; }
};

// Page-locked host memory (registered or allocated pinned): copies from and to it can be
// recorded in a CUDA graph.
bool is_pinned(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// A recorded graph keyed by the arguments that shaped it: replayed while the key holds,
// recorded again (on the capture stream `cap`) when it changes.
struct GraphSlot {
    cudaGraphExec_t exec = nullptr;
    std::vector<intptr_t> key;
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};

template <typename Enqueue>
int replay_or_record(GraphSlot &g, const std::vector<intptr_t> &key, cudaStream_t cap, cudaStream_t st,
                     Enqueue enqueue) {
    if (!g.exec || key != g.key) {
        g.reset();
        if (cudaStreamSynchronize(cap) != cudaSuccess) return BPS_ERR_CUDA;
        if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return BPS_ERR_CUDA;
        const int rc = enqueue(cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(cap, &graph);
        if (rc != BPS_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != BPS_OK ? rc : BPS_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            g.exec = nullptr;
            return BPS_ERR_CUDA;
        }
        g.key = key;
    }
    return cudaGraphLaunch(g.exec, st) == cudaSuccess ? BPS_OK : BPS_ERR_CUDA;
}

}  // namespace

struct bps_ctx {
    int W, H, D, Dp, Gp, levels, msg_type, cost_kind, msg_kind;
    Plan plan;
    LevelView lv[BPS_MAX_LEVELS];
    char *ws = nullptr;
    bool owns_ws = false;
    unsigned long long *trace = nullptr;
    void *partials = nullptr;
    uint8_t *img[2] = {nullptr, nullptr};
    int32_t *disp = nullptr;
    int64_t *e_i64 = nullptr;
    double *e_f64 = nullptr;
    bool has_cost = false;
    int last_levels = 0, last_trace_n = 0;  // scales and half-sweeps of the last solve
    cudaStream_t cap = nullptr;
    cudaGraphExec_t gexec = nullptr;
    GraphKey gkey;
    std::vector<cudaEvent_t> ev;
    PairDesc *d_desc = nullptr;      // this context as a batch of one (device)
    int *d_prefix = nullptr;         // [levels][2] sweep block prefix, then [2] read-out prefix
    unsigned *d_barrier = nullptr;   // {arrival count, error word} of the persistent kernel
    int grid = 0;                    // co-resident CTAs of the persistent kernel
    unsigned *lists[2] = {nullptr, nullptr};  // active lists of the even / odd pixels
    unsigned *list_counts = nullptr;          // entries appended during each half-sweep
    int variant[BPS_MAX_LEVELS] = {};         // u8 sweep kernel variant per scale
    int ncc_xs = 0, ncc_rows = 0;             // NCC CTA shape (0: default)
    int ncc_kernel = BPS_NCC_DEFAULT, ncc_tc_rows = 0;  // NCC kernel choice, tensor-core rows per strip
    void *ncc_fix = nullptr;                  // the tensor-core NCC's list for its FP64 pass
    size_t ncc_fix_bytes = 0;
    int prof_launches = 0;  // finest-scale sweep launches of the last profiled solve
    int prof_all = 0;       // all sweep launches of the last profiled solve
    int prof_first_trace = 0;
    int prof_trace_n = 0;   // trace entries covered by the profiled launches
    uint64_t config_version = 0;  // bumped when a kernel choice (variant, NCC shape) changes
    SparseView sv{};              // sparse candidates of the finest scale (K = 0: dense)
    int last_sparse_k = 0;        // K of the last solve (0: dense)
    GraphSlot host_graph;         // bps_stereo_host: copies in, pipeline, energy, copies out
    GraphSlot solve_graph;        // bps_bp_solve with BPS_FLAG_GRAPH
    std::vector<int> prof_span;  // half-sweeps each profiled launch covers (a cluster launch covers a scale)
};

namespace {

int sweep_blocks(const bps_ctx *c, int l) {
    const int groups = 256 / c->Gp;
    return (int)(((int64_t)c->plan.Hs[l] * c->plan.Whs[l] + groups - 1) / groups);
}

int wta_blocks(const bps_ctx *c) {
    const int groups = 256 / c->Gp;
    return (int)(((int64_t)c->W * c->H + groups - 1) / groups);
}

PairDesc make_desc(const bps_ctx *c) {
    PairDesc d;
    std::memset(&d, 0, sizeof(d));
    for (int l = 0; l < c->levels; ++l) d.lv[l] = c->lv[l];
    d.D = c->D;
    d.Dp = c->Dp;
    d.Gp = c->Gp;
    d.trace = c->trace;
    d.disp = nullptr;
    d.lists[0] = c->lists[0];
    d.lists[1] = c->lists[1];
    d.list_counts = c->list_counts;
    return d;
}

// Defaults of the per-scale sweep variant, from measurements on GB300 (the autotuner may
// replace them): active lists pay off from about 128 K pixels of a colour, and there the u8
// form's staged launches (dense and list) beat the plain ones (960x540 and 1920x1080 at 256
// labels: 1.53 ms against 1.79 ms, and 4.15 ms against 5.50 ms, for the finest scale's 20
// half-sweeps); the stencil forms stay ahead of the distance transform at every size.
int default_variant(int64_t slots, int Gp, int msg_kind) {
    int v = 0;
    if (slots >= 128 * 1024) v |= VARIANT_LISTS | (msg_kind == MSG_U8 ? VARIANT_STAGED | VARIANT_STAGED_LISTS : 0);
    // a scale of at most four passes of a 16 x 512-thread cluster runs as one cluster launch
    if (slots * Gp <= 4 * 16 * 512 && cluster_sweep_available()) v |= VARIANT_CLUSTER;
    return v;
}

// Whether a half-sweep of this form and variant builds and reads active lists: the u8 form's
// kernels and the fp16 form's packed one do; the generic kernels sweep densely.
bool sweep_takes_lists(int msg_kind, int variant, int trunc) {
    return msg_kind == MSG_U8 ||
           (msg_kind == MSG_F16 && sweep_f16_applies(trunc) && !(variant & VARIANT_GENERAL_DT));
}

constexpr unsigned long long BARRIER_TIMEOUT_NS = 4000000000ull;  // 4 s: far above any phase
constexpr unsigned long long TEST_TIMEOUT_NS = 2000000ull;        // 2 ms, for BPS_FLAG_TEST_TIMEOUT

}  // namespace

// The CUDA error behind the last BPS_ERR_CUDA of this thread (see bps_last_cuda_error).
static thread_local int g_last_cuda_error = 0;

static int cuda_failed(cudaError_t e) {
    g_last_cuda_error = (int)e;
    cudaGetLastError();  // clear a sticky launch error so the context stays usable
    return BPS_ERR_CUDA;
}

#define CK(x)                                          \
    do {                                               \
        const cudaError_t ck_e_ = (x);                 \
        if (ck_e_ != cudaSuccess) return cuda_failed(ck_e_); \
    } while (0)

extern "C" int bps_last_cuda_error(void) { return g_last_cuda_error; }

extern "C" const char *bps_cuda_error_string(int code) { return cudaGetErrorString((cudaError_t)code); }

extern "C" const char *bps_status_string(int s) {
    switch (s) {
    case BPS_OK: return "ok";
    case BPS_ERR_ARG: return "invalid argument";
    case BPS_ERR_UNSUPPORTED: return "unsupported by this build";
    case BPS_ERR_CUDA: return "CUDA error";
    case BPS_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case BPS_ERR_TIMEOUT: return "bounded device wait gave up";
    case BPS_ERR_STATE: return "call order violated";
    case BPS_ERR_INTERNAL: return "a device-side consistency check failed";
    default: return "unknown status";
    }
}

extern "C" size_t bps_workspace_bytes(int W, int H, int D, int levels, int msg_type) {
    Plan p;
    return make_plan(W, H, D, levels, msg_type, p) ? p.total : 0;
}

extern "C" int bps_create(bps_ctx **out, int W, int H, int D, int levels, int msg_type, void *d_workspace,
                          size_t workspace_bytes) {
    if (!out) return BPS_ERR_ARG;
    *out = nullptr;
    Plan p;
    if (!make_plan(W, H, D, levels, msg_type, p)) return BPS_ERR_ARG;
    if (d_workspace && (workspace_bytes < p.total || ((uintptr_t)d_workspace % ALIGN) != 0)) return BPS_ERR_WORKSPACE;
    bps_ctx *c = new (std::nothrow) bps_ctx();
    if (!c) return BPS_ERR_CUDA;
    c->W = W;
    c->H = H;
    c->D = D;
    c->Dp = pad_labels(D);
    int G = c->Dp / VEC, Gp = 1;
    while (Gp < G) Gp <<= 1;
    c->Gp = Gp;
    c->levels = levels;
    c->msg_type = msg_type;
    c->cost_kind = cost_kind_of(msg_type);
    c->msg_kind = msg_kind_of(msg_type);
    c->plan = p;
    if (d_workspace) {
        c->ws = static_cast<char *>(d_workspace);
    } else {
        if (acquire_memory(reinterpret_cast<void **>(&c->ws), p.total) != cudaSuccess) {
            delete c;
            return BPS_ERR_CUDA;
        }
        c->owns_ws = true;
    }
    for (int l = 0; l < levels; ++l) {
        LevelView &v = c->lv[l];
        v.W = p.Ws[l];
        v.H = p.Hs[l];
        v.Wh = p.Whs[l];
        v.eps = 0;  // the exact skip rule
        v.freeze = 0;
        v.bsum8 = 0;
        v.keep_flag = 0;
        v.start = 0;
        v.pWh = 0;
        v.pmsg[0] = v.pmsg[1] = nullptr;
        v.disp = nullptr;
        v.err = nullptr;  // set below, once the workspace is laid out
        for (int k = 0; k < 2; ++k) {
            v.cost[k] = c->ws + p.cost[l][k];
            v.msg[k] = c->ws + p.msg[l][k];
            v.dirty[k] = reinterpret_cast<unsigned *>(c->ws + p.dirty[l][k]);
        }
    }
    c->trace = reinterpret_cast<unsigned long long *>(c->ws + p.trace);
    c->partials = c->ws + p.partials;
    c->img[0] = reinterpret_cast<uint8_t *>(c->ws + p.img[0]);
    c->img[1] = reinterpret_cast<uint8_t *>(c->ws + p.img[1]);
    c->disp = reinterpret_cast<int32_t *>(c->ws + p.disp);
    c->e_i64 = reinterpret_cast<int64_t *>(c->ws + p.energy);
    c->e_f64 = reinterpret_cast<double *>(c->ws + p.energy + 8);
    c->d_desc = reinterpret_cast<PairDesc *>(c->ws + p.desc);
    c->d_prefix = reinterpret_cast<int *>(c->ws + p.prefix);
    c->d_barrier = reinterpret_cast<unsigned *>(c->ws + p.barrier);
    // words of the barrier area: arrivals and error of the persistent kernel, then the error word
    // of the bounded waits of the chained sweeps
    for (int l = 0; l < levels; ++l) c->lv[l].err = c->d_barrier + 2;
    c->lists[0] = reinterpret_cast<unsigned *>(c->ws + p.lists[0]);
    c->lists[1] = reinterpret_cast<unsigned *>(c->ws + p.lists[1]);
    c->list_counts = reinterpret_cast<unsigned *>(c->ws + p.list_counts);
    c->ncc_fix = p.ncc_fix_bytes ? c->ws + p.ncc_fix : nullptr;
    c->ncc_fix_bytes = p.ncc_fix_bytes;
    c->sv.cand[0] = reinterpret_cast<uint16_t *>(c->ws + p.sparse[0]);
    c->sv.cand[1] = reinterpret_cast<uint16_t *>(c->ws + p.sparse[1]);
    c->sv.K = c->sv.Kp = 0;
    for (int l = 0; l < levels; ++l) c->variant[l] = default_variant((int64_t)p.Hs[l] * p.Whs[l], c->Gp, c->msg_kind);
    PairDesc hd = make_desc(c);
    std::vector<int> prefix(2 * (levels + 1));
    for (int l = 0; l < levels; ++l) {
        prefix[2 * l] = 0;
        prefix[2 * l + 1] = sweep_blocks(c, l);
    }
    prefix[2 * levels] = 0;
    prefix[2 * levels + 1] = wta_blocks(c);
    bool ok = acquire_stream(&c->cap) == cudaSuccess;
    // every persistent kernel (one per minimisation form) is loaded and sized now, outside any capture
    for (int T = 1; ok && T <= 3; ++T) ok = persistent_grid(c->msg_kind, T, &c->grid) == cudaSuccess;
    // the NCC kernel's shared memory depends on D and the window; allow the largest window now so
    // that no attribute call happens while a launch sequence is being captured
    ok = ok && ncc_prepare(c->cost_kind, D, BPS_MAX_WINDOW) == cudaSuccess;
    ok = ok && ncc_rows_prepare(c->cost_kind, D, c->Dp) == cudaSuccess;
    ok = ok && ncc_tc_prepare(c->cost_kind, c->Dp) == cudaSuccess;
    ok = ok && preload_cost_kernels(c->cost_kind) == cudaSuccess;
    ok = ok && preload_bp_kernels(c->msg_kind) == cudaSuccess;
    ok = ok && (c->msg_kind != MSG_U8 || preload_sparse_kernels() == cudaSuccess);
    ok = ok && (c->msg_kind != MSG_F16 || preload_f16_kernels() == cudaSuccess);
    ok = ok && preload_readout_kernels(c->msg_kind) == cudaSuccess;
    ok = ok && cudaMemsetAsync(c->ws, 0, p.total, c->cap) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(c->d_desc, &hd, sizeof(hd), cudaMemcpyHostToDevice, c->cap) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(c->d_prefix, prefix.data(), sizeof(int) * prefix.size(), cudaMemcpyHostToDevice,
                               c->cap) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(c->cap) == cudaSuccess;
    if (!ok) {
        bps_destroy(c);
        return BPS_ERR_CUDA;
    }
    *out = c;
    return BPS_OK;
}

extern "C" int bps_destroy(bps_ctx *c) {
    if (!c) return BPS_OK;
    int rc = BPS_OK;
    if (c->cap && cudaStreamSynchronize(c->cap) != cudaSuccess) rc = BPS_ERR_CUDA;
    if (c->gexec) cudaGraphExecDestroy(c->gexec);
    c->host_graph.reset();
    c->solve_graph.reset();
    for (cudaEvent_t e : c->ev) cudaEventDestroy(e);
    if (c->cap) cudaStreamDestroy(c->cap);
    // cudaFree waits for the work in flight on the device before it releases the memory
    if (c->owns_ws && c->ws && cudaFree(c->ws) != cudaSuccess) rc = BPS_ERR_CUDA;
    delete c;
    return rc;
}

static int check_cost_args(bps_ctx *c, const uint8_t *L, const uint8_t *R, int pitch, int window, int trunc_data) {
    if (!c || !L || !R || pitch < c->W || window < 1 || (window & 1) == 0 || window > BPS_MAX_WINDOW ||
        trunc_data < 0 || trunc_data > 65535)
        return BPS_ERR_ARG;
    if (c->msg_type == BPS_MSG_U8) {
        int64_t top = trunc_data;
        for (int l = 1; l < c->levels; ++l) top *= 4;
        if (top > 27000) return BPS_ERR_UNSUPPORTED;  // keeps every belief below 2^15 (packed 16-bit sweep)
    }
    if (c->msg_type == BPS_MSG_INT32) {
        int64_t top = trunc_data;
        for (int l = 1; l < c->levels; ++l) top *= 4;
        if (top >= (1 << 24)) return BPS_ERR_UNSUPPORTED;
    }
    return BPS_OK;
}

static int enqueue_cost(bps_ctx *c, const uint8_t *L, const uint8_t *R, int pitch, int window, int trunc_data,
                        float *ncc_out, cudaStream_t st) {
    Range range("bps cost volume");
    const LevelView &v0 = c->lv[0];
    int first_pyramid = 1;
    const bool tc = c->ncc_kernel != BPS_NCC_ROWS && !ncc_out &&
                    ncc_tc_supported(c->cost_kind, c->Dp, window, trunc_data);
    if (tc) {
        // the tensor-core kernel (integer forms) writes scale 1 as well
        const bool fuse = c->levels > 1;
        CK(launch_ncc_tc(c->cost_kind, L, R, pitch, c->W, c->H, c->D, c->Dp, window, trunc_data, v0,
                         fuse ? &c->lv[1] : nullptr, st, c->ncc_tc_rows, c->ncc_fix, c->ncc_fix_bytes));
        if (fuse) first_pyramid = 2;
    } else if (window <= NCC_ROWS_MAX_WINDOW) {
        // the row-streaming kernel also writes scale 1 in the integer forms
        const bool fuse = c->levels > 1 && c->cost_kind != COST_F32;
        CK(launch_ncc_rows(c->cost_kind, L, R, pitch, c->W, c->H, c->D, c->Dp, window, trunc_data, v0,
                           fuse ? &c->lv[1] : nullptr, ncc_out, st, c->ncc_xs, c->ncc_rows));
        if (fuse) first_pyramid = 2;
    } else {
        CK(launch_ncc(c->cost_kind, L, R, pitch, c->W, c->H, c->D, c->Dp, window, trunc_data, v0.Wh, v0.cost[0],
                      v0.cost[1], ncc_out, st));
    }
    // two scales a launch, then a last single one
    int l = first_pyramid;
    for (; l + 1 < c->levels; l += 2)
        CK(launch_pyramid2(c->cost_kind, c->lv[l - 1], c->lv[l], c->lv[l + 1], c->Dp, st));
    if (l < c->levels) CK(launch_pyramid(c->cost_kind, c->lv[l - 1], c->lv[l], c->Dp, st));
    return BPS_OK;
}

extern "C" int bps_build_cost_volume(bps_ctx *c, const uint8_t *L, const uint8_t *R, int pitch, int window,
                                     int trunc_data, float *ncc_out, void *stream) {
    const int rc = check_cost_args(c, L, R, pitch, window, trunc_data);
    if (rc != BPS_OK) return rc;
    const int e = enqueue_cost(c, L, R, pitch, window, trunc_data, ncc_out, (cudaStream_t)stream);
    if (e == BPS_OK) c->has_cost = true;
    return e;
}

static int check_bp_args(bps_ctx *c, int levels, int iters, int lambda, int trunc, int flags, const void *init) {
    if (!c) return BPS_ERR_ARG;
    if (!c->has_cost) return BPS_ERR_STATE;
    if (levels < 1 || levels > c->levels || iters < 0 || iters > BPS_MAX_ITERS || lambda < 0 || trunc < 0 ||
        (flags & ~(BPS_FLAG_FAST_SKIP | BPS_FLAG_WARM_START | BPS_FLAG_GRAPH | BPS_FLAG_PROFILE |
                   BPS_FLAG_PERSISTENT | BPS_FLAG_TEST_TIMEOUT)) ||
        (int64_t)lambda * ((int64_t)c->Dp + trunc) >= ((int64_t)1 << 24) ||
        ((flags & BPS_FLAG_WARM_START) && !init))
        return BPS_ERR_ARG;
    if (c->msg_type == BPS_MSG_U8 && (int64_t)lambda * trunc > 255) return BPS_ERR_UNSUPPORTED;
    // sparse candidates: chained launches only; a warm start needs a dense coarser scale
    if (c->sv.K > 0 && ((flags & BPS_FLAG_PERSISTENT) || ((flags & BPS_FLAG_WARM_START) && levels == 1)))
        return BPS_ERR_UNSUPPORTED;
    return BPS_OK;
}

static int enqueue_bp_sweeps(bps_ctx *c, int levels, const Iters &its, int lambda, int trunc, int flags,
                             const void *init, cudaStream_t st, int32_t *readout = nullptr);

// The start messages of the coarsest scale: zero, or imported from the caller.
static int enqueue_start(bps_ctx *c, int top, int flags, const void *init, cudaStream_t st) {
    const LevelView &v = c->lv[top];
    if (flags & BPS_FLAG_WARM_START) {
        CK(launch_import_msgs(c->msg_kind, v, c->D, c->Dp, init, st));
    } else {
        for (int k = 0; k < 2; ++k)
            CK(cudaMemsetAsync(v.msg[k], 0, (size_t)v.H * v.Wh * 4 * c->Dp * msg_size(c->msg_type), st));
    }
    return BPS_OK;
}

static PersistParams persist_params(int npairs, const PairDesc *pairs, const int *sweep_prefix, const int *wta_prefix,
                                    unsigned *barrier, int levels, int iters, int lambda, int trunc, int flags) {
    PersistParams P;
    std::memset(&P, 0, sizeof(P));
    P.pairs = pairs;
    P.sweep_prefix = sweep_prefix;
    P.wta_prefix = wta_prefix;
    P.npairs = npairs;
    P.levels = levels;
    P.iters = iters;
    P.lam = lambda;
    P.lam_u8 = trunc == 0 ? 0 : lambda;  // with trunc 0 every message is 0 whatever lambda is
    P.trunc = trunc;
    P.skip = (flags & BPS_FLAG_FAST_SKIP) ? 1 : 0;
    P.barrier = barrier;
    P.extra_arrivals = (flags & BPS_FLAG_TEST_TIMEOUT) ? 1u : 0u;
    P.timeout_ns = (flags & BPS_FLAG_TEST_TIMEOUT) ? TEST_TIMEOUT_NS : BARRIER_TIMEOUT_NS;
    return P;
}

// The whole solve (and the read-out into disp when it is not NULL) as one persistent launch.
static int enqueue_bp(bps_ctx *c, int levels, const Iters &its, int lambda, int trunc, int flags, const void *init,
                      cudaStream_t st, int32_t *disp = nullptr) {
    if (!(flags & BPS_FLAG_PERSISTENT)) {
        // u8 form, exact skip rule: the finest scale's half-sweeps read out every pixel they
        // recompute, and only the even pixels the last half-sweep dirtied are read out after it
        const bool skip = (flags & BPS_FLAG_FAST_SKIP) != 0;
        // (the fp16 form where its packed sweep runs the finest scale, which forms the same belief)
        const bool packed_f16 = c->msg_kind == MSG_F16 && sweep_f16_applies(trunc) &&
                                !(c->variant[0] & VARIANT_GENERAL_DT);
        const bool fused = disp && (c->msg_kind == MSG_U8 || packed_f16) && c->sv.K == 0 && c->lv[0].eps == 0 &&
                           !c->lv[0].freeze && its.n[0] > 0;
        const int rc = enqueue_bp_sweeps(c, levels, its, lambda, trunc, flags, init, st, fused ? disp : nullptr);
        if (rc == BPS_OK && disp) {
            if (c->last_sparse_k) {
                CK(launch_sparse_wta(c->lv[0], c->sv, disp, st));
            } else if (fused) {
                // the last half-sweep's list of newly dirty even pixels, where the scale keeps lists
                const bool listed = skip && (c->variant[0] & VARIANT_LISTS) &&
                                    !(c->msg_kind == MSG_U8 && (c->variant[0] & VARIANT_CLUSTER));
                const int t_last = its.trace_len(levels) - 1;
                CK(launch_wta_rest(c->msg_kind, c->lv[0], c->D, c->Dp, c->Gp, skip ? 1 : 0,
                                   listed ? c->lists[0] : nullptr,
                                   listed ? c->list_counts + t_last : nullptr, disp, st));
            } else {
                CK(launch_wta(c->msg_kind, c->lv[0], c->D, c->Dp, c->Gp, disp, st));
            }
        }
        return rc;
    }
    const int top = levels - 1;
    const int iters = its.n[0];  // the persistent kernel runs the same count at every scale
    if (!its.uniform_over(levels)) return BPS_ERR_UNSUPPORTED;
    const int ntrace = levels * iters * 2;
    c->last_sparse_k = 0;
    if (ntrace) {
        CK(cudaMemsetAsync(c->trace, 0, sizeof(unsigned long long) * ntrace, st));
        CK(cudaMemsetAsync(c->list_counts, 0, sizeof(unsigned) * ntrace, st));
    }
    const int rc = enqueue_start(c, top, flags, init, st);
    if (rc != BPS_OK) return rc;
    CK(cudaMemsetAsync(c->d_barrier, 0, 2 * sizeof(unsigned), st));
    // a batch of one: the read-out target is patched into a private descriptor copy only when it
    // changes, so a captured graph keeps pointing at valid data
    PersistParams P = persist_params(1, c->d_desc, c->d_prefix, c->d_prefix + 2 * c->levels, c->d_barrier, levels,
                                     iters, lambda, trunc, flags);
    P.disp_override = disp;
    const bool prof = (flags & BPS_FLAG_PROFILE) != 0;
    if (prof) {
        while (c->ev.size() < 2) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->ev.push_back(e);
        }
        CK(cudaEventRecord(c->ev[0], st));
    }
    CK(launch_persistent(c->msg_kind, P, st));
    if (prof) {
        CK(cudaEventRecord(c->ev[1], st));
        c->prof_span.assign(1, 1);
        c->prof_all = 1;
        c->prof_launches = 1;
        c->prof_first_trace = 0;
        c->prof_trace_n = ntrace;
    }
    c->last_levels = levels;
    c->last_trace_n = ntrace;
    return BPS_OK;
}

static int enqueue_bp_sweeps(bps_ctx *c, int levels, const Iters &its, int lambda, int trunc, int flags,
                             const void *init, cudaStream_t st, int32_t *readout) {
    const bool skip = (flags & BPS_FLAG_FAST_SKIP) != 0;
    const bool prof = (flags & BPS_FLAG_PROFILE) != 0;
    const int top = levels - 1;
    const int ntrace = its.trace_len(levels);
    if (prof) {
        const size_t need = 2 * (size_t)ntrace;
        c->prof_span.assign((size_t)ntrace + 1, 1);
        while (c->ev.size() < need) {
            cudaEvent_t e;
            CK(cudaEventCreate(&e));
            c->ev.push_back(e);
        }
        c->prof_launches = 0;
        c->prof_all = 0;
        c->prof_first_trace = ntrace - 2 * its.n[0];
        c->prof_trace_n = 2 * its.n[0];
    }
    // a chain of kernels only (no memset nodes), so that every launch overlaps its predecessor
    const bool warm = (flags & BPS_FLAG_WARM_START) != 0;
    if (warm) CK(launch_import_msgs(c->msg_kind, c->lv[top], c->D, c->Dp, init, st));
    CK(launch_solve_start(c->msg_kind, c->lv[top], c->Dp, warm ? 0 : 1, skip ? 1 : 0, c->trace, c->list_counts, ntrace,
                          st));
    // u8 form with the skip, on scales whose variant asks for it (large, bandwidth-bound ones by
    // default): after a scale's first iteration each half-sweep runs over the active list its
    // predecessor built (entry count list_counts[t - 1]).  Small scales are latency-bound and
    // keep the dense launch, whose clean warps exit after one flag load.
    int t = 0;
    c->last_sparse_k = c->sv.K;
    static const char *scale_names[BPS_MAX_LEVELS] = {"bps scale 0", "bps scale 1", "bps scale 2", "bps scale 3",
                                                      "bps scale 4", "bps scale 5", "bps scale 6", "bps scale 7"};
    for (int l = top; l >= 0; --l) {
        Range range(scale_names[l]);
        const int iters = its.n[l];
        LevelView v = c->lv[l];
        if (l == 0) v.disp = readout;  // the finest scale's half-sweeps read out what they recompute
        // every message the sweeps read is one they wrote, normalised to [0, lambda * trunc], or a
        // zero start message, unless the caller gave the start messages
        v.bsum8 = (!warm && (int64_t)lambda * trunc <= 63) ? 1 : 0;
        if (l == 0 && c->sv.K > 0) {
            // the finest scale over sparse candidates: selection, start from the parent's messages
            // at each candidate's label, then the half-sweeps
            CK(launch_sparse_candidates(v, c->sv, c->D, c->Dp, c->Gp, st));
            CK(launch_sparse_start(v, top > 0 ? &c->lv[1] : nullptr, c->sv, c->Dp, st));
            for (int it = 0; it < iters; ++it)
                for (int colour = 0; colour < 2; ++colour, ++t) {
                    if (prof) CK(cudaEventRecord(c->ev[2 * c->prof_all], st));
                    CK(launch_sparse_sweep(v, c->sv, colour, lambda, trunc, skip ? 1 : 0, c->trace + t, st));
                    if (prof) {
                        CK(cudaEventRecord(c->ev[2 * c->prof_all + 1], st));
                        c->prof_span[c->prof_all] = 1;
                        ++c->prof_all;
                        ++c->prof_launches;
                    }
                }
            continue;
        }
        // only the even pixels' start messages are ever read: the first half-sweep overwrites every
        // existing incoming slot of the odd pixels (unless there is no sweep at all)
        // the odd pixels' start messages are read only without sweeps, or under the freeze rule
        // (its first half-sweep compares the even pixels' new messages with them).
        // u8 form: the first iteration reads the parent's records itself and recomputes every
        // pixel (the skip flags need no setting), so no copy is launched, except under the freeze
        // rule or for a one-launch (cluster) scale
        const bool fused_start = l < top && iters > 0 && c->msg_kind == MSG_U8 && !v.freeze &&
                                 !(c->variant[l] & VARIANT_CLUSTER);
        if (l < top && !fused_start)
            CK(launch_upsample(c->msg_kind, c->lv[l + 1], v, (iters == 0 || v.freeze) ? 1 : 0, c->Dp, skip ? 1 : 0,
                               st));
        LevelView first = v, second = v;  // the views of the scale's first two half-sweeps
        if (fused_start) {
            // the first half-sweep reads the even pixels' start messages from their parents'
            // records; the second compares its messages with the odd pixels' receivers' start
            // messages there (the receivers' own records are written whole only then)
            first.start = 1;
            second.start = 2;
            for (LevelView *fs : {&first, &second}) {
                fs->pWh = c->lv[l + 1].Wh;
                fs->pmsg[0] = c->lv[l + 1].msg[0];
                fs->pmsg[1] = c->lv[l + 1].msg[1];
            }
        }
        if (iters > 0 && c->msg_kind == MSG_U8 && (c->variant[l] & VARIANT_CLUSTER)) {
            if (prof) CK(cudaEventRecord(c->ev[2 * c->prof_all], st));
            CK(launch_sweep_level_cluster(v, c->D, c->Dp, c->Gp, lambda, trunc, skip, c->trace + t, iters,
                                          c->variant[l], st));
            if (prof) {
                CK(cudaEventRecord(c->ev[2 * c->prof_all + 1], st));
                c->prof_span[c->prof_all] = 2 * iters;
                ++c->prof_all;
                if (l == 0) c->prof_launches += 2 * iters;
            }
            t += 2 * iters;
            continue;
        }
        // the first iteration temporally blocked: both half-sweeps in one launch (u8, fused start, skip)
        const bool block2 = fused_start && skip && (c->variant[l] & VARIANT_BLOCK2);
        for (int it = 0; it < iters; ++it) {
            if (it == 0 && block2) {
                if (prof) CK(cudaEventRecord(c->ev[2 * c->prof_all], st));
                SweepLists sl{nullptr, nullptr, nullptr, nullptr};
                if ((c->variant[l] & VARIANT_LISTS) && sweep_takes_lists(c->msg_kind, c->variant[l], trunc)) {
                    sl.out = c->lists[0];  // the even pixels the second half marks, for the next iteration
                    sl.n_out = c->list_counts + t + 1;
                }
                LevelView a = first;
                a.keep_flag = 1;  // the even flags are cleared before the launch and only marked in it
                CK(launch_sweep_block2(a, second, c->D, c->Dp, c->Gp, lambda, trunc, c->trace + t, c->trace + t + 1,
                                       sl, st));
                if (prof) {
                    CK(cudaEventRecord(c->ev[2 * c->prof_all + 1], st));
                    c->prof_span[c->prof_all] = 2;
                    ++c->prof_all;
                    if (l == 0) c->prof_launches += 2;
                }
                t += 2;
                continue;
            }
            for (int colour = 0; colour < 2; ++colour, ++t) {
                if (prof) CK(cudaEventRecord(c->ev[2 * c->prof_all], st));
                SweepLists sl{nullptr, nullptr, nullptr, nullptr};
                const bool lists =
                    skip && (c->variant[l] & VARIANT_LISTS) && sweep_takes_lists(c->msg_kind, c->variant[l], trunc);
                // the scale's first half-sweep cannot grow a list: every flag is still set
                if (lists && (it > 0 || colour == 1)) {
                    sl.out = c->lists[colour ^ 1];
                    sl.n_out = c->list_counts + t;
                }
                if (lists && it > 0) {
                    sl.in = c->lists[colour];
                    sl.n_in = c->list_counts + t - 1;
                }
                const LevelView &vv = it > 0 ? v : (colour == 0 ? first : second);
                CK(launch_sweep(c->msg_kind, vv, colour, c->D, c->Dp, c->Gp, lambda, trunc, skip, c->trace + t, st, sl,
                                c->variant[l]));
                if (prof) {
                    CK(cudaEventRecord(c->ev[2 * c->prof_all + 1], st));
                    c->prof_span[c->prof_all] = 1;
                    ++c->prof_all;
                    if (l == 0) ++c->prof_launches;
                }
            }
        }
    }
    c->last_levels = levels;
    c->last_trace_n = ntrace;
    return BPS_OK;
}

// A solve with `its` iterations per scale: enqueued, or recorded once as a graph and replayed.
static int solve_iters(bps_ctx *c, int levels, const Iters &its, int lambda, int trunc, int flags, const void *init,
                       cudaStream_t st) {
    const int f = flags & ~BPS_FLAG_GRAPH;
    if (!(flags & BPS_FLAG_GRAPH) || (flags & BPS_FLAG_PROFILE)) return enqueue_bp(c, levels, its, lambda, trunc, f, init, st);
    // the solve recorded once as a graph, replayed while its arguments and the kernel choices hold
    std::vector<intptr_t> key = {levels, lambda, trunc, f, (intptr_t)init, (intptr_t)c->config_version};
    for (int l = 0; l < levels; ++l) key.push_back(its.n[l]);
    const int e = replay_or_record(c->solve_graph, key, c->cap, st, [&](cudaStream_t s) {
        return enqueue_bp(c, levels, its, lambda, trunc, f, init, s);
    });
    if (e == BPS_OK) {  // what recording set on the host, a replay sets again
        c->last_levels = levels;
        c->last_trace_n = its.trace_len(levels);
        c->last_sparse_k = (f & BPS_FLAG_PERSISTENT) ? 0 : c->sv.K;
    }
    return e;
}

extern "C" int bps_bp_solve(bps_ctx *c, int levels, int iters, int lambda, int trunc, int flags, const void *init,
                            void *stream) {
    const int rc = check_bp_args(c, levels, iters, lambda, trunc, flags & ~BPS_FLAG_GRAPH, init);
    if (rc != BPS_OK) return rc;
    return solve_iters(c, levels, Iters::uniform(levels, iters), lambda, trunc, flags, init, (cudaStream_t)stream);
}

extern "C" int bps_bp_solve_schedule(bps_ctx *c, int levels, const int *h_iters, int lambda, int trunc, int flags,
                                     const void *init, void *stream) {
    if (!c || !h_iters || levels < 1 || levels > c->levels) return BPS_ERR_ARG;
    Iters its;
    for (int l = 0; l < levels; ++l) {
        const int rc = check_bp_args(c, levels, h_iters[l], lambda, trunc, flags & ~BPS_FLAG_GRAPH, init);
        if (rc != BPS_OK) return rc;
        its.n[l] = h_iters[l];
    }
    if ((flags & BPS_FLAG_PERSISTENT) && !its.uniform_over(levels)) return BPS_ERR_UNSUPPORTED;
    return solve_iters(c, levels, its, lambda, trunc, flags, init, (cudaStream_t)stream);
}

extern "C" int bps_wta_disparity(bps_ctx *c, int32_t *disp, void *stream) {
    if (!c || !disp) return BPS_ERR_ARG;
    if (!c->has_cost) return BPS_ERR_STATE;
    if (c->last_sparse_k) CK(launch_sparse_wta(c->lv[0], c->sv, disp, (cudaStream_t)stream));
    else CK(launch_wta(c->msg_kind, c->lv[0], c->D, c->Dp, c->Gp, disp, (cudaStream_t)stream));
    return BPS_OK;
}

extern "C" int bps_energy(bps_ctx *c, const int32_t *disp, int lambda, int trunc, int64_t *e_i64, double *e_f64,
                          void *stream) {
    if (!c || !disp || lambda < 0 || trunc < 0) return BPS_ERR_ARG;
    if (!c->has_cost) return BPS_ERR_STATE;
    CK(launch_energy(c->cost_kind, c->lv[0], c->D, c->Dp, disp, lambda, trunc, c->partials, e_i64, e_f64,
                     (cudaStream_t)stream));
    return BPS_OK;
}

static int enqueue_stereo(bps_ctx *c, const uint8_t *L, const uint8_t *R, int pitch, int window, int trunc_data,
                          int iters, int lambda, int trunc, int flags, int32_t *disp, cudaStream_t st) {
    int rc = enqueue_cost(c, L, R, pitch, window, trunc_data, nullptr, st);
    if (rc != BPS_OK) return rc;
    return enqueue_bp(c, c->levels, Iters::uniform(c->levels, iters), lambda, trunc,
                      flags & (BPS_FLAG_FAST_SKIP | BPS_FLAG_PERSISTENT), nullptr,
                      st, disp);
}

extern "C" int bps_stereo(bps_ctx *c, const uint8_t *L, const uint8_t *R, int pitch, int window, int trunc_data,
                          int iters, int lambda, int trunc, int flags, int32_t *disp, void *stream) {
    int rc = check_cost_args(c, L, R, pitch, window, trunc_data);
    if (rc != BPS_OK) return rc;
    if (!disp || (flags & ~(BPS_FLAG_FAST_SKIP | BPS_FLAG_GRAPH | BPS_FLAG_PERSISTENT))) return BPS_ERR_ARG;
    const bool had_cost = c->has_cost;
    c->has_cost = true;  // the sequence builds the cost volume first
    rc = check_bp_args(c, c->levels, iters, lambda, trunc, flags & BPS_FLAG_FAST_SKIP, nullptr);
    if (rc != BPS_OK) {
        c->has_cost = had_cost;
        return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    if (!(flags & BPS_FLAG_GRAPH)) return enqueue_stereo(c, L, R, pitch, window, trunc_data, iters, lambda, trunc, flags, disp, st);

    GraphKey key;
    std::memset(&key, 0, sizeof(key));
    key.L = L;
    key.R = R;
    key.disp = disp;
    key.pitch = pitch;
    key.window = window;
    key.trunc_data = trunc_data;
    key.iters = iters;
    key.lambda = lambda;
    key.trunc = trunc;
    key.flags = flags;
    if (!c->gexec || !(key == c->gkey)) {
        if (c->gexec) {
            cudaGraphExecDestroy(c->gexec);
            c->gexec = nullptr;
        }
        CK(cudaStreamSynchronize(c->cap));
        CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
        rc = enqueue_stereo(c, L, R, pitch, window, trunc_data, iters, lambda, trunc, flags, disp, c->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(c->cap, &graph);
        if (rc != BPS_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != BPS_OK ? rc : BPS_ERR_CUDA;
        }
        const cudaError_t ei = cudaGraphInstantiate(&c->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            c->gexec = nullptr;
            return BPS_ERR_CUDA;
        }
        c->gkey = key;
    }
    CK(cudaGraphLaunch(c->gexec, st));
    c->last_levels = c->levels;  // what recording set on the host, a replay sets again
    c->last_trace_n = c->levels * iters * 2;
    c->last_sparse_k = (flags & BPS_FLAG_PERSISTENT) ? 0 : c->sv.K;
    return BPS_OK;
}

// Host images in, pipeline, energy, host disparity (and energies) out, on stream st.
static int enqueue_stereo_host(bps_ctx *c, const uint8_t *hL, const uint8_t *hR, int pitch, int window, int trunc_data,
                               int iters, int lambda, int trunc, int flags, int32_t *h_disp, int64_t *h_e_i64,
                               double *h_e_f64, cudaStream_t st) {
    CK(cudaMemcpy2DAsync(c->img[0], c->W, hL, pitch, c->W, c->H, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpy2DAsync(c->img[1], c->W, hR, pitch, c->W, c->H, cudaMemcpyHostToDevice, st));
    const int rc = enqueue_stereo(c, c->img[0], c->img[1], c->W, window, trunc_data, iters, lambda, trunc, flags,
                                  c->disp, st);
    if (rc != BPS_OK) return rc;
    if (h_e_i64 || h_e_f64) {
        CK(launch_energy(c->cost_kind, c->lv[0], c->D, c->Dp, c->disp, lambda, trunc, c->partials,
                         c->msg_type == BPS_MSG_FP16 ? nullptr : c->e_i64, c->e_f64, st));
    }
    CK(cudaMemcpyAsync(h_disp, c->disp, (size_t)c->W * c->H * 4, cudaMemcpyDeviceToHost, st));
    if (h_e_i64 && c->msg_type != BPS_MSG_FP16) CK(cudaMemcpyAsync(h_e_i64, c->e_i64, 8, cudaMemcpyDeviceToHost, st));
    if (h_e_f64) CK(cudaMemcpyAsync(h_e_f64, c->e_f64, 8, cudaMemcpyDeviceToHost, st));
    return BPS_OK;
}

extern "C" int bps_stereo_host(bps_ctx *c, const uint8_t *hL, const uint8_t *hR, int pitch, int window,
                               int trunc_data, int iters, int lambda, int trunc, int flags, int32_t *h_disp,
                               int64_t *h_e_i64, double *h_e_f64, void *stream) {
    if (!c || !hL || !hR || !h_disp || pitch < c->W) return BPS_ERR_ARG;
    int rc = check_cost_args(c, c->img[0], c->img[1], c->W, window, trunc_data);
    if (rc != BPS_OK) return rc;
    if (flags & ~(BPS_FLAG_FAST_SKIP | BPS_FLAG_GRAPH | BPS_FLAG_PERSISTENT | BPS_FLAG_ASYNC)) return BPS_ERR_ARG;
    const bool async = (flags & BPS_FLAG_ASYNC) != 0;
    flags &= ~BPS_FLAG_ASYNC;
    const bool had_cost = c->has_cost;
    c->has_cost = true;  // the sequence builds the cost volume first
    rc = check_bp_args(c, c->levels, iters, lambda, trunc, flags & (BPS_FLAG_FAST_SKIP | BPS_FLAG_PERSISTENT), nullptr);
    if (rc != BPS_OK) {
        c->has_cost = had_cost;
        return rc;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int f = flags & ~BPS_FLAG_GRAPH;
    // with page-locked buffers (checked when the graph is recorded) the whole call, copies
    // included, replays as one graph
    const std::vector<intptr_t> key = {(intptr_t)hL, (intptr_t)hR, (intptr_t)h_disp, (intptr_t)h_e_i64,
                                       (intptr_t)h_e_f64, pitch, window, trunc_data, iters, lambda, trunc, f,
                                       (intptr_t)c->config_version};
    const bool replay = (flags & BPS_FLAG_GRAPH) && c->host_graph.exec && key == c->host_graph.key;
    if (replay || ((flags & BPS_FLAG_GRAPH) && is_pinned(hL) && is_pinned(hR) && is_pinned(h_disp) &&
                   (!h_e_i64 || is_pinned(h_e_i64)) && (!h_e_f64 || is_pinned(h_e_f64)))) {
        rc = replay_or_record(c->host_graph, key, c->cap, st, [&](cudaStream_t s) {
            return enqueue_stereo_host(c, hL, hR, pitch, window, trunc_data, iters, lambda, trunc, f, h_disp, h_e_i64,
                                       h_e_f64, s);
        });
    } else {
        rc = enqueue_stereo_host(c, hL, hR, pitch, window, trunc_data, iters, lambda, trunc, f, h_disp, h_e_i64,
                                 h_e_f64, st);
    }
    if (rc != BPS_OK) return rc;
    if (async) return BPS_OK;
    CK(cudaStreamSynchronize(st));
    // only the persistent kernel's barrier can time out
    return (flags & BPS_FLAG_PERSISTENT) ? bps_get_error(c) : BPS_OK;
}

extern "C" int bps_peek_error_code(bps_ctx *c) {
    if (!c) return BPS_ERR_ARG;
    unsigned w = 0u;
    CK(cudaMemcpy(&w, c->d_barrier + 2, sizeof(w), cudaMemcpyDeviceToHost));
    return (int)w;
}

extern "C" int bps_test_fail_resources(int n) {
    g_fail_after.store(n < 0 ? -1 : n);
    return BPS_OK;
}

extern "C" int bps_get_error(bps_ctx *c) {
    if (!c) return BPS_ERR_ARG;
    unsigned w[3] = {0u, 0u, 0u};
    CK(cudaMemcpy(w, c->d_barrier, sizeof(w), cudaMemcpyDeviceToHost));
    if (w[2]) CK(cudaMemset(c->d_barrier + 2, 0, sizeof(unsigned)));  // reported once
    if (w[2] >= 2u) return BPS_ERR_INTERNAL;
    return (w[1] || w[2]) ? BPS_ERR_TIMEOUT : BPS_OK;
}

extern "C" int bps_get_trace(bps_ctx *c, int64_t *h_counts, int cap) {
    if (!c || (!h_counts && cap > 0) || cap < 0) return BPS_ERR_ARG;
    const int n = std::min(cap, c->last_trace_n);
    if (n <= 0) return 0;
    std::vector<unsigned long long> tmp(n);
    CK(cudaMemcpy(tmp.data(), c->trace, sizeof(unsigned long long) * n, cudaMemcpyDeviceToHost));
    for (int k = 0; k < n; ++k) h_counts[k] = (int64_t)tmp[k];
    return n;
}

extern "C" int bps_export_messages(bps_ctx *c, int level, void *d_out, void *stream) {
    if (!c || !d_out || level < 0 || level >= c->levels) return BPS_ERR_ARG;
    if (level == 0 && c->last_sparse_k) return BPS_ERR_STATE;  // the finest scale holds sparse messages
    CK(launch_export_msgs(c->msg_kind, c->lv[level], c->D, c->Dp, d_out, (cudaStream_t)stream));
    return BPS_OK;
}

extern "C" int bps_export_cost(bps_ctx *c, int level, void *d_out, void *stream) {
    if (!c || !d_out || level < 0 || level >= c->levels) return BPS_ERR_ARG;
    if (!c->has_cost) return BPS_ERR_STATE;
    CK(launch_export_cost(c->cost_kind, c->lv[level], c->D, c->Dp, d_out, (cudaStream_t)stream));
    return BPS_OK;
}

extern "C" int bps_read_profile(bps_ctx *c, int *h_launches, double *h_total_ms, int64_t *h_pixels) {
    if (!c || !h_launches || !h_total_ms || !h_pixels) return BPS_ERR_ARG;
    double total = 0.0;
    int covered = 0;
    for (int k = c->prof_all - 1; k >= 0 && covered < c->prof_launches; --k) {
        CK(cudaEventSynchronize(c->ev[2 * k + 1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
        total += ms;
        covered += (int)c->prof_span.size() > k ? c->prof_span[k] : 1;
    }
    int64_t px = 0;
    if (c->prof_launches && c->prof_trace_n) {
        std::vector<unsigned long long> tmp(c->prof_trace_n);
        CK(cudaMemcpy(tmp.data(), c->trace + c->prof_first_trace, sizeof(unsigned long long) * c->prof_trace_n,
                      cudaMemcpyDeviceToHost));
        for (unsigned long long v : tmp) px += (int64_t)v;
    }
    *h_launches = c->prof_launches;
    *h_total_ms = total;
    *h_pixels = px;
    return BPS_OK;
}

extern "C" int bps_read_launch_times(bps_ctx *c, double *h_ms, int cap) {
    if (!c || cap < 0 || (!h_ms && cap > 0)) return BPS_ERR_ARG;
    int n = 0;
    for (int k = 0; k < c->prof_all; ++k) {
        CK(cudaEventSynchronize(c->ev[2 * k + 1]));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, c->ev[2 * k], c->ev[2 * k + 1]));
        // a launch covering several half-sweeps (a cluster launch) is shared out evenly
        const int span = (int)c->prof_span.size() > k ? c->prof_span[k] : 1;
        for (int j = 0; j < span && n < cap; ++j) h_ms[n++] = ms / span;
    }
    return n;
}

// ------------------------------------------------------------------ batches of pairs

struct bps_batch {
    std::vector<bps_ctx *> ctxs;
    int levels = 0, msg_type = 0, msg_kind = 0;
    std::vector<cudaStream_t> streams;  // one branch stream per pair
    std::vector<cudaEvent_t> events;    // fork event, then one join event per pair
    cudaStream_t cap = nullptr;
    // lockstep persistent launch over all pairs
    PairDesc *d_desc = nullptr;
    int *d_prefix = nullptr;  // [levels][n + 1] sweep prefixes, then [n + 1] read-out prefix
    unsigned *d_barrier = nullptr;
    std::vector<PairDesc> h_desc;
    int grid = 0;
    // graph cache
    cudaGraphExec_t gexec = nullptr;
    std::vector<intptr_t> gkey;
    GraphSlot host_graph;  // bps_batch_stereo_host: copies in, pipelines, energies, copies out
};

namespace {

std::vector<intptr_t> batch_key(const bps_batch *b, const uint8_t *const *L, const uint8_t *const *R,
                                const int *pitches, const int *windows, int trunc_data, int iters, int lambda,
                                int trunc, int flags, int32_t *const *disps) {
    std::vector<intptr_t> k = {trunc_data, iters, lambda, trunc, flags};
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        k.push_back((intptr_t)L[i]);
        k.push_back((intptr_t)R[i]);
        k.push_back(pitches[i]);
        k.push_back(windows[i]);
        k.push_back((intptr_t)disps[i]);
        k.push_back((intptr_t)b->ctxs[i]->config_version);  // a member's kernel choices changed
    }
    return k;
}

void batch_free(bps_batch *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    b->host_graph.reset();
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->events) cudaEventDestroy(e);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_desc) cudaFree(b->d_desc);
    if (b->d_prefix) cudaFree(b->d_prefix);
    if (b->d_barrier) cudaFree(b->d_barrier);
    delete b;
}

}  // namespace

extern "C" int bps_batch_create(bps_batch **out, bps_ctx *const *ctxs, int n) {
    if (!out || !ctxs || n < 1 || n > BPS_MAX_BATCH) return BPS_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!ctxs[i] || ctxs[i]->levels != ctxs[0]->levels || ctxs[i]->msg_type != ctxs[0]->msg_type)
            return BPS_ERR_ARG;
    bps_batch *b = new (std::nothrow) bps_batch();
    if (!b) return BPS_ERR_CUDA;
    b->ctxs.assign(ctxs, ctxs + n);
    b->levels = ctxs[0]->levels;
    b->msg_type = ctxs[0]->msg_type;
    b->msg_kind = ctxs[0]->msg_kind;
    bool ok = acquire_stream(&b->cap) == cudaSuccess;
    for (int i = 0; ok && i < n; ++i) {
        cudaStream_t s;
        ok = acquire_stream(&s) == cudaSuccess;
        if (ok) b->streams.push_back(s);
    }
    for (int i = 0; ok && i <= n; ++i) {
        cudaEvent_t e;
        ok = acquire_event(&e) == cudaSuccess;
        if (ok) b->events.push_back(e);
    }
    // descriptors of the lockstep persistent launch
    const int L = b->levels;
    std::vector<int> prefix((size_t)(L + 1) * (n + 1), 0);
    for (int l = 0; l < L; ++l)
        for (int i = 0; i < n; ++i) prefix[(size_t)l * (n + 1) + i + 1] = prefix[(size_t)l * (n + 1) + i] + sweep_blocks(ctxs[i], l);
    for (int i = 0; i < n; ++i) prefix[(size_t)L * (n + 1) + i + 1] = prefix[(size_t)L * (n + 1) + i] + wta_blocks(ctxs[i]);
    for (int i = 0; i < n; ++i) b->h_desc.push_back(make_desc(ctxs[i]));
    ok = ok && acquire_memory(reinterpret_cast<void **>(&b->d_desc), sizeof(PairDesc) * n) == cudaSuccess;
    ok = ok && acquire_memory(reinterpret_cast<void **>(&b->d_prefix), sizeof(int) * prefix.size()) == cudaSuccess;
    ok = ok && acquire_memory(reinterpret_cast<void **>(&b->d_barrier), 2 * sizeof(unsigned)) == cudaSuccess;
    ok = ok && cudaMemcpy(b->d_desc, b->h_desc.data(), sizeof(PairDesc) * n, cudaMemcpyHostToDevice) == cudaSuccess;
    ok = ok && cudaMemcpy(b->d_prefix, prefix.data(), sizeof(int) * prefix.size(), cudaMemcpyHostToDevice) == cudaSuccess;
    for (int T = 1; ok && T <= 3; ++T) ok = persistent_grid(b->msg_kind, T, &b->grid) == cudaSuccess;
    if (!ok) {
        batch_free(b);
        return BPS_ERR_CUDA;
    }
    *out = b;
    return BPS_OK;
}

extern "C" int bps_batch_destroy(bps_batch *b) {
    if (!b) return BPS_OK;
    if (b->cap) cudaStreamSynchronize(b->cap);
    for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
    batch_free(b);
    return BPS_OK;
}

// Every pair's chain on its own branch stream, forked from and joined back into `st`.
// Host buffers of a batch call: images copied in at the head of each pair's branch, the
// disparity (and energy) copied out at its tail.
struct BatchHostIO {
    const uint8_t *const *lefts, *const *rights;
    const int *pitches;
    int32_t *const *disps;
    int64_t *energies;
};

static int enqueue_pair_input(bps_ctx *c, const BatchHostIO *io, int i, cudaStream_t st) {
    if (!io) return BPS_OK;
    CK(cudaMemcpy2DAsync(c->img[0], c->W, io->lefts[i], io->pitches[i], c->W, c->H, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpy2DAsync(c->img[1], c->W, io->rights[i], io->pitches[i], c->W, c->H, cudaMemcpyHostToDevice, st));
    return BPS_OK;
}

static int enqueue_pair_output(bps_ctx *c, const BatchHostIO *io, int i, int lambda, int trunc, cudaStream_t st) {
    if (!io) return BPS_OK;
    if (io->energies) {
        CK(launch_energy(c->cost_kind, c->lv[0], c->D, c->Dp, c->disp, lambda, trunc, c->partials,
                         c->msg_type == BPS_MSG_FP16 ? nullptr : c->e_i64, c->e_f64, st));
        CK(cudaMemcpyAsync(io->energies + i, c->e_i64, 8, cudaMemcpyDeviceToHost, st));
    }
    CK(cudaMemcpyAsync(io->disps[i], c->disp, (size_t)c->W * c->H * 4, cudaMemcpyDeviceToHost, st));
    return BPS_OK;
}

static int enqueue_batch(bps_batch *b, const uint8_t *const *L, const uint8_t *const *R, const int *pitches,
                         const int *windows, int trunc_data, int iters, int lambda, int trunc, int flags,
                         int32_t *const *disps, cudaStream_t st, const BatchHostIO *io = nullptr) {
    const int n = (int)b->ctxs.size();
    if (flags & BPS_FLAG_PERSISTENT) {
        // costs of every pair on the branches, then one lockstep launch for all pairs
        CK(cudaEventRecord(b->events[0], st));
        for (int i = 0; i < n; ++i) {
            bps_ctx *c = b->ctxs[i];
            CK(cudaStreamWaitEvent(b->streams[i], b->events[0], 0));
            int rc = enqueue_pair_input(c, io, i, b->streams[i]);
            if (rc == BPS_OK) rc = enqueue_cost(c, L[i], R[i], pitches[i], windows[i], trunc_data, nullptr, b->streams[i]);
            if (rc == BPS_OK) rc = enqueue_start(c, b->levels - 1, 0, nullptr, b->streams[i]);
            if (rc != BPS_OK) return rc;
            if (iters) {
                CK(cudaMemsetAsync(c->trace, 0, sizeof(unsigned long long) * b->levels * iters * 2, b->streams[i]));
                CK(cudaMemsetAsync(c->list_counts, 0, sizeof(unsigned) * b->levels * iters * 2, b->streams[i]));
            }
            CK(cudaEventRecord(b->events[i + 1], b->streams[i]));
            CK(cudaStreamWaitEvent(st, b->events[i + 1], 0));
        }
        CK(cudaMemsetAsync(b->d_barrier, 0, 2 * sizeof(unsigned), st));
        PersistParams P = persist_params(n, b->d_desc, b->d_prefix, b->d_prefix + (size_t)b->levels * (n + 1),
                                         b->d_barrier, b->levels, iters, lambda, trunc, flags);
        CK(launch_persistent(b->msg_kind, P, st));
        for (int i = 0; i < n; ++i) {
            bps_ctx *c = b->ctxs[i];
            c->last_levels = b->levels;
            c->last_trace_n = b->levels * iters * 2;
            const int rc = enqueue_pair_output(c, io, i, lambda, trunc, st);
            if (rc != BPS_OK) return rc;
        }
        return BPS_OK;
    }
    CK(cudaEventRecord(b->events[0], st));
    for (int i = 0; i < n; ++i) {
        CK(cudaStreamWaitEvent(b->streams[i], b->events[0], 0));
        int rc = enqueue_pair_input(b->ctxs[i], io, i, b->streams[i]);
        if (rc == BPS_OK)
            rc = enqueue_stereo(b->ctxs[i], L[i], R[i], pitches[i], windows[i], trunc_data, iters, lambda, trunc,
                                flags & BPS_FLAG_FAST_SKIP, disps[i], b->streams[i]);
        if (rc == BPS_OK) rc = enqueue_pair_output(b->ctxs[i], io, i, lambda, trunc, b->streams[i]);
        if (rc != BPS_OK) return rc;
        CK(cudaEventRecord(b->events[i + 1], b->streams[i]));
        CK(cudaStreamWaitEvent(st, b->events[i + 1], 0));
    }
    return BPS_OK;
}

// Argument checks of a batch call, and the persistent launch's read-out targets refreshed.
static int batch_prepare(bps_batch *b, const uint8_t *const *d_lefts, const uint8_t *const *d_rights,
                         const int *pitches, const int *windows, int trunc_data, int iters, int lambda, int trunc,
                         int flags, int32_t *const *d_disps, void *stream) {
    if (!b || !d_lefts || !d_rights || !pitches || !windows || !d_disps ||
        (flags & ~(BPS_FLAG_FAST_SKIP | BPS_FLAG_GRAPH | BPS_FLAG_PERSISTENT)))
        return BPS_ERR_ARG;
    const int n = (int)b->ctxs.size();
    for (int i = 0; i < n; ++i) {
        bps_ctx *c = b->ctxs[i];
        int rc = check_cost_args(c, d_lefts[i], d_rights[i], pitches[i], windows[i], trunc_data);
        if (rc != BPS_OK) return rc;
        if (!d_disps[i]) return BPS_ERR_ARG;
        const bool had = c->has_cost;
        c->has_cost = true;
        rc = check_bp_args(c, c->levels, iters, lambda, trunc, flags & (BPS_FLAG_FAST_SKIP | BPS_FLAG_PERSISTENT),
                           nullptr);
        if (rc != BPS_OK) {
            c->has_cost = had;
            return rc;
        }
    }
    if (flags & BPS_FLAG_PERSISTENT) {
        // the read-out targets live in the device descriptors: refresh them when they change
        bool changed = false;
        for (int i = 0; i < n; ++i) {
            if (b->h_desc[i].disp != d_disps[i]) {
                b->h_desc[i].disp = d_disps[i];
                changed = true;
            }
            const bps_ctx *c = b->ctxs[i];
            if (b->h_desc[i].lv[0].eps != c->lv[0].eps || b->h_desc[i].lv[0].freeze != c->lv[0].freeze) {
                for (int l = 0; l < c->levels; ++l) b->h_desc[i].lv[l] = c->lv[l];  // the skip rule changed
                changed = true;
            }
        }
        if (changed) {
            for (cudaStream_t s : b->streams) CK(cudaStreamSynchronize(s));
            CK(cudaStreamSynchronize((cudaStream_t)stream));
            CK(cudaMemcpy(b->d_desc, b->h_desc.data(), sizeof(PairDesc) * n, cudaMemcpyHostToDevice));
        }
    }
    return BPS_OK;
}

extern "C" int bps_batch_stereo(bps_batch *b, const uint8_t *const *d_lefts, const uint8_t *const *d_rights,
                                const int *pitches, const int *windows, int trunc_data, int iters, int lambda, int trunc,
                                int flags, int32_t *const *d_disps, void *stream) {
    const int prc = batch_prepare(b, d_lefts, d_rights, pitches, windows, trunc_data, iters, lambda, trunc, flags,
                                  d_disps, stream);
    if (prc != BPS_OK) return prc;
    cudaStream_t st = (cudaStream_t)stream;
    if (!(flags & BPS_FLAG_GRAPH))
        return enqueue_batch(b, d_lefts, d_rights, pitches, windows, trunc_data, iters, lambda, trunc, flags, d_disps, st);
    std::vector<intptr_t> key = batch_key(b, d_lefts, d_rights, pitches, windows, trunc_data, iters, lambda, trunc,
                                          flags, d_disps);
    if (!b->gexec || key != b->gkey) {
        if (b->gexec) {
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        CK(cudaStreamSynchronize(b->cap));
        CK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        const int rc = enqueue_batch(b, d_lefts, d_rights, pitches, windows, trunc_data, iters, lambda, trunc, flags,
                                     d_disps, b->cap);
        cudaGraph_t graph = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(b->cap, &graph);
        if (rc != BPS_OK || ec != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return rc != BPS_OK ? rc : cuda_failed(ec);
        }
        const cudaError_t ei = cudaGraphInstantiate(&b->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            b->gexec = nullptr;
            return cuda_failed(ei);
        }
        b->gkey = key;
    }
    CK(cudaGraphLaunch(b->gexec, st));
    return BPS_OK;
}

extern "C" int bps_batch_get_error(bps_batch *b) {
    if (!b) return BPS_ERR_ARG;
    unsigned w[2] = {0u, 0u};
    CK(cudaMemcpy(w, b->d_barrier, sizeof(w), cudaMemcpyDeviceToHost));
    return w[1] ? BPS_ERR_TIMEOUT : BPS_OK;
}

extern "C" int bps_batch_stereo_host(bps_batch *b, const uint8_t *const *h_lefts, const uint8_t *const *h_rights,
                                     const int *pitches, const int *windows, int trunc_data, int iters, int lambda,
                                     int trunc, int flags, int32_t *const *h_disps, int64_t *h_energies,
                                     void *stream) {
    if (!b || !h_lefts || !h_rights || !pitches || !windows || !h_disps) return BPS_ERR_ARG;
    const bool async = (flags & BPS_FLAG_ASYNC) != 0;
    flags &= ~BPS_FLAG_ASYNC;
    const int n = (int)b->ctxs.size();
    std::vector<const uint8_t *> L(n), R(n);
    std::vector<int> pitch(n);
    std::vector<int32_t *> disp(n);
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i) {
        bps_ctx *c = b->ctxs[i];
        if (!h_lefts[i] || !h_rights[i] || !h_disps[i] || pitches[i] < c->W) return BPS_ERR_ARG;
        L[i] = c->img[0];
        R[i] = c->img[1];
        pitch[i] = c->W;
        disp[i] = c->disp;
    }
    std::vector<intptr_t> key = batch_key(b, L.data(), R.data(), pitch.data(), windows, trunc_data, iters, lambda,
                                          trunc, flags, disp.data());
    key.push_back((intptr_t)h_energies);
    for (int i = 0; i < n; ++i) {
        key.push_back((intptr_t)h_lefts[i]);
        key.push_back((intptr_t)h_rights[i]);
        key.push_back(pitches[i]);
        key.push_back((intptr_t)h_disps[i]);
    }
    // page-locked buffers (checked when the graph is recorded): the whole call, copies
    // included, replays as one graph
    bool pinned = (flags & BPS_FLAG_GRAPH) != 0;
    if (pinned && !(b->host_graph.exec && key == b->host_graph.key)) {
        pinned = !h_energies || is_pinned(h_energies);
        for (int i = 0; i < n && pinned; ++i)
            pinned = is_pinned(h_lefts[i]) && is_pinned(h_rights[i]) && is_pinned(h_disps[i]);
    }
    const BatchHostIO io{h_lefts, h_rights, pitches, h_disps, h_energies};
    int rc;
    if (pinned) {
        rc = batch_prepare(b, L.data(), R.data(), pitch.data(), windows, trunc_data, iters, lambda, trunc, flags,
                           disp.data(), stream);
        if (rc != BPS_OK) return rc;
        rc = replay_or_record(b->host_graph, key, b->cap, st, [&](cudaStream_t s) {
            return enqueue_batch(b, L.data(), R.data(), pitch.data(), windows, trunc_data, iters, lambda, trunc, flags,
                                 disp.data(), s, &io);
        });
    } else {
        for (int i = 0; i < n; ++i) {
            rc = enqueue_pair_input(b->ctxs[i], &io, i, st);
            if (rc != BPS_OK) return rc;
        }
        rc = bps_batch_stereo(b, L.data(), R.data(), pitch.data(), windows, trunc_data, iters, lambda, trunc, flags,
                              disp.data(), stream);
        for (int i = 0; i < n && rc == BPS_OK; ++i) rc = enqueue_pair_output(b->ctxs[i], &io, i, lambda, trunc, st);
    }
    if (rc != BPS_OK) return rc;
    if (async) return BPS_OK;
    CK(cudaStreamSynchronize(st));
    return (flags & BPS_FLAG_PERSISTENT) ? bps_batch_get_error(b) : BPS_OK;
}

extern "C" int bps_set_sweep_variant(bps_ctx *c, int level, int variant) {
    if (!c || level < 0 || level >= c->levels || variant < -1 ||
        variant > (BPS_VARIANT_GENERAL_DT | BPS_VARIANT_LISTS | BPS_VARIANT_CLUSTER | BPS_VARIANT_EAGER |
                   BPS_VARIANT_DPAR | BPS_VARIANT_DPAR_LISTS | BPS_VARIANT_STAGED | BPS_VARIANT_STAGED_LISTS |
                   BPS_VARIANT_BULK | BPS_VARIANT_BULK_LISTS | BPS_VARIANT_BLOCK2))
        return BPS_ERR_ARG;
    if (variant > 0 && (variant & VARIANT_CLUSTER) && !cluster_sweep_available()) return BPS_ERR_UNSUPPORTED;
    c->variant[level] = variant < 0 ? default_variant((int64_t)c->plan.Hs[level] * c->plan.Whs[level], c->Gp, c->msg_kind)
                                       : variant;
    ++c->config_version;
    if (c->gexec) {  // a recorded graph holds the old kernels
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return BPS_OK;
}

extern "C" int bps_set_candidates(bps_ctx *c, int K) {
    if (!c || K < 0 || K > BPS_MAX_CANDIDATES || K > c->D) return BPS_ERR_ARG;
    if (K > 0 && (c->msg_kind != MSG_U8 || c->lv[0].eps || c->lv[0].freeze)) return BPS_ERR_UNSUPPORTED;
    int Kp = 1;
    while (Kp < K) Kp *= 2;
    c->sv.K = K;
    c->sv.Kp = K ? Kp : 0;
    ++c->config_version;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return BPS_OK;
}

extern "C" int bps_export_sparse(bps_ctx *c, int32_t *d_cand, int32_t *d_msgs, void *stream) {
    if (!c || !d_cand || !d_msgs) return BPS_ERR_ARG;
    if (!c->last_sparse_k || c->last_sparse_k != c->sv.K) return BPS_ERR_STATE;
    CK(launch_sparse_export(c->lv[0], c->sv, d_cand, d_msgs, (cudaStream_t)stream));
    return BPS_OK;
}

extern "C" int bps_set_skip_rule(bps_ctx *c, int eps, int freeze) {
    if (!c || eps < 0 || eps > 255 || (freeze != 0 && freeze != 1)) return BPS_ERR_ARG;
    if ((eps || freeze) && c->msg_kind != MSG_U8) return BPS_ERR_UNSUPPORTED;
    if ((eps || freeze) && c->sv.K) return BPS_ERR_UNSUPPORTED;  // the sparse solve keeps the exact rule
    for (int l = 0; l < c->levels; ++l) {
        c->lv[l].eps = eps;
        c->lv[l].freeze = freeze;
    }
    // this context's own descriptor (the persistent form) carries the level views
    PairDesc hd = make_desc(c);
    CK(cudaMemcpy(c->d_desc, &hd, sizeof(hd), cudaMemcpyHostToDevice));
    ++c->config_version;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return BPS_OK;
}

extern "C" int bps_get_sweep_variant(bps_ctx *c, int level) {
    if (!c || level < 0 || level >= c->levels) return BPS_ERR_ARG;
    return c->variant[level];
}

extern "C" int bps_set_ncc_kernel(bps_ctx *c, int kernel, int rows) {
    if (!c || kernel < BPS_NCC_DEFAULT || kernel > BPS_NCC_TENSOR || rows < 0 || (rows & 1)) return BPS_ERR_ARG;
    c->ncc_kernel = kernel;
    c->ncc_tc_rows = rows;
    ++c->config_version;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return BPS_OK;
}

extern "C" int bps_get_ncc_kernel(bps_ctx *c, int window, int trunc_data) {
    if (!c) return BPS_ERR_ARG;
    const bool tc = c->ncc_kernel != BPS_NCC_ROWS && ncc_tc_supported(c->cost_kind, c->Dp, window, trunc_data);
    return tc ? BPS_NCC_TENSOR : BPS_NCC_ROWS;
}

extern "C" int bps_set_ncc_shape(bps_ctx *c, int column_groups, int rows) {
    if (!c || column_groups < 0 || rows < 0 || (rows & 1) || column_groups * c->Dp > 512 ||
        (column_groups > 0 && column_groups * c->Dp < 32))
        return BPS_ERR_ARG;
    c->ncc_xs = column_groups;
    c->ncc_rows = rows;
    ++c->config_version;
    if (c->gexec) {
        cudaGraphExecDestroy(c->gexec);
        c->gexec = nullptr;
    }
    return BPS_OK;
}
