// kp_api.cu -- the C ABI declared in include/kpynq.h.
//
// Host-side runtime of the library: argument checking, device state
// allocation, the per-iteration launch sequence, and the fit loop, which is
// recorded once per context as a CUDA graph whose body (filter -> survivor ->
// update) runs under a device-side `while` conditional node: the update
// kernel evaluates the stop rule and sets the loop condition, so a fit costs
// one graph launch and one final synchronisation.
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "kp_common.cuh"

namespace kp {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace kp

using namespace kp;

static thread_local char g_init_error[512] = "";
// set while the batched form creates its problems' contexts: those run inside
// the batch's graph and never launch a fit graph of their own
static thread_local bool t_ctx_in_batch = false;

namespace kp {
void set_thread_error(const char *msg) { snprintf(g_init_error, sizeof(g_init_error), "%s", msg); }
}  // namespace kp

struct kmeans_ctx {
    int dev = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only to record graphs
    kmeans_options opt{};
    Params p{};
    float *X_own = nullptr;
    int tcap = 0;
    bool use_tc = false;   // dense passes on the tensor cores
    // learned proposal (kmeans_set_proposal): the network (tensor-core
    // inference), the predictions and the centroid-distance table
    bool proposal = false;
    kmeans_mlp *net = nullptr;
    float *cc_table = nullptr;
    int32_t *pred = nullptr;
    bool have_final = false;  // a fit finished: its final-assignment record is kept
    // sharded iterations (kmeans_shard_*): the cluster sums of every
    // assignment are rebuilt from this shard's points about the current
    // centroids, so that every shard's sums share one reference point
    bool shard = false;
    bool shard_pending = false;  // an assignment waits for its update
    int t_host = 0;        // iterations run (mirrors ctrl->t after each call)
    int v_host = 0;        // table version (mirrors ctrl->v)
    bool broken = false;
    char err[512] = "";
    // fit graph
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaGraphConditionalHandle cond = 0;
    Ctrl *ctrl_host = nullptr;  // pinned mirror of the control block
    int *flag_dev = nullptr;
    std::vector<void *> allocs;
    long long kernels_base = 0;  // device kernel count before the last reset
    // profiling (kmeans_options.profile): CUDA events around every launch
    bool capturing = false;
    double prof_ms[KM_KERNEL_KINDS] = {};
    long long prof_n[KM_KERNEL_KINDS] = {};
    struct Pending {
        int kind;
        cudaEvent_t a, b;
    };
    std::vector<Pending> pending;
    std::vector<cudaEvent_t> ev_pool;
};

namespace {

int set_err(kmeans_ctx *c, int code, const char *fmt, ...) {
    char *buf = c ? c->err : g_init_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    if (c && (code == KM_ECUDA || code == KM_ETIMEOUT)) c->broken = true;
    return code;
}

#define KP_CUDA(c, call)                                                                          \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) {                                                                  \
            int code_ = (e_ == cudaErrorMemoryAllocation) ? KM_ENOMEM : KM_ECUDA;                 \
            return set_err((c), code_, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                           __FILE__, __LINE__);                                                   \
        }                                                                                         \
    } while (0)

// Restores the caller's current device on scope exit.
struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool is_device_ptr(const void *ptr) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Every context allocates from one library-owned memory pool per device
// (stream-ordered, on the context's stream; everything a context allocates is
// used on that stream or after a synchronisation).  Freed blocks stay in the
// pool up to 32 GiB, so that contexts made one after another -- a job that
// creates a context per data set -- reuse memory instead of paying
// cudaMalloc / cudaFree each time.
std::mutex g_pool_mu;
cudaMemPool_t g_pool[256] = {};

cudaError_t lib_pool(int dev, cudaMemPool_t *out) {
    if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        cudaError_t e = cudaMemPoolCreate(&pool, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = (uint64_t)32 << 30;
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) {
            cudaMemPoolDestroy(pool);
            return e;
        }
        g_pool[dev] = pool;
    }
    *out = g_pool[dev];
    return cudaSuccess;
}

// Allocation-failure hook (kmeans_debug_fail_alloc): when >= 0, the number of
// context allocations still allowed before each further one fails as out of
// memory (a host-side stand-in for a full device, for testing KM_ENOMEM)
std::atomic<long long> g_alloc_budget{-1};

template <class T>
cudaError_t dalloc(kmeans_ctx *c, T **p, size_t count) {
    long long b = g_alloc_budget.load();
    while (b >= 0) {
        if (b == 0) return cudaErrorMemoryAllocation;
        if (g_alloc_budget.compare_exchange_weak(b, b - 1)) break;
    }
    cudaMemPool_t pool;
    cudaError_t e = lib_pool(c->dev, &pool);
    if (e != cudaSuccess) return e;
    void *q = nullptr;
    e = cudaMallocFromPoolAsync(&q, count * sizeof(T) + 16, pool, c->stream);
    if (e != cudaSuccess) return e;
    c->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

int padded_stride_c(int D) {
    int dp = dense_dp(D);
    int base = dp > 0 ? dp : ((D + 3) & ~3);
    // an odd number of 16-byte units per row keeps lane-per-centroid float4
    // reads of shared memory free of bank conflicts
    return ((base / 4) % 2 == 0) ? base + 4 : base;
}

float f32_up(double x) {
    float f = (float)x;
    if ((double)f < x) f = nextafterf(f, INFINITY);
    return f;
}
float f32_dn(double x) {
    float f = (float)x;
    if ((double)f > x) f = nextafterf(f, -INFINITY);
    return f;
}

cudaEvent_t take_event(kmeans_ctx *c) {
    if (!c->ev_pool.empty()) {
        cudaEvent_t e = c->ev_pool.back();
        c->ev_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

// Launch through `fn`; when profiling (and not recording a graph), bracket it
// with CUDA events on the context's stream.
template <class F>
cudaError_t timed(kmeans_ctx *c, cudaStream_t s, int kind, F fn) {
    if (!c->opt.profile || c->capturing) return fn();
    cudaEvent_t a = take_event(c), b = take_event(c);
    if (!a || !b) return cudaErrorMemoryAllocation;
    cudaError_t e = cudaEventRecord(a, s);
    if (e != cudaSuccess) return e;
    e = fn();
    if (e != cudaSuccess) return e;
    e = cudaEventRecord(b, s);
    if (e != cudaSuccess) return e;
    c->pending.push_back({kind, a, b});
    return cudaSuccess;
}

// after a stream synchronisation: fold the recorded event pairs in
void collect_profile(kmeans_ctx *c) {
    for (auto &q : c->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
            c->prof_ms[q.kind] += ms;
            c->prof_n[q.kind] += 1;
        }
        c->ev_pool.push_back(q.a);
        c->ev_pool.push_back(q.b);
    }
    c->pending.clear();
}

int sync_and_check(kmeans_ctx *c) {
    KP_CUDA(c, cudaStreamSynchronize(c->stream));
    collect_profile(c);
    KP_CUDA(c, cudaMemcpy(c->ctrl_host, c->p.ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost));
    c->t_host = c->ctrl_host->t;
    c->v_host = c->ctrl_host->v;
    if (c->ctrl_host->err == kErrLabel)
        return set_err(c, KM_ECUDA, "an assignment pass left a label outside [0, K)");
    if (c->ctrl_host->err == kErrQueue)
        return set_err(c, KM_ECUDA, "a work queue held an entry out of range");
    if (c->ctrl_host->err)
        return set_err(c, KM_ETIMEOUT, "a bounded device-side wait gave up (code %d)", c->ctrl_host->err);
    return KM_OK;
}

// Drift tables must hold `need` more versions: rebase (and grow) if not.
int ensure_tables(kmeans_ctx *c, int need) {
    if (c->v_host + need < c->tcap) return KM_OK;
    Params &p = c->p;
    if (p.algo == KM_ALGO_FILTERED && c->t_host > 0) {
        KP_CUDA(c, launch_rebase(p, c->stream, c->num_sms));
    } else {
        Params q = p;
        q.N = 0;
        KP_CUDA(c, launch_rebase(q, c->stream, c->num_sms));
    }
    c->v_host = 0;
    if (need < c->tcap) return KM_OK;
    KP_CUDA(c, cudaStreamSynchronize(c->stream));
    int tcap = ((need + 1 + 63) / 64) * 64;
    if (tcap > 65536) return set_err(c, KM_EINVAL, "max_iter too large (at most 65534)");
    float *Dc, *Dg, *Dm;
    KP_CUDA(c, dalloc(c, &Dc, (size_t)tcap * p.K));
    KP_CUDA(c, dalloc(c, &Dg, (size_t)tcap * p.Gp));
    KP_CUDA(c, dalloc(c, &Dm, (size_t)tcap));
    KP_CUDA(c, cudaMemsetAsync(Dc, 0, (size_t)tcap * p.K * 4, c->stream));
    KP_CUDA(c, cudaMemsetAsync(Dg, 0, (size_t)tcap * p.Gp * 4, c->stream));
    KP_CUDA(c, cudaMemsetAsync(Dm, 0, (size_t)tcap * 4, c->stream));
    p.Dc = Dc;
    p.Dg = Dg;
    p.Dm = Dm;
    c->tcap = tcap;
    if (c->graph_exec) {  // recorded with the old table pointers
        cudaGraphExecDestroy(c->graph_exec);
        cudaGraphDestroy(c->graph);
        c->graph_exec = nullptr;
        c->graph = nullptr;
    }
    return KM_OK;
}

// Centroids and labels in the caller's numbering (the context may hold its
// centroids in another order; Params::orig maps internal -> caller index).
cudaError_t centroids_in(kmeans_ctx *c, const float *src) {
    const Params &p = c->p;
    cudaStream_t s = c->stream;
    if (!p.orig)
        return cudaMemcpy2DAsync(p.C, (size_t)p.Dp * 4, src, (size_t)p.D * 4, (size_t)p.D * 4, p.K, cudaMemcpyDefault,
                                 s);
    const float *d = src;
    float *tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!is_device_ptr(src)) {
        e = pool_alloc(c->dev, reinterpret_cast<void **>(&tmp), (size_t)p.K * p.D * 4, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tmp, src, (size_t)p.K * p.D * 4, cudaMemcpyDefault, s);
        d = tmp;
    }
    if (e == cudaSuccess) e = launch_rows_in(d, p.D, p.K, p.Dp, p.orig, p.C, s, c->num_sms);
    if (tmp) cudaFreeAsync(tmp, s);
    return e;
}
cudaError_t centroids_out(kmeans_ctx *c, float *dst, cudaStream_t s) {
    const Params &p = c->p;
    if (!p.orig)
        return cudaMemcpy2DAsync(dst, (size_t)p.D * 4, p.C, (size_t)p.Dp * 4, (size_t)p.D * 4, p.K, cudaMemcpyDefault,
                                 s);
    const bool dev = is_device_ptr(dst);
    float *out = dst;
    cudaError_t e = cudaSuccess;
    if (!dev) e = pool_alloc(c->dev, reinterpret_cast<void **>(&out), (size_t)p.K * p.D * 4, s);
    if (e == cudaSuccess) e = launch_rows_out(p.C, p.Dp, p.D, p.K, p.orig, out, s, c->num_sms);
    if (!dev && e == cudaSuccess) e = cudaMemcpyAsync(dst, out, (size_t)p.K * p.D * 4, cudaMemcpyDeviceToHost, s);
    if (!dev && out) cudaFreeAsync(out, s);
    return e;
}
cudaError_t labels_out(kmeans_ctx *c, int32_t *dst, cudaStream_t s) {
    const Params &p = c->p;
    if (!p.orig) return cudaMemcpyAsync(dst, p.label, (size_t)p.N * 4, cudaMemcpyDefault, s);
    const bool dev = is_device_ptr(dst);
    int32_t *out = dst;
    cudaError_t e = cudaSuccess;
    if (!dev) e = pool_alloc(c->dev, reinterpret_cast<void **>(&out), (size_t)p.N * 4, s);
    if (e == cudaSuccess) e = launch_labels_out(p.label, p.N, p.orig, p.K, out, s, c->num_sms);
    if (!dev && e == cudaSuccess) e = cudaMemcpyAsync(dst, out, (size_t)p.N * 4, cudaMemcpyDeviceToHost, s);
    if (!dev && out) cudaFreeAsync(out, s);
    return e;
}

// One assignment (dense when `dense`, filtered otherwise), stream-ordered.
// Cluster statistics after an assignment: the full recompute or the moved
// points' changes, chosen on the device.
cudaError_t enqueue_stats(kmeans_ctx *c, const Params &p, cudaStream_t s, int all_points, int respect_done) {
    const int n = c->num_sms;
    // the sorted path takes both modes (full recompute or moved points only,
    // chosen on the device); the per-point moves are for the other layouts
    if (stats_full_supported(p))
        return timed(c, s, KM_KERNEL_STATS, [&] { return launch_stats_full(p, s, all_points, respect_done, n); });
    return timed(c, s, KM_KERNEL_MOVES, [&] { return launch_apply_moves(p, s, all_points, respect_done, n); });
}

cudaError_t enqueue_assign(kmeans_ctx *c, const Params &p, cudaStream_t s, bool dense, bool first, int respect_done) {
    cudaError_t e;
    const int n = c->num_sms;
    if (dense) {
        e = timed(c, s, KM_KERNEL_DENSE, [&] {
            return c->use_tc ? launch_dense_tc(p, s, first, respect_done, n, c->smem_optin)
                             : launch_dense_assign(p, s, first, respect_done, n);
        });
        if (e != cudaSuccess) return e;
        if (c->use_tc) {
            e = timed(c, s, KM_KERNEL_SETTLE, [&] { return launch_settle(p, s, first, respect_done, n); });
            if (e != cudaSuccess) return e;
        }
        return enqueue_stats(c, p, s, (first || c->shard) ? 1 : 0, respect_done);
    }
    // filtered: global filter, then either the survivor kernel or -- when the
    // filter kernel finds too many survivors -- the dense pass (each of the
    // two exits at once when the device chose the other)
    e = timed(c, s, KM_KERNEL_FILTER, [&] { return launch_filter(p, s, respect_done, n); });
    if (e != cudaSuccess) return e;
    e = timed(c, s, KM_KERNEL_SURVIVOR, [&] { return launch_survivor(p, s, respect_done, n, c->smem_optin); });
    if (e != cudaSuccess) return e;
    e = timed(c, s, KM_KERNEL_DENSE, [&] {
        return c->use_tc ? launch_dense_tc(p, s, 0, respect_done, n, c->smem_optin, 1)
                         : launch_dense_assign(p, s, 0, respect_done, n, 1);
    });
    if (e != cudaSuccess) return e;
    if (c->use_tc) {  // no rows queued unless the dense pass ran
        e = timed(c, s, KM_KERNEL_SETTLE, [&] { return launch_settle(p, s, 0, respect_done, n); });
        if (e != cudaSuccess) return e;
    }
    // both the survivor kernel and the dense pass append to the moved-point list
    // (a seeded iteration 0 recomputes every cluster sum)
    return enqueue_stats(c, p, s, (first || c->shard) ? 1 : 0, respect_done);
}

cudaError_t enqueue_update(kmeans_ctx *c, const Params &p, cudaStream_t s, int final_only, int respect_done) {
    return timed(c, s, KM_KERNEL_UPDATE, [&] { return launch_update(p, s, final_only, respect_done); });
}

// Iteration 0 seeded by the learned proposal: predictions, the centroid
// table and the seeded bounds (the filtered assignment follows).
cudaError_t enqueue_proposal(kmeans_ctx *c, const Params &p, cudaStream_t s, int respect_done) {
    return timed(c, s, KM_KERNEL_PROPOSAL, [&] {
        if (mlp_predict_enqueue(c->net, p.X, p.N, c->pred, s) != KM_OK) return cudaErrorLaunchFailure;
        return launch_proposal_seed(p, c->pred, c->cc_table, s, respect_done, c->num_sms);
    });
}

// One full iteration: assignment, then update.
cudaError_t enqueue_iteration(kmeans_ctx *c, const Params &p, cudaStream_t s, bool first, int respect_done) {
    if (first && c->proposal && p.algo == KM_ALGO_FILTERED) {
        cudaError_t e = enqueue_proposal(c, p, s, respect_done);
        if (e != cudaSuccess) return e;
        e = enqueue_assign(c, p, s, false, true, respect_done);
        if (e != cudaSuccess) return e;
        return enqueue_update(c, p, s, 0, respect_done);
    }
    const bool dense = first || p.algo == KM_ALGO_LLOYD;
    cudaError_t e = enqueue_assign(c, p, s, dense, first, respect_done);
    if (e != cudaSuccess) return e;
    return enqueue_update(c, p, s, 0, respect_done);
}

// Record the fit graph: set_cond -> while(cond){ iteration } -> final
// assignment -> objective.
int build_fit_graph_impl(kmeans_ctx *c);
int build_fit_graph(kmeans_ctx *c) {
    c->capturing = true;
    int rc = build_fit_graph_impl(c);
    c->capturing = false;
    return rc;
}
int build_fit_graph_impl(kmeans_ctx *c) {
    cudaGraph_t g = nullptr;
    KP_CUDA(c, cudaGraphCreate(&g, 0));
    cudaGraphConditionalHandle h;
    KP_CUDA(c, cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    Params p = c->p;
    p.cond = (unsigned long long)h;

    KP_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_set_cond(p, c->cap_stream);
    cudaGraph_t g2 = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g2);
    KP_CUDA(c, e);
    KP_CUDA(c, e2);

    size_t nn = 0;
    KP_CUDA(c, cudaGraphGetNodes(g, nullptr, &nn));
    std::vector<cudaGraphNode_t> nodes(nn);
    KP_CUDA(c, cudaGraphGetNodes(g, nodes.data(), &nn));
    if (nn != 1) return set_err(c, KM_ECUDA, "unexpected graph prologue (%zu nodes)", nn);

    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond_node;
    KP_CUDA(c, cudaGraphAddNode(&cond_node, g, nodes.data(), nullptr, 1, &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];

    KP_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    e = enqueue_iteration(c, p, c->cap_stream, false, 1);
    e2 = cudaStreamEndCapture(c->cap_stream, &body);
    KP_CUDA(c, e);
    KP_CUDA(c, e2);

    // epilogue: final assignment to the returned centroids, then J
    Params pf = c->p;
    pf.cond = 0;
    KP_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, g, &cond_node, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    e = enqueue_assign(c, pf, c->cap_stream, pf.algo == KM_ALGO_LLOYD, false, 0);
    if (e == cudaSuccess) e = enqueue_update(c, pf, c->cap_stream, 1, 0);
    e2 = cudaStreamEndCapture(c->cap_stream, &g);
    KP_CUDA(c, e);
    KP_CUDA(c, e2);

    cudaGraphExec_t ex = nullptr;
    KP_CUDA(c, cudaGraphInstantiate(&ex, g, 0));
    c->graph = g;
    c->graph_exec = ex;
    c->cond = h;
    return KM_OK;
}

// Append one problem's whole fit to graph g as an independent chain:
// arm(max_iter, tol) -> [iteration 0] -> set_cond -> while(cond){ iteration }
// -> final assignment -> objective.  Used by the batched form, which records
// every problem's chain into one graph.
int append_fit_chain(kmeans_ctx *c, cudaGraph_t g, int max_iter, double tol, bool first) {
    c->capturing = true;
    struct Off {
        kmeans_ctx *c;
        ~Off() { c->capturing = false; }
    } off{c};
    cudaGraphConditionalHandle h;
    KP_CUDA(c, cudaGraphConditionalHandleCreate(&h, g, 0, 0));
    Params p = c->p;
    p.tcap = c->tcap;
    Params pc = p;
    pc.cond = (unsigned long long)h;

    KP_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, g, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = launch_arm(p, c->cap_stream, max_iter, tol);
    if (e == cudaSuccess && first) e = enqueue_iteration(c, p, c->cap_stream, true, 1);
    if (e == cudaSuccess) e = launch_set_cond(pc, c->cap_stream);
    std::vector<cudaGraphNode_t> leaf;
    if (e == cudaSuccess) {
        cudaStreamCaptureStatus st;
        const cudaGraphNode_t *deps = nullptr;
        size_t nd = 0;
        e = cudaStreamGetCaptureInfo(c->cap_stream, &st, nullptr, nullptr, &deps, nullptr, &nd);
        if (e == cudaSuccess) leaf.assign(deps, deps + nd);
    }
    cudaGraph_t g2 = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->cap_stream, &g2);
    KP_CUDA(c, e);
    KP_CUDA(c, e2);
    if (leaf.empty()) return set_err(c, KM_ECUDA, "empty chain prologue");

    cudaGraphNodeParams cp = {cudaGraphNodeTypeConditional};
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cond_node;
    KP_CUDA(c, cudaGraphAddNode(&cond_node, g, leaf.data(), nullptr, leaf.size(), &cp));
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    KP_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    e = enqueue_iteration(c, pc, c->cap_stream, false, 1);
    e2 = cudaStreamEndCapture(c->cap_stream, &body);
    KP_CUDA(c, e);
    KP_CUDA(c, e2);

    KP_CUDA(c, cudaStreamBeginCaptureToGraph(c->cap_stream, g, &cond_node, nullptr, 1, cudaStreamCaptureModeThreadLocal));
    e = enqueue_assign(c, p, c->cap_stream, p.algo == KM_ALGO_LLOYD, false, 0);
    if (e == cudaSuccess) e = enqueue_update(c, p, c->cap_stream, 1, 0);
    e2 = cudaStreamEndCapture(c->cap_stream, &g);
    KP_CUDA(c, e);
    KP_CUDA(c, e2);
    return KM_OK;
}

int check_ctx(kmeans_ctx *c) {
    if (!c) return KM_EINVAL;
    if (c->broken) return set_err(c, KM_ESTATE, "context unusable after an earlier failure");
    return KM_OK;
}

}  // namespace

cudaError_t kp::pool_alloc(int dev, void **p, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool;
    cudaError_t e = lib_pool(dev, &pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(p, std::max<size_t>(bytes, 1), pool, s);
}

extern "C" {

KM_API void kmeans_default_options(kmeans_options *opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->algo = KM_ALGO_FILTERED;
    opt->grouping = KM_GROUP_CONTIGUOUS;
}

KM_API int kmeans_init(kmeans_ctx **out, const float *X, int64_t N, int32_t D, int32_t K, int32_t G,
                       const float *init_centroids, const kmeans_options *opt) {
    if (!out) return set_err(nullptr, KM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!X || !init_centroids) return set_err(nullptr, KM_EINVAL, "X or init_centroids is NULL");
    if (N < 1 || N >= (int64_t)1 << 31) return set_err(nullptr, KM_EINVAL, "N=%lld out of range [1, 2^31)", (long long)N);
    if (D < 1 || D > 4096) return set_err(nullptr, KM_EINVAL, "D=%d out of range [1, 4096]", D);
    if (K < 1 || K > 65535 || (int64_t)K > N) return set_err(nullptr, KM_EINVAL, "K=%d must be in [1, min(N, 65535)]", K);
    if (G < 1 || G > K) return set_err(nullptr, KM_EINVAL, "G=%d must be in [1, K]", G);
    kmeans_options o;
    kmeans_default_options(&o);
    if (opt) o = *opt;
    if (o.algo != KM_ALGO_FILTERED && o.algo != KM_ALGO_LLOYD) return set_err(nullptr, KM_EINVAL, "unknown algo %d", o.algo);
    if (o.grouping != KM_GROUP_CONTIGUOUS && o.grouping != KM_GROUP_CLUSTERED)
        return set_err(nullptr, KM_EINVAL, "unknown grouping %d", o.grouping);
    if (o.dense != KM_DENSE_AUTO && o.dense != KM_DENSE_FP32) return set_err(nullptr, KM_EINVAL, "unknown dense %d", o.dense);
    if (!(o.dense_switch >= 0.0f)) return set_err(nullptr, KM_EINVAL, "dense_switch must be >= 0");
    if (o.dtype != KM_DTYPE_F32 && o.dtype != KM_DTYPE_BF16) return set_err(nullptr, KM_EINVAL, "unknown dtype %d", o.dtype);
    if (o.pad0 || o.pad1) return set_err(nullptr, KM_EINVAL, "reserved option fields must be zero");
    for (int i = 0; i < 3; ++i)
        if (o.reserved[i]) return set_err(nullptr, KM_EINVAL, "reserved option fields must be zero");
    if (o.surv_grab != 0 && (o.surv_grab < 32 || o.surv_grab > 1024 || o.surv_grab % 32 != 0))
        return set_err(nullptr, KM_EINVAL, "surv_grab must be 0 or a multiple of 32 in [32, 1024]");

    kmeans_ctx *c = new (std::nothrow) kmeans_ctx();
    if (!c) return set_err(nullptr, KM_ENOMEM, "host allocation failed");
    int rc = KM_OK;
    auto fail = [&](int code) {
        snprintf(g_init_error, sizeof(g_init_error), "%s", c->err);
        kmeans_destroy(c);
        return code;
    };
#define INIT_CUDA(call)                                                                             \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) {                                                                    \
            set_err(c, e_ == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA, "%s failed: %s",     \
                    #call, cudaGetErrorString(e_));                                                 \
            return fail(e_ == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA);                    \
        }                                                                                           \
    } while (0)

    c->opt = o;
    c->stream = static_cast<cudaStream_t>(o.stream);
    INIT_CUDA(cudaGetDevice(&c->dev));
    INIT_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev));
    int optin = 0;
    INIT_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev));
    c->smem_optin = (size_t)optin;
    INIT_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    INIT_CUDA(cudaMallocHost(&c->ctrl_host, sizeof(Ctrl)));

    // clustered grouping: plain Lloyd over the K initial centroids, seeded by
    // their first G rows, 5 iterations (kp_group.cu); empty groups are
    // dropped and the centroids are ordered group by group (ascending caller
    // index within a group), so that every kernel sees each group as a run
    // of indices.  Ties between equal distances are broken by the caller's
    // index (Params::orig).
    std::vector<int32_t> cl_orig, cl_grp, cl_start;
    if (o.grouping == KM_GROUP_CLUSTERED) {
        cudaStream_t s0 = c->stream;
        float *cd = nullptr;
        float *cen = nullptr;
        int32_t *gd = nullptr;
        std::vector<int32_t> lab(K);
        cudaError_t e = pool_alloc(c->dev, reinterpret_cast<void **>(&cd), (size_t)K * D * 4, s0);
        if (e == cudaSuccess) e = pool_alloc(c->dev, reinterpret_cast<void **>(&cen), (size_t)G * D * 4, s0);
        if (e == cudaSuccess) e = pool_alloc(c->dev, reinterpret_cast<void **>(&gd), (size_t)K * 4, s0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(cd, init_centroids, (size_t)K * D * 4, cudaMemcpyDefault, s0);
        if (e == cudaSuccess) e = launch_clustered_groups(cd, K, D, G, 5, gd, cen, s0, c->num_sms);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lab.data(), gd, (size_t)K * 4, cudaMemcpyDeviceToHost, s0);
        for (void *q : {(void *)cd, (void *)cen, (void *)gd})
            if (q) cudaFreeAsync(q, s0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s0);
        INIT_CUDA(e);
        std::vector<int32_t> cnt(G, 0), newid(G, -1);
        for (int k = 0; k < K; ++k) {
            if ((unsigned)lab[k] >= (unsigned)G) {
                set_err(c, KM_ECUDA, "grouping produced a label out of range");
                return fail(KM_ECUDA);
            }
            ++cnt[lab[k]];
        }
        int ge = 0;
        for (int g = 0; g < G; ++g)
            if (cnt[g]) newid[g] = ge++;
        cl_start.assign(ge + 1, 0);
        for (int g = 0; g < G; ++g)
            if (cnt[g]) cl_start[newid[g] + 1] = cnt[g];
        for (int g = 0; g < ge; ++g) cl_start[g + 1] += cl_start[g];
        std::vector<int32_t> pos(cl_start.begin(), cl_start.end() - 1);
        cl_orig.resize(K);
        cl_grp.resize(K);
        for (int k = 0; k < K; ++k) {
            const int g = newid[lab[k]];
            const int kk = pos[g]++;
            cl_orig[kk] = k;
            cl_grp[kk] = g;
        }
        G = ge;
    }

    Params &p = c->p;
    p.N = N;
    p.D = D;
    p.K = K;
    p.G = G;
    p.Dp = padded_stride_c(D);
    p.Gp = (G + 3) & ~3;
    p.algo = o.algo;
    const bool filtered = o.algo == KM_ALGO_FILTERED;

    // X: borrowed when FP32 on the device, copied otherwise (bfloat16: an
    // exact FP32 copy)
    const float *x_host_dev = nullptr;  // host X readable by the device (copied later)
    if (o.dtype == KM_DTYPE_BF16) {
        INIT_CUDA(dalloc(c, &c->X_own, (size_t)N * D));
        const uint16_t *xb = reinterpret_cast<const uint16_t *>(X);
        uint16_t *tmp = nullptr;
        if (!is_device_ptr(X)) {
            INIT_CUDA(pool_alloc(c->dev, reinterpret_cast<void **>(&tmp), (size_t)N * D * 2, c->stream));
            INIT_CUDA(cudaMemcpyAsync(tmp, X, (size_t)N * D * 2, cudaMemcpyDefault, c->stream));
            xb = tmp;
        }
        INIT_CUDA(launch_bf16_to_f32(xb, (int64_t)N * D, c->X_own, c->stream, c->num_sms));
        if (tmp) INIT_CUDA(cudaFreeAsync(tmp, c->stream));
        p.X = c->X_own;
    } else if (is_device_ptr(X)) {
        p.X = X;
    } else {
        INIT_CUDA(dalloc(c, &c->X_own, (size_t)N * D));
        // page-locked host memory the device can read: the tensor-core
        // split below copies and splits in one pass over it; otherwise copy
        cudaPointerAttributes pa;
        if (cudaPointerGetAttributes(&pa, X) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer &&
            D % 4 == 0 && (reinterpret_cast<uintptr_t>(pa.devicePointer) & 15) == 0)
            x_host_dev = static_cast<const float *>(pa.devicePointer);
        else
            INIT_CUDA(cudaMemcpyAsync(c->X_own, X, (size_t)N * D * 4, cudaMemcpyDefault, c->stream));
        cudaGetLastError();
        p.X = c->X_own;
    }
    p.x_vec4 = (D % 4 == 0) && ((reinterpret_cast<uintptr_t>(p.X) & 15) == 0);

    INIT_CUDA(dalloc(c, &p.label, (size_t)N));
    INIT_CUDA(dalloc(c, &p.moved, (size_t)N));
    INIT_CUDA(dalloc(c, &p.moved_old, (size_t)N));
    INIT_CUDA(dalloc(c, &p.perm, (size_t)N));
    INIT_CUDA(dalloc(c, &p.slab, (size_t)N));
    INIT_CUDA(dalloc(c, &p.hcount, (size_t)K));
    INIT_CUDA(dalloc(c, &p.hcur, (size_t)K));
    INIT_CUDA(cudaMemsetAsync(p.hcount, 0, (size_t)K * 4, c->stream));
    p.hist_smem_k = 8192;
    if (filtered) {
        INIT_CUDA(dalloc(c, &p.u, (size_t)N));
        INIT_CUDA(dalloc(c, &p.lbg, (size_t)N));
        INIT_CUDA(dalloc(c, &p.stamp, (size_t)N));
        INIT_CUDA(dalloc(c, &p.lb, (size_t)N * p.Gp));
        INIT_CUDA(cudaMemsetAsync(p.lb, 0, (size_t)N * p.Gp * 4, c->stream));  // padding columns stay 0
        INIT_CUDA(dalloc(c, &p.queue, (size_t)N));
        // survivor queue buckets: labels >> bshift, at most 4096 buckets
        p.bshift = 0;
        while (((K - 1) >> p.bshift) >= 4096) ++p.bshift;
        p.nbucket = ((K - 1) >> p.bshift) + 1;
        INIT_CUDA(dalloc(c, &p.bcount, (size_t)p.nbucket));
        INIT_CUDA(dalloc(c, &p.bcursor, (size_t)p.nbucket));
        INIT_CUDA(cudaMemsetAsync(p.bcount, 0, (size_t)p.nbucket * 4, c->stream));
    }
    INIT_CUDA(dalloc(c, &p.C, (size_t)K * p.Dp));
    INIT_CUDA(dalloc(c, &p.S, (size_t)K * D));
    INIT_CUDA(dalloc(c, &p.Q, (size_t)K));
    INIT_CUDA(dalloc(c, &p.R, (size_t)K * p.Dp));
    INIT_CUDA(dalloc(c, &p.cnt, (size_t)K));
    INIT_CUDA(dalloc(c, &p.delta, (size_t)K));
    INIT_CUDA(dalloc(c, &p.Jk, (size_t)K));
    int32_t *grp, *gstart;
    INIT_CUDA(dalloc(c, &grp, (size_t)K));
    INIT_CUDA(dalloc(c, &gstart, (size_t)G + 1));
    p.grp = grp;
    p.gstart = gstart;
    INIT_CUDA(dalloc(c, &p.ctrl, 1));
    INIT_CUDA(dalloc(c, &p.stats, (size_t)kStatsCap + 1));  // + the final assignment
    INIT_CUDA(dalloc(c, &c->flag_dev, 1));
    c->tcap = 64;
    INIT_CUDA(dalloc(c, &p.Dc, (size_t)c->tcap * K));
    INIT_CUDA(dalloc(c, &p.Dg, (size_t)c->tcap * p.Gp));
    INIT_CUDA(dalloc(c, &p.Dm, (size_t)c->tcap));
    p.tcap = c->tcap;

    cudaStream_t s = c->stream;
    INIT_CUDA(cudaMemsetAsync(p.C, 0, (size_t)K * p.Dp * 4, s));
    if (!cl_orig.empty()) {
        int32_t *orig;
        INIT_CUDA(dalloc(c, &orig, (size_t)K));
        // (cl_orig, like the group tables below, lives until the final wait)
        INIT_CUDA(cudaMemcpyAsync(orig, cl_orig.data(), (size_t)K * 4, cudaMemcpyHostToDevice, s));
        p.orig = orig;
    }
    INIT_CUDA(centroids_in(c, init_centroids));
    INIT_CUDA(cudaMemcpyAsync(p.R, p.C, (size_t)K * p.Dp * 4, cudaMemcpyDeviceToDevice, s));
    INIT_CUDA(cudaMemsetAsync(p.S, 0, (size_t)K * D * 8, s));
    INIT_CUDA(cudaMemsetAsync(p.Q, 0, (size_t)K * 8, s));
    INIT_CUDA(cudaMemsetAsync(p.cnt, 0, (size_t)K * 8, s));
    INIT_CUDA(cudaMemsetAsync(p.Dc, 0, (size_t)c->tcap * K * 4, s));
    INIT_CUDA(cudaMemsetAsync(p.Dg, 0, (size_t)c->tcap * p.Gp * 4, s));
    INIT_CUDA(cudaMemsetAsync(p.Dm, 0, (size_t)c->tcap * 4, s));
    INIT_CUDA(cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), s));
    INIT_CUDA(cudaMemsetAsync(p.stats, 0, sizeof(kmeans_iter_stats) * (kStatsCap + 1), s));

    // contiguous grouping: centroid j -> floor(j G / K); clustered: the runs made above
    std::vector<int32_t> hg(K), hs(G + 1);
    if (!cl_grp.empty()) {
        hg = cl_grp;
        hs = cl_start;
    } else {
        for (int j = 0; j < K; ++j) hg[j] = (int32_t)(((int64_t)j * G) / K);
        for (int g = 0; g <= G; ++g) hs[g] = (int32_t)(((int64_t)g * K + G - 1) / G);
    }
    INIT_CUDA(cudaMemcpyAsync(grp, hg.data(), (size_t)K * 4, cudaMemcpyHostToDevice, s));
    INIT_CUDA(cudaMemcpyAsync(gstart, hs.data(), (size_t)(G + 1) * 4, cudaMemcpyHostToDevice, s));

    // FP32 distance error bound: s_fp32 in s [(1-u)^2 (1-g_D), (1+u)^2 (1+g_D)],
    // u = 2^-24, g_D = D u / (1 - D u) (recursive or tree summation of D
    // squares, Higham Thm 4.4): eps = (D + 4) u with margin.
    const double u24 = std::ldexp(1.0, -24);
    const double eps = (D + 4) * u24 * (1.0 + 1.0 / 1024);
    p.eps_hi = f32_up(1.0 + 2.0 * eps);
    p.eps_lo = f32_dn(1.0 - eps);
    p.tiny = std::ldexp((float)(D + 4), -149);
    c->use_tc = o.dense == KM_DENSE_AUTO && (reinterpret_cast<uintptr_t>(p.X) & 15) == 0 &&
                (dense_tc_eligible(p, c->smem_optin) || dense_tcb_eligible(p, c->smem_optin));
    // default switch: the tensor-core dense pass costs about as much as the
    // survivor kernel with 70% of the points surviving; the FP32 one more
    p.dense_frac = o.dense_switch > 0.0f ? o.dense_switch : (c->use_tc ? 0.7f : 0.9f);
    p.surv_grab = o.surv_grab;
    if (c->use_tc && !filtered && K > 256) {
        // plain Lloyd with streamed centroid blocks: the pass still writes
        // group bounds, so that the exact settle of a row visits only the
        // groups that can hold its winner instead of all K centroids
        INIT_CUDA(dalloc(c, &p.lb, (size_t)N * p.Gp));
        INIT_CUDA(cudaMemsetAsync(p.lb, 0, (size_t)N * p.Gp * 4, s));
    }
    if (c->use_tc) {
        // the tensor-core passes work on x - mu and c - mu, mu the mean of the
        // initial centroids: distances do not change, but the error window of
        // the bfloat16 products scales with ||x - mu|| ||c - mu|| instead of
        // ||x|| ||c||, which matters for data far from the origin
        // (computed on the device from the context's copy of C^0, without a
        // round trip through the host)
        float *mu;
        INIT_CUDA(dalloc(c, &mu, (size_t)p.Dp));
        INIT_CUDA(launch_centroid_mean(p.C, K, D, p.Dp, mu, s));
        p.mu = mu;
        // x - mu and c - mu are each rounded once (relative 2^-24 per coordinate):
        // |s' - s| <= 2 u (1 + u) R^2 + 3 (u (1 + u) R)^2 for R = ||x - mu|| + ||c - mu||
        p.e_cen = (float)(std::ldexp(1.0, -23) * 1.01);
    }
    if (c->use_tc) {  // the two bfloat16 halves of X, made once
        uint16_t *xh, *xl;
        const int Dt = tc_dim(D);  // zero-padded width of the operand copies
        float *xnorm;
        INIT_CUDA(dalloc(c, &xh, (size_t)N * Dt));
        INIT_CUDA(dalloc(c, &xl, (size_t)N * Dt));
        INIT_CUDA(dalloc(c, &xnorm, (size_t)N));
        // from the host copy when X is still there (the FP32 copy is made in the same pass)
        INIT_CUDA(launch_split_x(x_host_dev ? x_host_dev : p.X, N, D, Dt, xh, xl, s, c->num_sms,
                                 x_host_dev ? c->X_own : nullptr, p.mu, xnorm));
        x_host_dev = nullptr;
        p.Xh = xh;
        p.Xl = xl;
        p.xnorm = xnorm;
        SettleReq *sq;
        INIT_CUDA(dalloc(c, &sq, (size_t)N));
        p.sreq = sq;
        uint32_t *sb;
        int32_t *sqq;
        INIT_CUDA(dalloc(c, &sb, (size_t)((N + 127) / 128) * 4));
        INIT_CUDA(cudaMemsetAsync(sb, 0, (size_t)((N + 127) / 128) * 16, s));
        INIT_CUDA(dalloc(c, &sqq, (size_t)N));
        p.sbits = sb;
        p.squeue = sqq;
        if (K > 256) {  // the centroid blocks stream from a split copy made each pass
            const int kp = dense_tcb_kp(p);
            INIT_CUDA(dalloc(c, &p.Ch, (size_t)kp * Dt));
            INIT_CUDA(dalloc(c, &p.Cl, (size_t)kp * Dt));
            INIT_CUDA(dalloc(c, &p.cnorm, (size_t)K));
        }
    }

    if (x_host_dev) INIT_CUDA(cudaMemcpyAsync(c->X_own, X, (size_t)N * D * 4, cudaMemcpyDefault, s));
    if (o.validate) {
        INIT_CUDA(cudaMemsetAsync(c->flag_dev, 0, 4, s));
        INIT_CUDA(launch_check_finite(p.X, N * D, c->flag_dev, s, c->num_sms));
        INIT_CUDA(launch_check_finite(p.C, (int64_t)K * p.Dp, c->flag_dev, s, c->num_sms));
        int h = 0;
        INIT_CUDA(cudaMemcpyAsync(&h, c->flag_dev, 4, cudaMemcpyDeviceToHost, s));
        INIT_CUDA(cudaStreamSynchronize(s));
        if (h) {
            set_err(c, KM_EINVAL, "X or init_centroids holds NaN or Inf");
            return fail(KM_EINVAL);
        }
    }
    // the fit graph, recorded now: the host's recording overlaps the device
    // work enqueued above (with a host X, its copy and split), which the
    // synchronisation below waits for in any case
    if (!t_ctx_in_batch && !o.profile) {
        const int grc = build_fit_graph(c);
        if (grc != KM_OK) return fail(grc);
    }
    INIT_CUDA(cudaStreamSynchronize(s));
    *out = c;
    (void)rc;
    return KM_OK;
#undef INIT_CUDA
}

KM_API int kmeans_iterate(kmeans_ctx *c, kmeans_iter_stats *stats) {
    int rc = check_ctx(c);
    if (rc) return rc;
    DeviceGuard dg(c->dev);
    if ((rc = ensure_tables(c, 2))) return rc;
    Params &p = c->p;
    p.tcap = c->tcap;
    KP_CUDA(c, timed(c, c->stream, KM_KERNEL_OTHER, [&] { return launch_arm(p, c->stream, 1, 0.0); }));
    KP_CUDA(c, enqueue_iteration(c, p, c->stream, c->t_host == 0, 0));
    const int t = c->t_host;
    if ((rc = sync_and_check(c))) return rc;
    if (stats) KP_CUDA(c, cudaMemcpy(stats, p.stats + (t % kStatsCap), sizeof(*stats), cudaMemcpyDeviceToHost));
    return KM_OK;
}

KM_API int kmeans_shard_assign(kmeans_ctx *c, double tol, double *S, double *Q, int64_t *cnt,
                               int64_t *n_changed) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!S || !Q || !cnt || !n_changed) return set_err(c, KM_EINVAL, "a pointer argument is NULL");
    if (!(tol >= 0.0)) return set_err(c, KM_EINVAL, "tol must be >= 0");
    if (c->shard_pending) return set_err(c, KM_ESTATE, "the previous shard assignment has not been updated");
    if (c->proposal) return set_err(c, KM_EINVAL, "sharded iterations do not take a learned proposal");
    DeviceGuard dg(c->dev);
    if ((rc = ensure_tables(c, 2))) return rc;
    Params &p = c->p;
    p.tcap = c->tcap;
    cudaStream_t s = c->stream;
    c->shard = true;
    // a stop rule without an iteration budget: the caller stops on stats.done
    KP_CUDA(c, timed(c, s, KM_KERNEL_OTHER, [&] { return launch_arm(p, s, 1 << 30, tol); }));
    const bool first = c->t_host == 0;
    KP_CUDA(c, enqueue_assign(c, p, s, first || p.algo == KM_ALGO_LLOYD, first, 0));
    if ((rc = sync_and_check(c))) return rc;
    KP_CUDA(c, cudaMemcpyAsync(S, p.S, (size_t)p.K * p.D * 8, cudaMemcpyDefault, s));
    KP_CUDA(c, cudaMemcpyAsync(Q, p.Q, (size_t)p.K * 8, cudaMemcpyDefault, s));
    KP_CUDA(c, cudaMemcpyAsync(cnt, p.cnt, (size_t)p.K * 8, cudaMemcpyDefault, s));
    KP_CUDA(c, cudaStreamSynchronize(s));
    *n_changed = (int64_t)c->ctrl_host->n_changed;
    c->shard_pending = true;
    return KM_OK;
}

KM_API int kmeans_shard_update(kmeans_ctx *c, int32_t final_pass, const double *S, const double *Q,
                               const int64_t *cnt, int64_t n_changed, kmeans_iter_stats *stats, double *objective) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!S || !Q || !cnt) return set_err(c, KM_EINVAL, "a pointer argument is NULL");
    if (!c->shard_pending) return set_err(c, KM_ESTATE, "no shard assignment is waiting for its update");
    if (n_changed < 0) return set_err(c, KM_EINVAL, "n_changed must be >= 0");
    DeviceGuard dg(c->dev);
    Params &p = c->p;
    cudaStream_t s = c->stream;
    KP_CUDA(c, cudaMemcpyAsync(p.S, S, (size_t)p.K * p.D * 8, cudaMemcpyDefault, s));
    KP_CUDA(c, cudaMemcpyAsync(p.Q, Q, (size_t)p.K * 8, cudaMemcpyDefault, s));
    KP_CUDA(c, cudaMemcpyAsync(p.cnt, cnt, (size_t)p.K * 8, cudaMemcpyDefault, s));
    const unsigned long long nc = (unsigned long long)n_changed;
    KP_CUDA(c, cudaMemcpyAsync(&p.ctrl->n_changed, &nc, 8, cudaMemcpyHostToDevice, s));
    c->shard_pending = false;
    const int t = c->t_host;
    KP_CUDA(c, enqueue_update(c, p, s, final_pass ? 1 : 0, 0));
    if ((rc = sync_and_check(c))) return rc;
    const int slot = final_pass ? kStatsCap : (t % kStatsCap);
    if (stats) KP_CUDA(c, cudaMemcpy(stats, p.stats + slot, sizeof(*stats), cudaMemcpyDeviceToHost));
    if (final_pass && objective) KP_CUDA(c, cudaMemcpy(objective, &p.ctrl->jfinal, 8, cudaMemcpyDefault));
    if (final_pass) c->have_final = true;
    return KM_OK;
}

KM_API int kmeans_fit(kmeans_ctx *c, int32_t max_iter, double tol, int32_t *labels, float *centroids,
                      double *objective, int32_t *n_iter) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (max_iter < 0 || !(tol >= 0.0)) return set_err(c, KM_EINVAL, "max_iter must be >= 0 and tol >= 0");
    DeviceGuard dg(c->dev);
    if ((rc = ensure_tables(c, max_iter + 2))) return rc;
    Params &p = c->p;
    p.tcap = c->tcap;
    KP_CUDA(c, timed(c, c->stream, KM_KERNEL_OTHER, [&] { return launch_arm(p, c->stream, max_iter, tol); }));
    if (c->t_host == 0 && max_iter == 0) {
        // nothing to iterate and no bounds yet: a dense assignment to C^0
        KP_CUDA(c, enqueue_assign(c, p, c->stream, true, true, 0));
        KP_CUDA(c, enqueue_update(c, p, c->stream, 1, 0));
    } else if (c->opt.profile) {
        // launch by launch, reading the stop rule back after each iteration
        if (c->t_host == 0) KP_CUDA(c, enqueue_iteration(c, p, c->stream, true, 1));
        for (;;) {
            if ((rc = sync_and_check(c))) return rc;
            if (c->ctrl_host->done) break;
            KP_CUDA(c, enqueue_iteration(c, p, c->stream, false, 1));
        }
        KP_CUDA(c, enqueue_assign(c, p, c->stream, p.algo == KM_ALGO_LLOYD, false, 0));
        KP_CUDA(c, enqueue_update(c, p, c->stream, 1, 0));
    } else {
        if (!c->graph_exec && (rc = build_fit_graph(c))) return rc;
        if (c->t_host == 0) KP_CUDA(c, enqueue_iteration(c, p, c->stream, true, 1));
        KP_CUDA(c, cudaGraphLaunch(c->graph_exec, c->stream));
    }
    if ((rc = sync_and_check(c))) return rc;
    cudaStream_t s = c->stream;
    if (labels) KP_CUDA(c, labels_out(c, labels, s));
    if (centroids) KP_CUDA(c, centroids_out(c, centroids, s));
    if (objective) KP_CUDA(c, cudaMemcpyAsync(objective, &p.ctrl->jfinal, 8, cudaMemcpyDefault, s));
    KP_CUDA(c, cudaStreamSynchronize(s));
    c->have_final = true;
    if (n_iter) {
        int32_t ni = c->ctrl_host->fit_n_iter;
        if (is_device_ptr(n_iter)) KP_CUDA(c, cudaMemcpy(n_iter, &ni, 4, cudaMemcpyHostToDevice));
        else *n_iter = ni;
    }
    return KM_OK;
}

KM_API int kmeans_get_labels(kmeans_ctx *c, int32_t *labels) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!labels) return set_err(c, KM_EINVAL, "labels is NULL");
    DeviceGuard dg(c->dev);
    KP_CUDA(c, labels_out(c, labels, c->stream));
    KP_CUDA(c, cudaStreamSynchronize(c->stream));
    return KM_OK;
}

KM_API int kmeans_get_centroids(kmeans_ctx *c, float *C) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!C) return set_err(c, KM_EINVAL, "C is NULL");
    DeviceGuard dg(c->dev);
    KP_CUDA(c, centroids_out(c, C, c->stream));
    KP_CUDA(c, cudaStreamSynchronize(c->stream));
    return KM_OK;
}

KM_API int kmeans_get_stats(kmeans_ctx *c, int32_t t, kmeans_iter_stats *stats) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!stats) return set_err(c, KM_EINVAL, "stats is NULL");
    if (t == -1) {
        if (!c->have_final) return set_err(c, KM_ESTATE, "no kmeans_fit has finished");
    } else if (t < 0 || t >= c->t_host || t < c->t_host - kStatsCap) {
        return set_err(c, KM_EINVAL, "no statistics kept for iteration %d", t);
    }
    DeviceGuard dg(c->dev);
    const size_t slot = t == -1 ? (size_t)kStatsCap : (size_t)(t % kStatsCap);
    KP_CUDA(c, cudaMemcpyAsync(stats, c->p.stats + slot, sizeof(*stats), cudaMemcpyDefault, c->stream));
    KP_CUDA(c, cudaStreamSynchronize(c->stream));
    return KM_OK;
}

KM_API int kmeans_get_bounds(kmeans_ctx *c, float *u, float *lbg, float *lb) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (c->p.algo != KM_ALGO_FILTERED || c->t_host == 0)
        return set_err(c, KM_EINVAL, "bounds exist only for the filtered algorithm after an iteration");
    DeviceGuard dg(c->dev);
    const Params &p = c->p;
    float *outs[3] = {u, lbg, lb};
    size_t sizes[3] = {(size_t)p.N, (size_t)p.N, (size_t)p.N * p.G};
    float *dev[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < 3; ++i) {
        if (!outs[i]) continue;
        if (is_device_ptr(outs[i])) dev[i] = outs[i];
        else KP_CUDA(c, pool_alloc(c->dev, reinterpret_cast<void **>(&dev[i]), sizes[i] * 4, c->stream));
    }
    KP_CUDA(c, launch_bounds_out(p, c->stream, dev[0], dev[1], dev[2], c->num_sms));
    for (int i = 0; i < 3; ++i) {
        if (outs[i] && dev[i] != outs[i]) {
            KP_CUDA(c, cudaMemcpyAsync(outs[i], dev[i], sizes[i] * 4, cudaMemcpyDeviceToHost, c->stream));
            KP_CUDA(c, cudaFreeAsync(dev[i], c->stream));
        }
    }
    KP_CUDA(c, cudaStreamSynchronize(c->stream));
    return KM_OK;
}

KM_API int kmeans_get_kernel_count(const kmeans_ctx *c, int64_t *n) {
    if (!c || !n) return KM_EINVAL;
    *n = (int64_t)(c->kernels_base + (long long)c->ctrl_host->kernels);
    return KM_OK;
}

KM_API int kmeans_reset(kmeans_ctx *c, const float *init_centroids) {
    int rc = check_ctx(c);
    if (rc) return rc;
    if (!init_centroids) return set_err(c, KM_EINVAL, "init_centroids is NULL");
    DeviceGuard dg(c->dev);
    Params &p = c->p;
    cudaStream_t s = c->stream;
    if ((rc = sync_and_check(c))) return rc;
    c->kernels_base += (long long)c->ctrl_host->kernels;
    KP_CUDA(c, centroids_in(c, init_centroids));
    KP_CUDA(c, cudaMemcpyAsync(p.R, p.C, (size_t)p.K * p.Dp * 4, cudaMemcpyDeviceToDevice, s));
    c->shard_pending = false;
    KP_CUDA(c, cudaMemsetAsync(p.S, 0, (size_t)p.K * p.D * 8, s));
    KP_CUDA(c, cudaMemsetAsync(p.Q, 0, (size_t)p.K * 8, s));
    KP_CUDA(c, cudaMemsetAsync(p.cnt, 0, (size_t)p.K * 8, s));
    KP_CUDA(c, cudaMemsetAsync(p.Dc, 0, (size_t)c->tcap * p.K * 4, s));
    KP_CUDA(c, cudaMemsetAsync(p.Dg, 0, (size_t)c->tcap * p.Gp * 4, s));
    KP_CUDA(c, cudaMemsetAsync(p.Dm, 0, (size_t)c->tcap * 4, s));
    KP_CUDA(c, cudaMemsetAsync(p.ctrl, 0, sizeof(Ctrl), s));
    KP_CUDA(c, cudaMemsetAsync(p.stats, 0, sizeof(kmeans_iter_stats) * (kStatsCap + 1), s));
    if (p.bcount) KP_CUDA(c, cudaMemsetAsync(p.bcount, 0, (size_t)p.nbucket * 4, s));
    if (p.hcount) KP_CUDA(c, cudaMemsetAsync(p.hcount, 0, (size_t)p.K * 4, s));
    KP_CUDA(c, cudaStreamSynchronize(s));
    memset(c->ctrl_host, 0, sizeof(Ctrl));
    c->t_host = 0;
    c->have_final = false;
    c->v_host = 0;
    for (int k = 0; k < KM_KERNEL_KINDS; ++k) {
        c->prof_ms[k] = 0.0;
        c->prof_n[k] = 0;
    }
    return KM_OK;
}

KM_API int kmeans_get_profile(kmeans_ctx *c, int32_t kind, int64_t *launches, double *ms) {
    if (!c || kind < 0 || kind >= KM_KERNEL_KINDS) return KM_EINVAL;
    if (launches) *launches = c->prof_n[kind];
    if (ms) *ms = c->prof_ms[kind];
    return KM_OK;
}

KM_API int kmeans_get_groups(kmeans_ctx *c, int32_t *grp, int32_t *n_groups) {
    int rc = check_ctx(c);
    if (rc) return rc;
    DeviceGuard dg(c->dev);
    const Params &p = c->p;
    if (n_groups) *n_groups = p.G;
    if (!grp) return KM_OK;
    std::vector<int32_t> g(p.K), o(p.K);
    KP_CUDA(c, cudaMemcpy(g.data(), p.grp, (size_t)p.K * 4, cudaMemcpyDeviceToHost));
    if (p.orig) KP_CUDA(c, cudaMemcpy(o.data(), p.orig, (size_t)p.K * 4, cudaMemcpyDeviceToHost));
    std::vector<int32_t> out(p.K);
    for (int k = 0; k < p.K; ++k) out[p.orig ? o[k] : k] = g[k];
    KP_CUDA(c, cudaMemcpy(grp, out.data(), (size_t)p.K * 4, cudaMemcpyDefault));
    return KM_OK;
}

KM_API int kmeans_get_iteration(const kmeans_ctx *c, int32_t *t) {
    if (!c || !t) return KM_EINVAL;
    *t = c->t_host;
    return KM_OK;
}

KM_API void kmeans_destroy(kmeans_ctx *c) {
    if (!c) return;
    DeviceGuard dg(c->dev);
    if (c->stream || c->cap_stream) cudaStreamSynchronize(c->stream);
    if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
    if (c->graph) cudaGraphDestroy(c->graph);
    if (c->net) kmeans_mlp_destroy(c->net);
    for (auto &q : c->pending) {
        c->ev_pool.push_back(q.a);
        c->ev_pool.push_back(q.b);
    }
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (void *q : c->allocs) cudaFreeAsync(q, c->stream);
    cudaStreamSynchronize(c->stream);
    if (c->ctrl_host) cudaFreeHost(c->ctrl_host);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

KM_API int kmeans_set_proposal(kmeans_ctx *c, const float *W1, const float *b1, const float *W2, const float *b2,
                               const float *W3, const float *b3, int32_t hidden) {
    int rc = check_ctx(c);
    if (rc) return rc;
    const bool none = !W1 && !b1 && !W2 && !b2 && !W3 && !b3;
    if (!none && (!W1 || !b1 || !W2 || !b2 || !W3 || !b3))
        return set_err(c, KM_EINVAL, "the proposal needs all six weight arrays (or none)");
    if (!none && c->p.algo != KM_ALGO_FILTERED)
        return set_err(c, KM_EINVAL, "the proposal seeds the filtered method's bounds (KM_ALGO_FILTERED only)");
    if (!none && (hidden < 1 || hidden > 256)) return set_err(c, KM_EINVAL, "hidden=%d outside [1, 256]", hidden);
    if (!none && (c->p.D > 256 || c->p.G > 512))
        return set_err(c, KM_EINVAL, "the proposal network takes D <= 256 and G <= 512");
    if (!none && c->p.orig)
        return set_err(c, KM_EINVAL, "the proposal predicts contiguous groups (KM_GROUP_CONTIGUOUS only)");
    DeviceGuard dg(c->dev);
    if ((rc = sync_and_check(c))) return rc;
    Params &p = c->p;
    if (c->net) {
        kmeans_mlp_destroy(c->net);
        c->net = nullptr;
    }
    c->proposal = false;
    if (!none) {
        kmeans_mlp *net = nullptr;
        if ((rc = kmeans_mlp_create(&net, p.D, hidden, p.G, 0, c->stream)))
            return set_err(c, rc, "proposal network: %s", kmeans_last_error(nullptr));
        c->net = net;
        if ((rc = kmeans_mlp_set_params(net, W1, b1, W2, b2, W3, b3)) || (rc = mlp_prepare(net, p.N)))
            return set_err(c, rc, "proposal network: %s", mlp_message(net));
        if (!c->pred) KP_CUDA(c, dalloc(c, &c->pred, (size_t)p.N));
        if (!c->cc_table) KP_CUDA(c, dalloc(c, &c->cc_table, (size_t)p.K * p.G));
        KP_CUDA(c, cudaStreamSynchronize(c->stream));
        c->proposal = true;
    }
    if (c->graph_exec) {  // recorded with the other iteration 0
        cudaGraphExecDestroy(c->graph_exec);
        cudaGraphDestroy(c->graph);
        c->graph_exec = nullptr;
        c->graph = nullptr;
    }
    return KM_OK;
}

KM_API int kmeans_mlp_predict(const float *X, int64_t N, int32_t D, const float *W1, const float *b1,
                              const float *W2, const float *b2, const float *W3, const float *b3, int32_t hidden,
                              int32_t classes, int32_t *pred, void *stream) {
    auto fail = [](int code, const char *msg) {
        set_thread_error(msg);
        return code;
    };
    if (!X || !W1 || !b1 || !W2 || !b2 || !W3 || !b3 || !pred) return fail(KM_EINVAL, "a pointer argument is NULL");
    if (N < 1 || D < 1 || D > 256 || hidden < 1 || hidden > 256 || classes < 1 || classes > 512)
        return fail(KM_EINVAL, "N >= 1, D in [1, 256], hidden in [1, 256] and classes in [1, 512] required");
    kmeans_mlp *net = nullptr;
    int rc = kmeans_mlp_create(&net, D, hidden, classes, 0, stream);
    if (rc) return rc;  // message already set for this thread
    if (!rc) rc = kmeans_mlp_set_params(net, W1, b1, W2, b2, W3, b3);
    if (!rc) rc = kmeans_mlp_predict_net(net, X, N, pred);
    if (rc) set_thread_error(kmeans_mlp_last_error(net));
    kmeans_mlp_destroy(net);
    return rc;
}

KM_API const char *kmeans_last_error(const kmeans_ctx *c) { return c ? c->err : g_init_error; }

KM_API void kmeans_debug_fail_alloc(int64_t after) { g_alloc_budget.store(after < 0 ? -1 : after); }

KM_API int64_t kmeans_launch_count(void) { return (int64_t)g_launches.load(std::memory_order_relaxed); }


// ---------------------------------------------------------------------------
// Batched form: many independent problems in one CUDA graph
// ---------------------------------------------------------------------------
}  // extern "C"

struct kmeans_batch {
    int dev = 0;
    cudaStream_t stream = nullptr;
    std::vector<kmeans_ctx *> ctx;
    std::vector<float *> c0;         // device copies of the initial centroids
    std::vector<float> sw;           // dense switch chosen per problem
    std::vector<int> dense, grab;    // dense engine and survivor queue schedule per problem
    cudaGraph_t graph = nullptr;     // every problem's fit, recorded once
    cudaGraphExec_t exec = nullptr;
    int rec_max_iter = -1;
    double rec_tol = -1.0;
    bool rec_first = false;
    std::vector<int> rec_tcap;
    char err[512] = "";
};

namespace {

int batch_err(kmeans_batch *b, int code, const char *fmt, ...) {
    char *buf = b ? b->err : g_init_error;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    if (b) set_thread_error(buf);
    return code;
}

// ---- autotuner: settings per size bucket ----------------------------------
// A bucket is (D, ceil log2 K, ceil log2 N).  For every bucket of the batch
// the tuner times short fits (10 iterations) of the bucket's largest problem
// and keeps the fastest in points x iterations per second, one setting at a
// time: the dense/filtered switch, then the dense engine, then the survivor
// queue schedule.  The choices are cached in a text file, one
// "D logK logN switch dense grab" line per bucket, and read back later.
struct TuneKey {
    int D, lk, ln;
    bool operator<(const TuneKey &o) const {
        return D != o.D ? D < o.D : (lk != o.lk ? lk < o.lk : ln < o.ln);
    }
};
struct TuneVal {
    float sw;
    int dense;
    int grab;
};
int ceil_log2(int64_t v) {
    int l = 0;
    while (((int64_t)1 << l) < v) ++l;
    return l;
}
const float kTuneSwitches[] = {0.5f, 0.7f, 0.9f, 1.0f};
const int kTuneGrabs[] = {32, 64, 128};

// points x iterations per second of a 10-iteration fit with these settings
// (< 0 when the settings do not run)
double tune_rate(const kmeans_problem &pr, const kmeans_options &base, const TuneVal &v, cudaStream_t s,
                 bool *used_tc) {
    kmeans_options o = base;
    o.dense_switch = v.sw;
    o.dense = v.dense;
    o.surv_grab = v.grab;
    o.stream = s;
    o.profile = 0;
    kmeans_ctx *c = nullptr;
    if (kmeans_init(&c, static_cast<const float *>(pr.X), pr.N, pr.D, pr.K, pr.G, pr.init_centroids, &o) != KM_OK)
        return -1.0;
    if (used_tc) *used_tc = c->use_tc;
    int32_t n_it = 0;
    kmeans_fit(c, 2, 0.0, nullptr, nullptr, nullptr, &n_it);  // warm-up: records the graph
    kmeans_reset(c, pr.init_centroids);
    cudaEvent_t a, z;
    cudaEventCreate(&a);
    cudaEventCreate(&z);
    cudaEventRecord(a, s);
    const int rc = kmeans_fit(c, 10, 0.0, nullptr, nullptr, nullptr, &n_it);
    cudaEventRecord(z, s);
    cudaEventSynchronize(z);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, z);
    cudaEventDestroy(a);
    cudaEventDestroy(z);
    kmeans_destroy(c);
    if (rc != KM_OK || ms <= 0.f) return -1.0;
    return (double)pr.N * (n_it + 1) / ms;
}

TuneVal tune_one(const kmeans_problem &pr, const kmeans_options &base, cudaStream_t s) {
    TuneVal best{0.0f, base.dense, 32};
    double best_rate = -1.0;
    bool tc = false;
    for (float sw : kTuneSwitches) {
        TuneVal v = best;
        v.sw = sw;
        const double r = tune_rate(pr, base, v, s, &tc);
        if (r > best_rate) {
            best_rate = r;
            best = v;
        }
    }
    if (base.dense == KM_DENSE_AUTO && tc) {  // the other engine, when the tensor cores take the shape
        TuneVal v = best;
        v.dense = KM_DENSE_FP32;
        const double r = tune_rate(pr, base, v, s, nullptr);
        if (r > best_rate) {
            best_rate = r;
            best = v;
        }
    }
    for (int g : kTuneGrabs) {
        if (g == best.grab) continue;
        TuneVal v = best;
        v.grab = g;
        const double r = tune_rate(pr, base, v, s, nullptr);
        if (r > best_rate) {
            best_rate = r;
            best = v;
        }
    }
    return best;
}

void tune_batch(const kmeans_problem *probs, int n, const kmeans_options &base, const char *cache, cudaStream_t s,
                std::vector<TuneVal> &out) {
    std::map<TuneKey, TuneVal> table;
    if (FILE *f = fopen(cache, "r")) {
        char line[256];
        while (fgets(line, sizeof(line), f)) {
            int D, lk, ln, dense = base.dense, grab = 32;
            float v;
            const int got = sscanf(line, "%d %d %d %f %d %d", &D, &lk, &ln, &v, &dense, &grab);
            if (got >= 4) table[{D, lk, ln}] = TuneVal{v, got >= 5 ? dense : base.dense, got >= 6 ? grab : 32};
        }
        fclose(f);
    }
    std::map<TuneKey, int> rep;  // the bucket's largest problem
    for (int i = 0; i < n; ++i) {
        const TuneKey k{probs[i].D, ceil_log2(probs[i].K), ceil_log2(probs[i].N)};
        auto it = rep.find(k);
        if (it == rep.end() || probs[i].N > probs[it->second].N) rep[k] = i;
    }
    bool grew = false;
    for (auto &kv : rep) {
        if (table.count(kv.first)) continue;
        table[kv.first] = tune_one(probs[kv.second], base, s);
        grew = true;
    }
    if (grew) {
        if (FILE *f = fopen(cache, "w")) {
            for (auto &kv : table)
                fprintf(f, "%d %d %d %.3f %d %d\n", kv.first.D, kv.first.lk, kv.first.ln, kv.second.sw,
                        kv.second.dense, kv.second.grab);
            fclose(f);
        }
    }
    out.resize(n);
    for (int i = 0; i < n; ++i) out[i] = table[{probs[i].D, ceil_log2(probs[i].K), ceil_log2(probs[i].N)}];
}

int batch_record(kmeans_batch *b, int max_iter, double tol, bool first) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaGraphCreate(&b->graph, 0);
    if (e != cudaSuccess) return batch_err(b, KM_ECUDA, "cudaGraphCreate: %s", cudaGetErrorString(e));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        int rc = append_fit_chain(b->ctx[i], b->graph, max_iter, tol, first);
        if (rc) return batch_err(b, rc, "problem %zu: %s", i, b->ctx[i]->err);
    }
    e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return batch_err(b, KM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
    b->rec_max_iter = max_iter;
    b->rec_tol = tol;
    b->rec_first = first;
    b->rec_tcap.resize(b->ctx.size());
    for (size_t i = 0; i < b->ctx.size(); ++i) b->rec_tcap[i] = b->ctx[i]->tcap;
    return KM_OK;
}

}  // namespace

extern "C" {

KM_API int kmeans_batch_init(kmeans_batch **out, int32_t n_problems, const kmeans_problem *problems,
                             const kmeans_options *opt, const char *tune_cache) {
    if (!out) return batch_err(nullptr, KM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_problems < 1 || !problems) return batch_err(nullptr, KM_EINVAL, "n_problems must be >= 1 with a problem array");
    kmeans_options base;
    if (opt) base = *opt;
    else kmeans_default_options(&base);
    if (base.profile) return batch_err(nullptr, KM_EINVAL, "profile is not supported in a batch");
    kmeans_batch *b = new kmeans_batch;
    cudaGetDevice(&b->dev);
    b->stream = static_cast<cudaStream_t>(base.stream);
    std::vector<TuneVal> tv(n_problems, TuneVal{base.dense_switch, base.dense, base.surv_grab});
    if (tune_cache && tune_cache[0]) tune_batch(problems, n_problems, base, tune_cache, b->stream, tv);
    for (const TuneVal &v : tv) {
        b->sw.push_back(v.sw);
        b->dense.push_back(v.dense);
        b->grab.push_back(v.grab);
    }
    for (int i = 0; i < n_problems; ++i) {
        const kmeans_problem &pr = problems[i];
        kmeans_options o = base;
        o.dense_switch = tv[i].sw;
        o.dense = tv[i].dense;
        o.surv_grab = tv[i].grab;
        kmeans_ctx *c = nullptr;
        t_ctx_in_batch = true;
        int rc = kmeans_init(&c, static_cast<const float *>(pr.X), pr.N, pr.D, pr.K, pr.G, pr.init_centroids, &o);
        t_ctx_in_batch = false;
        if (rc) {
            batch_err(b, rc, "problem %d: %s", i, kmeans_last_error(nullptr));
            int keep = rc;
            char msg[512];
            memcpy(msg, b->err, sizeof(msg));
            kmeans_batch_destroy(b);
            return batch_err(nullptr, keep, "%s", msg);
        }
        b->ctx.push_back(c);
        float *d0 = nullptr;
        cudaError_t e = cudaMalloc(&d0, (size_t)pr.K * pr.D * 4);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d0, pr.init_centroids, (size_t)pr.K * pr.D * 4, cudaMemcpyDefault, b->stream);
        b->c0.push_back(d0);
        if (e != cudaSuccess) {
            kmeans_batch_destroy(b);
            return batch_err(nullptr, KM_ECUDA, "problem %d: %s", i, cudaGetErrorString(e));
        }
    }
    cudaStreamSynchronize(b->stream);
    *out = b;
    return KM_OK;
}

KM_API int kmeans_batch_fit(kmeans_batch *b, int32_t max_iter, double tol) {
    if (!b) return KM_EINVAL;
    if (max_iter < 1 || !(tol >= 0.0)) return batch_err(b, KM_EINVAL, "max_iter must be >= 1 and tol >= 0");
    DeviceGuard dg(b->dev);
    bool first = true, any_started = false;
    for (kmeans_ctx *c : b->ctx) {
        if (c->broken) return batch_err(b, KM_ESTATE, "a problem's context is unusable");
        first = first && c->t_host == 0;
        any_started = any_started || c->t_host > 0;
        int rc = ensure_tables(c, max_iter + 2);
        if (rc) return batch_err(b, rc, "%s", c->err);
    }
    if (any_started && first == false) {
        for (kmeans_ctx *c : b->ctx)
            if (c->t_host == 0) return batch_err(b, KM_ESTATE, "problems at different iterations: reset the batch");
    }
    bool same = b->exec && b->rec_max_iter == max_iter && b->rec_tol == tol && b->rec_first == first;
    for (size_t i = 0; same && i < b->ctx.size(); ++i) same = b->rec_tcap[i] == b->ctx[i]->tcap;
    if (!same) {
        int rc = batch_record(b, max_iter, tol, first);
        if (rc) return rc;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, b->stream);
    if (e != cudaSuccess) return batch_err(b, KM_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        int rc = sync_and_check(b->ctx[i]);
        if (rc) return batch_err(b, rc, "problem %zu: %s", i, b->ctx[i]->err);
        b->ctx[i]->have_final = true;
    }
    return KM_OK;
}

KM_API int kmeans_batch_get(kmeans_batch *b, int32_t i, int32_t *labels, float *centroids, double *objective,
                            int32_t *n_iter) {
    if (!b) return KM_EINVAL;
    if (i < 0 || i >= (int32_t)b->ctx.size()) return batch_err(b, KM_EINVAL, "problem %d out of range", i);
    kmeans_ctx *c = b->ctx[i];
    DeviceGuard dg(b->dev);
    const Params &p = c->p;
    cudaStream_t s = c->stream;
    cudaError_t e = cudaSuccess;
    if (labels) e = labels_out(c, labels, s);
    if (e == cudaSuccess && centroids) e = centroids_out(c, centroids, s);
    if (e == cudaSuccess && objective) e = cudaMemcpyAsync(objective, &p.ctrl->jfinal, 8, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return batch_err(b, KM_ECUDA, "%s", cudaGetErrorString(e));
    if (n_iter) *n_iter = c->ctrl_host->fit_n_iter;
    return KM_OK;
}

KM_API int kmeans_batch_reset(kmeans_batch *b) {
    if (!b) return KM_EINVAL;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        int rc = kmeans_reset(b->ctx[i], b->c0[i]);
        if (rc) return batch_err(b, rc, "problem %zu: %s", i, b->ctx[i]->err);
    }
    return KM_OK;
}

KM_API int kmeans_batch_get_tuning(const kmeans_batch *b, int32_t i, float *dense_switch, int32_t *dense,
                                   int32_t *surv_grab) {
    if (!b || i < 0 || i >= (int32_t)b->ctx.size()) return KM_EINVAL;
    if (dense_switch) *dense_switch = b->sw[i];
    if (dense) *dense = b->dense[i];
    if (surv_grab) *surv_grab = b->grab[i];
    return KM_OK;
}

KM_API int kmeans_batch_get_switch(const kmeans_batch *b, int32_t i, float *dense_switch) {
    if (!b || !dense_switch || i < 0 || i >= (int32_t)b->ctx.size()) return KM_EINVAL;
    *dense_switch = b->sw[i];
    return KM_OK;
}

KM_API void kmeans_batch_destroy(kmeans_batch *b) {
    if (!b) return;
    DeviceGuard dg(b->dev);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (kmeans_ctx *c : b->ctx) kmeans_destroy(c);
    for (float *d : b->c0) cudaFree(d);
    delete b;
}

KM_API const char *kmeans_batch_last_error(const kmeans_batch *b) { return b ? b->err : g_init_error; }

}  // extern "C"
