// kp_common.cuh -- state layout, launch parameters and device helpers shared
// by the kernels of libkpynq (GB300, sm_103a).
//
// Bounds (KPynq Sec. I: the multi-level filters test per-point distance
// bounds; the bookkeeping follows the Yinyang group/point filter scheme):
//   u(x)     >= ||x - c_a||                 upper bound, own centroid
//   lbg(x)   <= ||x - c||, every c != a     global lower bound
//   lb_g(x)  <= ||x - c||, c in group g, c != a
// They are stored LAZILY: each point keeps the centroid-table version at which
// its values were exact, and the drift accumulated since then is applied when
// the point is read.  Cumulative drift tables (all rounded up):
//   Dc[v][k] = sum_{s<=v} delta_k(s)      per centroid
//   Dg[v][g] = sum_{s<=v} max_{k in g} delta_k(s)
//   Dm[v]    = sum_{s<=v} max_k delta_k(s)
// so that, for a point stamped at version w and centroids at version v,
//   u_eff   = u + (Dc[v][a] - Dc[w][a])          (rounded up)
//   lbg_eff = lbg - (Dm[v] - Dm[w])              (rounded down)
//   lb_eff  = lb_g - (Dg[v][g] - Dg[w][g])       (rounded down)
// Rounding every cumulative sum upward makes each difference an upper bound on
// the true drift over (w, v], so the bounds stay valid in FP32.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kpynq.h"

namespace kp {

constexpr int kWarp = 32;
constexpr int kStatsCap = 4096;

// Device-side control block (one per context).
struct Ctrl {
    int32_t v;            // version of the current centroids C (table row)
    int32_t t;            // iterations run so far
    int32_t done;         // stop rule met (fit loop)
    int32_t err;          // nonzero: a bounded device wait gave up
    int32_t iters_left;   // iterations left in the current fit call
    int32_t have_jprev;   // J_{t-1} known
    int32_t queue_count;  // survivors appended by the filter kernel
    int32_t moved_count;  // moved points appended by the dense kernel
    uint32_t ticket;      // last-block-done counter of the update kernel
    int32_t final_pass;   // the current assignment is a fit's final one
    double tol;
    double jprev;
    double jfinal;
    unsigned long long n_changed, n_survivors, n_scanned, n_dist, n_recheck;
    int32_t fit_n_iter;   // iterations performed by the current fit call
    int32_t path;         // KM_PATH_* of the current assignment
    int32_t dense_mode;   // the current filtered iteration runs the dense pass
    uint32_t filter_ticket;  // last-block-done counter of the filter kernel
    unsigned long long kernels;  // kernels of this context run on the device
    int32_t settle_count;  // rows queued for the exact settle by the tensor-core pass
    int32_t surv_next;     // next queue entry to hand out in the survivor kernel
    int32_t stats_full;    // the cluster sums of this iteration are recomputed in full
    uint32_t stats_ticket; // last-block-done counter of k_stats_hist
    int32_t settle_next;   // next settle request to hand out
};

// Device-side error codes in Ctrl::err (0 = none).
constexpr int32_t kErrLabel = 0x4c41;  // an assignment left a label outside [0, K)
constexpr int32_t kErrQueue = 0x5155;  // a work queue held a count or an entry out of range

// every kernel of a context counts itself once (block 0, thread 0)
__device__ __forceinline__ void count_kernel(Ctrl *c) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&c->kernels, 1ull);
}

// A row the tensor-core pass could not decide: its runner-up lies inside the
// error window of the winner.
struct SettleReq {
    int32_t n;       // point
    int32_t old;     // label before this pass (-1: none)
    int32_t i1;      // tensor-core winner (the bounds were written for it)
    float lb_alt;    // group bound that holds for every column (from the smallest estimate)
    unsigned long long gmask;  // groups that can hold the winner (all ones: every group;
                               // zero: the groups g with lb[n][g] <= lim)
    float lim;       // bound of the window's edge (used when gmask is zero)
};

// Everything a kernel needs, passed by value.
struct Params {
    const float *X;      // N x D, row-major
    const uint16_t *Xh;  // N x D bfloat16: bf16(x)            (tensor-core path)
    const uint16_t *Xl;  // N x D bfloat16: bf16(x - bf16(x))  (tensor-core path)
    const float *xnorm;  // N: ||x - mu||^2 of the values split into Xh / Xl, FP32 (tensor-core path)
    int64_t N;
    int32_t D, K, G;
    int32_t Dp;          // centroid row stride (floats), >= D, multiple of 4
    int32_t Gp;          // lb row stride (floats), >= G, multiple of 4
    int32_t tcap;        // rows of the drift tables
    int32_t x_vec4;      // X rows are 16-byte aligned and D % 4 == 0

    int32_t *label;      // N
    float *u;            // N
    float *lbg;          // N
    float *lb;           // N x Gp
    uint32_t *stamp;     // N: (version of u) << 16 | (version of lbg, lb)

    float *C;            // K x Dp (padding columns are zero)
    const float *mu;     // Dp: centre subtracted from points and centroids before the
                         // tensor-core products (distances do not depend on it); NULL: none
    float e_cen;         // the rounding of x - mu and c - mu moves a squared distance by
                         // at most e_cen (||x - mu|| + max ||c - mu||)^2 (0 without mu)
    double *S;           // K x D   cluster sums (FP64)
    double *Q;           // K       sum of ||x - R_k||^2 per cluster (FP64)
    float *R;            // K x Dp  reference point of each cluster's Q (a copy of C made
                         //         whenever the sums are rebuilt from zero)
    unsigned long long *cnt;  // K  cluster sizes

    float *Dc;           // tcap x K
    float *Dg;           // tcap x Gp
    float *Dm;           // tcap
    const int32_t *grp;  // K: group of each centroid
    const int32_t *orig; // K: caller's index of each centroid (the context may order its
                         // centroids so that every group is a run of indices); NULL: identity
    const int32_t *gstart;  // G + 1: centroids of group g are [gstart[g], gstart[g+1])

    int32_t *queue;      // N: survivors of the global filter, grouped by label bucket
    int32_t *bcount;     // nbucket: survivors per label bucket (label >> bshift)
    int32_t *bcursor;    // nbucket: next free queue slot of each bucket
    int32_t nbucket, bshift;
    struct SettleReq *sreq;  // N, indexed by row: rows the tensor-core pass left to the exact settle
    uint32_t *sbits;     // ceil(N / 128) * 4 words: bit n set = row n has a settle request
    uint16_t *Ch, *Cl;   // Kp x D bfloat16 halves of C (tensor-core pass with K > 256)
    float *cnorm;        // K: ||c||^2 of that pass
    int32_t *squeue;     // N: the rows with a request, compacted from the bitmap
    int32_t *perm;       // N: point ids sorted by label (full recompute of the cluster sums)
    int32_t *slab;       // N: their labels
    int32_t *hcount;     // K: points per label (zero between uses)
    int32_t *hcur;       // K: next free slot of each label's segment
    int32_t hist_smem_k; // largest K whose label histograms live in shared memory
    int32_t *moved;      // N: points whose label changed (dense path)
    int32_t *moved_old;  // N: their previous label (-1: none)
    float *delta;        // K: drift of the last update
    double *Jk;          // K: per-cluster objective terms

    Ctrl *ctrl;
    kmeans_iter_stats *stats;  // kStatsCap ring

    float eps_hi;        // s_true <= s_fp32 * eps_hi + tiny
    float eps_lo;        // s_true >= s_fp32 * eps_lo - tiny
    float tiny;          // absolute slack for underflow
    int32_t algo;
    float dense_frac;    // survivor fraction above which an iteration runs dense
    int32_t surv_grab;   // survivor queue entries a warp claims at a time (multiple of 32; 0: 32)
    unsigned long long cond;  // cudaGraphConditionalHandle of the fit loop (0: none)
};

// ---------------------------------------------------------------------------
// square-root bounds
// ---------------------------------------------------------------------------
// The hardware approximation (sqrt.approx.f32) lies within one step of the
// bit pattern of the correctly rounded square root for every non-negative
// float: measured over all 2^31 inputs, and re-checked on the running device
// by kmeans_selftest_sqrt.  The correctly rounded root has its neighbours on
// either side of the exact root, so two steps below / above the
// approximation bound sqrt(v) from below / above.  (One instruction and an
// integer add, against the branching directed-rounding square root.)
__device__ __forceinline__ float sqrt_approx(float v) {
    float r;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float sqrt_lo(float v) {  // <= sqrt(max(v, 0))
    const float a = sqrt_approx(fmaxf(v, 0.f));
    return a > 0.f ? __int_as_float(__float_as_int(a) - 2) : 0.f;
}
__device__ __forceinline__ float sqrt_hi(float v) {  // >= sqrt(max(v, 0))
    const float a = sqrt_approx(fmaxf(v, 0.f));
    return a < INFINITY ? __int_as_float(__float_as_int(a) + 2) : INFINITY;
}

// ---------------------------------------------------------------------------
// distance bounds from an FP32 squared distance
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dist_up(float s, const Params &p) {
    return sqrt_hi(__fadd_ru(__fmul_ru(s, p.eps_hi), p.tiny));
}
__device__ __forceinline__ float dist_dn(float s, const Params &p) {
    return sqrt_lo(__fsub_rd(__fmul_rd(s, p.eps_lo), p.tiny));
}
// true squared distances of a (computed sa) and b (computed sb) may be ordered
// either way: the FP32 results cannot settle the argmin
__device__ __forceinline__ bool unresolved(float sa, float sb, const Params &p) {
    return __fsub_rd(__fmul_rd(sb, p.eps_lo), p.tiny) <= __fadd_ru(__fmul_ru(sa, p.eps_hi), p.tiny);
}

// FP64 squared distance with the summation order of the FP64 definition
// (i ascending, no fused multiply-add): used to settle near-ties exactly.
__device__ __forceinline__ double dist2_f64(const float *x, const float *c, int D) {
    double s = 0.0;
    for (int i = 0; i < D; ++i) {
        double t = __dsub_rn((double)x[i], (double)c[i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

// ---------------------------------------------------------------------------
// warp reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
// (value, index) minimum, ties to the lower index; every lane gets the result
__device__ __forceinline__ void warp_argmin(float &v, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov < v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
}
// the key that breaks ties between equal distances: the caller's index of
// centroid c (the lowest wins); indices outside [0, K) (sentinels) keep their value
__device__ __forceinline__ int tie_key(const Params &p, int c) {
    return (p.orig && (unsigned)c < (unsigned)p.K) ? p.orig[c] : c;
}
// (value, index) minimum over the warp, ties to the lowest tie_key
__device__ __forceinline__ void warp_argmin_d_key(double &v, int &i, const Params &p) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov < v || (ov == v && tie_key(p, oi) < tie_key(p, i))) { v = ov; i = oi; }
    }
}
__device__ __forceinline__ void warp_argmin_d(double &v, int &i) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, v, o);
        int oi = __shfl_xor_sync(0xffffffffu, i, o);
        if (ov < v || (ov == v && oi < i)) { v = ov; i = oi; }
    }
}

// ---------------------------------------------------------------------------
// TMA bulk copy global -> shared, completed on an mbarrier (bounded waits)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// one bulk copy; dst, src 16-byte aligned, bytes a multiple of 16
__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t phase) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(phase)
        : "memory");
    return ok != 0;
}
// Wait for phase `phase` of the barrier, giving up after `limit` polls (each
// try_wait itself blocks for a bounded time).  Returns false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t phase, uint32_t limit) {
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, phase)) return true;
    return false;
}
constexpr uint32_t kWaitPolls = 1u << 20;

// Stage `bytes` (multiple of 16, in chunks) from global to shared with TMA bulk
// copies issued by thread 0; all threads of the block wait.  On a time-out the
// block records KM_ETIMEOUT in ctrl->err, waits (bounded) once more for the
// copies in flight and returns false.
__device__ inline bool stage_to_smem(void *dst, const void *src, uint32_t bytes, uint64_t *bar, Ctrl *ctrl) {
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        constexpr uint32_t kChunk = 1u << 16;
        mbar_arrive_expect_tx(bar, bytes);
        for (uint32_t off = 0; off < bytes; off += kChunk) {
            uint32_t n = bytes - off < kChunk ? bytes - off : kChunk;
            tma_bulk_g2s(static_cast<char *>(dst) + off, static_cast<const char *>(src) + off, n, bar);
        }
    }
    __syncthreads();
    bool ok = mbar_wait_bounded(bar, 0, kWaitPolls);
    if (!ok) {
        atomicExch(&ctrl->err, (int)KM_ETIMEOUT);
        mbar_wait_bounded(bar, 0, kWaitPolls);
    }
    return __syncthreads_and(ok) != 0;
}

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t stamp_u(uint32_t s) { return s >> 16; }
__device__ __forceinline__ uint32_t stamp_l(uint32_t s) { return s & 0xffffu; }
__device__ __forceinline__ uint32_t make_stamp(uint32_t vu, uint32_t vl) { return (vu << 16) | vl; }

// A label read back from the label array; outside [0, K) (which no kernel
// writes) records kErrLabel and returns -1 so that the caller skips the point.
__device__ __forceinline__ int checked_label(const Params &p, int64_t n) {
    const int k = p.label[n];
    if ((unsigned)k >= (unsigned)p.K) {
        atomicExch(&p.ctrl->err, kErrLabel);
        return -1;
    }
    return k;
}

// drift of centroid k between versions w and v (upper bound)
__device__ __forceinline__ float drift_c(const Params &p, int v, int w, int k) {
    return v == w ? 0.0f : __fsub_ru(p.Dc[(size_t)v * p.K + k], p.Dc[(size_t)w * p.K + k]);
}
__device__ __forceinline__ float drift_g(const Params &p, int v, int w, int g) {
    return v == w ? 0.0f : __fsub_ru(p.Dg[(size_t)v * p.Gp + g], p.Dg[(size_t)w * p.Gp + g]);
}
__device__ __forceinline__ float drift_m(const Params &p, int v, int w) {
    return v == w ? 0.0f : __fsub_ru(p.Dm[v], p.Dm[w]);
}

// ---------------------------------------------------------------------------
// host-side launchers (one translation unit each)
// ---------------------------------------------------------------------------
void count_launch();
void set_thread_error(const char *msg);  // message for kmeans_last_error(NULL)
int dense_dp(int D);  // register tile width used for D (0 = generic path)

// `if_dense`: run only when the filter kernel chose the dense pass for this iteration
cudaError_t launch_dense_assign(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms,
                                int if_dense = 0);
// Width of the bfloat16 operand copies of the tensor-core passes: rows of 32
// coordinates are zero-padded to 64 (the padding adds exact zeros to every
// product); 0 = no tensor-core pass for this D.
__host__ __device__ inline int tc_dim(int D) { return D == 32 || D == 64 ? 64 : (D == 128 ? 128 : 0); }
bool dense_tc_eligible(const Params &p, size_t smem_limit);
bool dense_tcb_eligible(const Params &p, size_t smem_limit);
// the proposal network on the tensor cores (kp_mlp.cu): buffers for N rows,
// then the predicted class of every row, ordered on s (KM_* status)
int mlp_prepare(kmeans_mlp *m, int64_t N);
int mlp_predict_enqueue(kmeans_mlp *m, const float *X, int64_t N, int32_t *pred, cudaStream_t s);
int mlp_error_flag(kmeans_mlp *m);  // synchronises; KM_ETIMEOUT if a bounded wait gave up
const char *mlp_message(const kmeans_mlp *m);
cudaError_t launch_proposal_seed(const Params &p, const int32_t *pred, float *T, cudaStream_t s, int respect_done,
                                 int num_sms);
int dense_tcb_kp(const Params &p);  // padded K of the split centroid copy
cudaError_t launch_dense_tcb(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms,
                             size_t smem_limit, int if_dense);
cudaError_t launch_split_x(const float *X, int64_t N, int D, int Dt, uint16_t *Xh, uint16_t *Xl, cudaStream_t s,
                           int num_sms, float *Xcopy = nullptr, const float *mu = nullptr, float *xnorm = nullptr);
cudaError_t launch_dense_tc(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms,
                            size_t smem_limit, int if_dense = 0);
cudaError_t launch_settle(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms);
// full recompute of the cluster statistics (k_stats_hist decides on the
// device; k_apply_moves then skips itself); needs the label-sort buffers
bool stats_full_supported(const Params &p);
cudaError_t launch_stats_full(const Params &p, cudaStream_t s, int all_points, int respect_done, int num_sms);
cudaError_t launch_apply_moves(const Params &p, cudaStream_t s, int all_points, int respect_done, int num_sms,
                               int if_dense = 0);
cudaError_t launch_filter(const Params &p, cudaStream_t s, int respect_done, int num_sms);
cudaError_t launch_survivor(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem_limit);
bool survivor_tp_eligible(const Params &p);
cudaError_t launch_survivor_tp(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem_limit);
cudaError_t launch_update(const Params &p, cudaStream_t s, int final_only, int respect_done);
cudaError_t launch_arm(const Params &p, cudaStream_t s, int max_iter, double tol);
cudaError_t launch_set_cond(const Params &p, cudaStream_t s);
cudaError_t launch_rebase(const Params &p, cudaStream_t s, int num_sms);
cudaError_t launch_bounds_out(const Params &p, cudaStream_t s, float *u, float *lbg, float *lb, int num_sms);
// k-means++ seeding (kp_kmeanspp.cu): K centres of X into C / idx; dmin (N
// doubles), bsum (ceil(N / 1024)) and state (kmeanspp_state_bytes()) are
// scratch; *err_out (host) is set nonzero if a drawn index fell out of range
cudaError_t launch_kmeanspp(const float *X, int64_t N, int D, int K, const double *u, float *C, long long *idx,
                            double *dmin, unsigned long long *bsum, void *state, cudaStream_t s, int num_sms,
                            long long *err_out);
size_t kmeanspp_state_bytes();
// stream-ordered allocation from the library's own pool on `dev` (it keeps
// freed memory mapped across synchronisations, unlike the default pool with
// its zero release threshold); free with cudaFreeAsync
cudaError_t pool_alloc(int dev, void **p, size_t bytes, cudaStream_t s);

// clustered grouping (kp_group.cu): grp[K] from C (K x D, dense rows), G
// centres seeded by the first G rows, `iters` Lloyd iterations; cen (G x D
// floats) is scratch
cudaError_t launch_clustered_groups(const float *C, int K, int D, int G, int iters, int32_t *grp, float *cen,
                                    cudaStream_t s, int num_sms);
// the caller's centroid numbering (kp_update.cu)
cudaError_t launch_labels_out(const int32_t *label, int64_t N, const int32_t *orig, int K, int32_t *out,
                              cudaStream_t s, int num_sms);
cudaError_t launch_rows_out(const float *C, int Dp, int D, int K, const int32_t *orig, float *out, cudaStream_t s,
                            int num_sms);
cudaError_t launch_rows_in(const float *in, int D, int K, int Dp, const int32_t *orig, float *C, cudaStream_t s,
                           int num_sms);
cudaError_t launch_check_finite(const float *a, int64_t n, int *flag, cudaStream_t s, int num_sms);
cudaError_t launch_bf16_to_f32(const uint16_t *in, int64_t n, float *out, cudaStream_t s, int num_sms);
// mu (Dp floats) = the mean of C's K rows (stride Dp), zero in the padding
cudaError_t launch_centroid_mean(const float *C, int K, int D, int Dp, float *mu, cudaStream_t s);

}  // namespace kp
