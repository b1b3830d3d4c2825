// kp_update.cu -- centroid update, drift, objective and loop control.
//
// The update step of K-means (the centroid of each cluster becomes the mean of
// its points; an empty cluster keeps its centroid) from FP64 cluster sums
// S_k = sum x, Q_k = sum ||x - r_k||^2 and counts n_k, which the assignment
// kernels keep up to date by moving each relabelled point between clusters
// (r_k: the cluster's reference point, its centroid when the sums were last
// rebuilt from zero).  The objective of the assignment just made comes from
// the same sums: with e = c_k - r_k,
//   J_t = sum_k ( Q_k - 2 e . (S_k - n_k r_k) + n_k ||e||^2 ),   c = C^t,
// so no pass over X is needed, and because r_k stays near c_k no large terms
// cancel, however far the data lie from the origin.  The drift of each centroid,
// delta_k = ||c_k^{t+1} - c_k^t|| (rounded up), extends the cumulative drift
// tables that the filters use to age the bounds (KPynq Sec. I: the filters
// test bounds that must stay valid as centroids move).
#include "kp_common.cuh"

namespace kp {

constexpr int kUpdWarps = 8;

__device__ __forceinline__ float round_up_f(double x) { return __double2float_ru(x); }

// One warp per centroid; the last block to finish reduces over centroids.
__global__ void __launch_bounds__(kUpdWarps * 32) k_update(Params p, int final_only, int respect_done) {
    __shared__ double red_d[kUpdWarps * 32];
    __shared__ float red_f[kUpdWarps * 32];
    __shared__ int is_last;
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    const int v = ctrl->v;
    const int lane = threadIdx.x & 31;
    const int k = blockIdx.x * kUpdWarps + (threadIdx.x >> 5);
    const int D = p.D;
    if (k < p.K) {
        const unsigned long long nk = p.cnt[k];
        const double nkd = (double)nk;
        double j1 = 0.0, j2 = 0.0, dd = 0.0;
        float *crow = p.C + (size_t)k * p.Dp;
        const float *rrow = p.R + (size_t)k * p.Dp;
        const double *srow = p.S + (size_t)k * D;
        for (int i = lane; i < D; i += 32) {
            const float co = crow[i];
            const double s = srow[i];
            const double e = (double)co - (double)rrow[i];  // exact; read before C is written
            j1 += e * (s - nkd * (double)rrow[i]);
            j2 += e * e;
            if (!final_only) {
                const float cn = nk ? (float)(s / nkd) : co;
                const double t = (double)cn - (double)co;
                dd += t * t;
                crow[i] = cn;
            }
        }
        j1 = warp_sum_d(j1);
        j2 = warp_sum_d(j2);
        dd = warp_sum_d(dd);
        if (lane == 0) {
            p.Jk[k] = p.Q[k] - 2.0 * j1 + nkd * j2;
            if (!final_only) {
                // sqrt of an FP64 sum of D squares: relative error below
                // (D + 4) 2^-53; inflate by that, then round up to FP32
                const double dk = sqrt(dd) * (1.0 + (double)(D + 4) * 1.1102230246251565e-16);
                const float dlt = round_up_f(dk);
                p.delta[k] = dlt;
                p.Dc[(size_t)(v + 1) * p.K + k] = __fadd_ru(p.Dc[(size_t)v * p.K + k], dlt);
            }
        }
    }
    // last block done?
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned t = atomicAdd(&ctrl->ticket, 1u);
        is_last = (t == gridDim.x - 1);
    }
    __syncthreads();
    if (!is_last) return;
    __threadfence();

    // objective, in a fixed order (deterministic)
    double jp = 0.0;
    for (int kk = threadIdx.x; kk < p.K; kk += blockDim.x) jp += p.Jk[kk];
    red_d[threadIdx.x] = jp;
    float dmax = 0.f;
    if (!final_only) {
        for (int g = threadIdx.x; g < p.G; g += blockDim.x) {
            float m = 0.f;
            for (int kk = p.gstart[g]; kk < p.gstart[g + 1]; ++kk) m = fmaxf(m, p.delta[kk]);
            p.Dg[(size_t)(v + 1) * p.Gp + g] = __fadd_ru(p.Dg[(size_t)v * p.Gp + g], m);
            dmax = fmaxf(dmax, m);
        }
    }
    red_f[threadIdx.x] = dmax;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            red_d[threadIdx.x] += red_d[threadIdx.x + s];
            red_f[threadIdx.x] = fmaxf(red_f[threadIdx.x], red_f[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double J = red_d[0];
        const float dm = red_f[0];
        const int t = ctrl->t;
        kmeans_iter_stats st;
        memset(&st, 0, sizeof(st));
        st.iter = t;
        st.n_changed = (int64_t)ctrl->n_changed;
        st.n_survivors = (int64_t)ctrl->n_survivors;
        st.n_scanned = (int64_t)ctrl->n_scanned;
        st.n_dist = (int64_t)ctrl->n_dist;
        st.n_recheck = (int64_t)ctrl->n_recheck;
        st.path = ctrl->path;
        st.n_settle = ctrl->settle_count;
        st.objective = J;
        if (final_only) {
            ctrl->jfinal = J;
            st.done = 1;
            p.stats[kStatsCap] = st;  // the final assignment's record
        } else {
            p.Dm[v + 1] = __fadd_ru(p.Dm[v], dm);
            st.max_drift = (double)dm;
            ctrl->iters_left -= 1;
            int stop = ctrl->iters_left <= 0 || st.n_changed == 0 ||
                       (ctrl->have_jprev && (ctrl->jprev - J) < ctrl->tol * ctrl->jprev);
            st.done = stop;
            ctrl->done = stop;
            ctrl->jprev = J;
            ctrl->have_jprev = 1;
            ctrl->v = v + 1;
            ctrl->t = t + 1;
            ctrl->fit_n_iter += 1;
            p.stats[t % kStatsCap] = st;
            if (p.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)p.cond, stop ? 0u : 1u);
        }
        ctrl->n_changed = ctrl->n_survivors = ctrl->n_scanned = ctrl->n_dist = ctrl->n_recheck = 0;
        ctrl->queue_count = 0;
        ctrl->moved_count = 0;
        ctrl->settle_count = 0;
        ctrl->surv_next = 0;
        ctrl->settle_next = 0;
        ctrl->path = KM_PATH_FILTERED;
        ctrl->dense_mode = 0;
        __threadfence();
        ctrl->ticket = 0;
    }
}

// Start of a fit / iterate call: loop state for the device-side stop rule.
__global__ void k_arm(Params p, int max_iter, double tol) {
    Ctrl *c = p.ctrl;
    c->kernels += 1;
    c->done = max_iter <= 0;
    c->iters_left = max_iter;
    c->tol = tol;
    c->fit_n_iter = 0;
    c->err = 0;
}

// First node of the fit graph: enter the device-side loop only if the stop
// rule does not already hold.
__global__ void k_set_cond(Params p) {
    p.ctrl->kernels += 1;
    if (p.cond) cudaGraphSetConditional((cudaGraphConditionalHandle)p.cond, p.ctrl->done ? 0u : 1u);
}

// Make every stored bound exact at the current version and restart the drift
// tables at row 0 (run when the tables are about to fill).
__global__ void k_rebase_points(Params p) {
    count_kernel(p.ctrl);
    const int v = p.ctrl->v;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t st = p.stamp[n];
        const int wu = (int)stamp_u(st), wl = (int)stamp_l(st);
        const int a = p.label[n];
        p.u[n] = __fadd_ru(p.u[n], drift_c(p, v, wu, a));
        p.lbg[n] = __fsub_rd(p.lbg[n], drift_m(p, v, wl));
        for (int g = 0; g < p.G; ++g)
            p.lb[n * p.Gp + g] = __fsub_rd(p.lb[n * p.Gp + g], drift_g(p, v, wl, g));
        p.stamp[n] = 0;
    }
}
__global__ void k_rebase_tables(Params p) {
    count_kernel(p.ctrl);
    for (int k = threadIdx.x; k < p.K; k += blockDim.x) p.Dc[k] = 0.f;
    for (int g = threadIdx.x; g < p.Gp; g += blockDim.x) p.Dg[g] = 0.f;
    if (threadIdx.x == 0) {
        p.Dm[0] = 0.f;
        p.ctrl->v = 0;
    }
}

// Bounds made valid for the current centroids, written to caller buffers.
__global__ void k_bounds_out(Params p, float *u, float *lbg, float *lb) {
    count_kernel(p.ctrl);
    const int v = p.ctrl->v;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < p.N; n += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t st = p.stamp[n];
        const int wu = (int)stamp_u(st), wl = (int)stamp_l(st);
        if (u) u[n] = __fadd_ru(p.u[n], drift_c(p, v, wu, p.label[n]));
        if (lbg) lbg[n] = __fsub_rd(p.lbg[n], drift_m(p, v, wl));
        if (lb)
            for (int g = 0; g < p.G; ++g)
                lb[n * p.G + g] = __fsub_rd(p.lb[n * p.Gp + g], drift_g(p, v, wl, g));
    }
}

// flag = 1 if any element is NaN or +-Inf
__global__ void k_check_finite(const float *a, int64_t n, int *flag) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(a[i])) *flag = 1;
}

cudaError_t launch_update(const Params &p, cudaStream_t s, int final_only, int respect_done) {
    count_launch();
    k_update<<<(p.K + kUpdWarps - 1) / kUpdWarps, kUpdWarps * 32, 0, s>>>(p, final_only, respect_done);
    return cudaGetLastError();
}
cudaError_t launch_arm(const Params &p, cudaStream_t s, int max_iter, double tol) {
    count_launch();
    k_arm<<<1, 1, 0, s>>>(p, max_iter, tol);
    return cudaGetLastError();
}
cudaError_t launch_set_cond(const Params &p, cudaStream_t s) {
    count_launch();
    k_set_cond<<<1, 1, 0, s>>>(p);
    return cudaGetLastError();
}
cudaError_t launch_rebase(const Params &p, cudaStream_t s, int num_sms) {
    int64_t grid = std::min<int64_t>((p.N + 255) / 256, (int64_t)num_sms * 8);
    count_launch();
    k_rebase_points<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(p);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_rebase_tables<<<1, 256, 0, s>>>(p);
    return cudaGetLastError();
}
cudaError_t launch_bounds_out(const Params &p, cudaStream_t s, float *u, float *lbg, float *lb, int num_sms) {
    int64_t grid = std::min<int64_t>((p.N + 255) / 256, (int64_t)num_sms * 8);
    count_launch();
    k_bounds_out<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(p, u, lbg, lb);
    return cudaGetLastError();
}
// bfloat16 bit patterns -> FP32 (exact: a bfloat16 is the top half of an FP32)
// mu[d] = mean over the K rows of C (row stride Dp) of coordinate d, for
// d < D, summed in FP64 (each thread a strided run of rows in ascending order,
// then a fixed tree: deterministic) and rounded to FP32; mu[d] = 0 for the
// padding D <= d < Dp.  One block per coordinate.
__global__ void __launch_bounds__(256) k_centroid_mean(const float *C, int K, int D, int Dp, float *mu) {
    __shared__ double part[256];
    const int d = blockIdx.x;
    double m = 0.0;
    if (d < D)
        for (int k = threadIdx.x; k < K; k += blockDim.x) m += (double)C[(size_t)k * Dp + d];
    part[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) mu[d] = d < D ? (float)(part[0] / (double)K) : 0.f;
}

__global__ void k_bf16_to_f32(const uint16_t *in, int64_t n, float *out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __uint_as_float((uint32_t)in[i] << 16);
}

// The caller's centroid numbering (a context may order its centroids group by
// group): labels out[n] = orig[label[n]], centroid rows out[orig[k]] = C[k]
// and C[k] = in[orig[k]].
__global__ void k_labels_out(const int32_t *label, int64_t N, const int32_t *orig, int K, int32_t *out) {
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < N; n += (int64_t)gridDim.x * blockDim.x) {
        const int k = label[n];
        out[n] = (unsigned)k < (unsigned)K ? orig[k] : k;
    }
}
__global__ void k_rows_out(const float *C, int Dp, int D, int K, const int32_t *orig, float *out) {
    const int64_t total = (int64_t)K * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / D), d = (int)(i - (int64_t)k * D);
        out[(int64_t)orig[k] * D + d] = C[(int64_t)k * Dp + d];
    }
}
__global__ void k_rows_in(const float *in, int D, int K, int Dp, const int32_t *orig, float *C) {
    const int64_t total = (int64_t)K * D;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / D), d = (int)(i - (int64_t)k * D);
        C[(int64_t)k * Dp + d] = in[(int64_t)orig[k] * D + d];
    }
}

cudaError_t launch_labels_out(const int32_t *label, int64_t N, const int32_t *orig, int K, int32_t *out,
                              cudaStream_t s, int num_sms) {
    count_launch();
    k_labels_out<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>((N + 255) / 256, (int64_t)num_sms * 8)), 256, 0,
                   s>>>(label, N, orig, K, out);
    return cudaGetLastError();
}
cudaError_t launch_rows_out(const float *C, int Dp, int D, int K, const int32_t *orig, float *out, cudaStream_t s,
                            int num_sms) {
    count_launch();
    k_rows_out<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)K * D + 255) / 256, (int64_t)num_sms * 8)),
                 256, 0, s>>>(C, Dp, D, K, orig, out);
    return cudaGetLastError();
}
cudaError_t launch_rows_in(const float *in, int D, int K, int Dp, const int32_t *orig, float *C, cudaStream_t s,
                           int num_sms) {
    count_launch();
    k_rows_in<<<(unsigned)std::max<int64_t>(1, std::min<int64_t>(((int64_t)K * D + 255) / 256, (int64_t)num_sms * 8)),
                256, 0, s>>>(in, D, K, Dp, orig, C);
    return cudaGetLastError();
}

cudaError_t launch_centroid_mean(const float *C, int K, int D, int Dp, float *mu, cudaStream_t s) {
    count_launch();
    k_centroid_mean<<<(unsigned)Dp, 256, 0, s>>>(C, K, D, Dp, mu);
    return cudaGetLastError();
}
cudaError_t launch_bf16_to_f32(const uint16_t *in, int64_t n, float *out, cudaStream_t s, int num_sms) {
    count_launch();
    k_bf16_to_f32<<<num_sms * 8, 256, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

cudaError_t launch_check_finite(const float *a, int64_t n, int *flag, cudaStream_t s, int num_sms) {
    int64_t grid = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 8);
    count_launch();
    k_check_finite<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(a, n, flag);
    return cudaGetLastError();
}

}  // namespace kp
