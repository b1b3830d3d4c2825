// kp_proposal.cu -- the learned group proposal: an MLP that predicts each
// point's group, and the iteration-0 bounds seeded from that prediction.
//
// The paper's filters (Sec. I) start from bounds that the first, dense
// iteration makes exact.  A proposal can stand in for that pass: with a
// predicted group g(x), the exact FP32 distances to g(x)'s centroids give a
// label candidate c and an upper bound u(x) >= d(x, c); the triangle
// inequality d(x, c') >= d(c, c') - d(x, c) then bounds every other group
// from below by min_{c' in g'} d(c, c') - u(x), from a K x G table of
// centroid-to-centroid distances.  The ordinary filtered iteration that
// follows (global filter, group and point filters, distance calculator) makes
// the labels exact whatever the prediction: a wrong guess only costs work.
//
// The network itself (D -> H -> H -> G, GELU, the group with the largest
// logit) runs on the tensor cores (kp_mlp.cu).
#include "kp_common.cuh"

namespace kp {
namespace {

// T[k][g] = min over c in group g, c != k, of a lower bound of d(c_k, c)
// (FP32 direct difference, rounded down); +inf for a group with no such c.
__global__ void __launch_bounds__(256) k_cc_table(Params p, float *T) {
    extern __shared__ __align__(16) float sm_cc[];  // ck (D) | tmin (G, as int bits)
    float *ck = sm_cc;
    int *tmin = reinterpret_cast<int *>(sm_cc + p.D);
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    const int D = p.D, K = p.K, G = p.G;
    for (int k = blockIdx.x; k < K; k += gridDim.x) {
        for (int d = threadIdx.x; d < D; d += blockDim.x) ck[d] = p.C[(size_t)k * p.Dp + d];
        for (int g = threadIdx.x; g < G; g += blockDim.x) tmin[g] = __float_as_int(INFINITY);
        __syncthreads();
        for (int c = threadIdx.x; c < K; c += blockDim.x) {
            if (c == k) continue;
            const float *cc = p.C + (size_t)c * p.Dp;
            float s = 0.f;
            for (int d = 0; d < D; ++d) {
                const float t = ck[d] - cc[d];
                s = fmaf(t, t, s);
            }
            const int g = p.grp[c];
            if ((unsigned)g < (unsigned)G) atomicMin(&tmin[g], __float_as_int(dist_dn(s, p)));  // non-negative
        }
        __syncthreads();
        for (int g = threadIdx.x; g < G; g += blockDim.x) T[(size_t)k * G + g] = __int_as_float(tmin[g]);
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&ctrl->n_dist, (unsigned long long)K * (K - 1));
}

// Iteration-0 bounds from the prediction: warp per point, lanes over the
// predicted group's centroids (exact FP32 distances), then over the groups.
__global__ void __launch_bounds__(256) k_seed(Params p, const int32_t *pred, const float *T, int respect_done) {
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int D = p.D, G = p.G, K = p.K;
    const int v = ctrl->v;
    unsigned long long c_dist = 0;
    for (int64_t n = w0; n < p.N; n += nw) {
        int pg = pred[n];
        if ((unsigned)pg >= (unsigned)G) pg = 0;  // a prediction outside the groups: group 0
        const int c0 = p.gstart[pg], c1 = p.gstart[pg + 1];
        const float *x = p.X + n * D;
        // smallest (lowest index on ties) and second smallest within the group
        float s1 = INFINITY, s2 = INFINITY;
        int i1 = 0x7fffffff;
        for (int c = c0 + lane; c < c1; c += 32) {
            const float *cc = p.C + (size_t)c * p.Dp;
            float s = 0.f;
            for (int d = 0; d < D; ++d) {
                const float t = __ldg(x + d) - cc[d];
                s = fmaf(t, t, s);
            }
            if (s < s1) {
                s2 = s1;
                s1 = s;
                i1 = c;
            } else {
                s2 = fminf(s2, s);
            }
        }
        float bs = s1;
        int bi = i1;
        warp_argmin(bs, bi);
        const float sec = warp_min(i1 == bi ? s2 : s1);
        c_dist += lane == 0 ? (unsigned long long)(c1 - c0) : 0ull;
        if ((unsigned)bi >= (unsigned)K) bi = c0;  // cannot happen: the group is not empty
        const float u = dist_up(bs, p);
        const float lin = sec == INFINITY ? INFINITY : dist_dn(sec, p);  // the group's other centroids
        const float *Tr = T + (size_t)bi * G;
        float gmin = INFINITY;
        for (int g = lane; g < G; g += 32) {
            float l;
            if (g == pg) {
                l = lin;
            } else {
                const float t = Tr[g];
                l = t == INFINITY ? INFINITY : fmaxf(__fsub_rd(t, u), 0.f);
            }
            p.lb[n * p.Gp + g] = l;
            gmin = fminf(gmin, l);
        }
        gmin = warp_min(gmin);
        if (lane == 0) {
            p.label[n] = bi;
            p.u[n] = u;
            p.lbg[n] = gmin;
            p.stamp[n] = make_stamp(v, v);
        }
    }
    if (lane == 0 && c_dist) atomicAdd(&ctrl->n_dist, c_dist);
}

}  // namespace

cudaError_t launch_proposal_seed(const Params &p, const int32_t *pred, float *T, cudaStream_t s, int respect_done,
                                 int num_sms) {
    const size_t smem = (size_t)p.D * 4 + (size_t)p.G * 4;
    count_launch();
    k_cc_table<<<(unsigned)std::min(p.K, num_sms * 8), 256, smem, s>>>(p, T);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t warps = std::min<int64_t>(p.N, (int64_t)num_sms * 64);
    count_launch();
    k_seed<<<(unsigned)((warps + 7) / 8), 256, 0, s>>>(p, pred, T, respect_done);
    return cudaGetLastError();
}

}  // namespace kp
