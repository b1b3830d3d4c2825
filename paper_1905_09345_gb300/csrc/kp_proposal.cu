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
// The MLP (D -> H -> H -> G, GELU, the group with the largest logit) runs in
// FP32 on the CUDA cores: tiled GEMMs with the bias and activation fused,
// the last layer fused with the argmax so that no logits are stored.
#include "kp_common.cuh"

namespace kp {
namespace {

constexpr int kBM = 64, kBN = 64, kBK = 16;  // GEMM tile: rows x outputs x inner

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }

// One 64 x 64 tile of  A (M x Kd, row-major) . W^T (W: Nout x Kd, row-major),
// accumulated into acc[4][4] (thread: rows 4ty.., outputs 4tx..).
__device__ __forceinline__ void gemm_tile(const float *A, int64_t M, int Kd, const float *W, int Nout, int64_t m0,
                                          int j0, float (&As)[kBK][kBM + 4], float (&Ws)[kBK][kBN + 4],
                                          float (&acc)[4][4]) {
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < Kd; k0 += kBK) {
        // 64 x 16 of A and of W, four elements per thread, stored transposed
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + r * 256, row = e >> 4, kk = e & 15;
            const int64_t m = m0 + row;
            const int k = k0 + kk, j = j0 + row;
            As[kk][row] = (m < M && k < Kd) ? A[m * Kd + k] : 0.f;
            Ws[kk][row] = (j < Nout && k < Kd) ? W[(int64_t)j * Kd + k] : 0.f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < kBK; ++kk) {
            const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
            const float4 w = *reinterpret_cast<const float4 *>(&Ws[kk][tx * 4]);
            const float av[4] = {a.x, a.y, a.z, a.w}, wv[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], wv[j], acc[i][j]);
        }
        __syncthreads();
    }
}

// out = GELU(A W^T + b)  (M x Nout)
__global__ void __launch_bounds__(256) k_mlp_layer(const float *A, int64_t M, int Kd, const float *W, const float *b,
                                                   int Nout, float *out) {
    __shared__ __align__(16) float As[kBK][kBM + 4];
    __shared__ __align__(16) float Ws[kBK][kBN + 4];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * kBM;
    const int j0 = blockIdx.y * kBN;
    float acc[4][4];
    gemm_tile(A, M, Kd, W, Nout, m0, j0, As, Ws, acc);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t m = m0 + ty * 4 + i;
        if (m >= M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int jj = j0 + tx * 4 + j;
            if (jj < Nout) out[m * Nout + jj] = gelu_f(acc[i][j] + b[jj]);
        }
    }
}

// pred[m] = argmax_j (A W^T + b)[m][j]  (first maximum), over all Nout outputs
__global__ void __launch_bounds__(256) k_mlp_out_argmax(const float *A, int64_t M, int Kd, const float *W,
                                                        const float *b, int Nout, int32_t *pred) {
    __shared__ __align__(16) float As[kBK][kBM + 4];
    __shared__ __align__(16) float Ws[kBK][kBN + 4];
    __shared__ float Cs[kBM][kBN + 1];
    __shared__ float best_v[kBM];
    __shared__ int best_i[kBM];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int64_t m0 = (int64_t)blockIdx.x * kBM;
    if (threadIdx.x < kBM) {
        best_v[threadIdx.x] = -INFINITY;
        best_i[threadIdx.x] = 0;
    }
    for (int j0 = 0; j0 < Nout; j0 += kBN) {
        float acc[4][4];
        gemm_tile(A, M, Kd, W, Nout, m0, j0, As, Ws, acc);
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int jj = j0 + tx * 4 + j;
                Cs[ty * 4 + i][tx * 4 + j] = jj < Nout ? acc[i][j] + b[jj] : -INFINITY;
            }
        __syncthreads();
        if (threadIdx.x < kBM) {  // one thread per row, outputs in ascending order
            float bv = best_v[threadIdx.x];
            int bi = best_i[threadIdx.x];
            for (int j = 0; j < kBN && j0 + j < Nout; ++j) {
                const float v = Cs[threadIdx.x][j];
                if (v > bv) {
                    bv = v;
                    bi = j0 + j;
                }
            }
            best_v[threadIdx.x] = bv;
            best_i[threadIdx.x] = bi;
        }
        __syncthreads();
    }
    if (threadIdx.x < kBM && m0 + threadIdx.x < M) pred[m0 + threadIdx.x] = best_i[threadIdx.x];
}

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

cudaError_t launch_mlp_predict(const float *X, int64_t N, int D, const float *W1, const float *b1, const float *W2,
                               const float *b2, const float *W3, const float *b3, int H, int G, int32_t *pred,
                               float *A1, float *A2, int64_t chunk, cudaStream_t s) {
    for (int64_t r0 = 0; r0 < N; r0 += chunk) {
        const int64_t m = std::min(chunk, N - r0);
        const unsigned gm = (unsigned)((m + kBM - 1) / kBM);
        dim3 gh(gm, (unsigned)((H + kBN - 1) / kBN));
        count_launch();
        k_mlp_layer<<<gh, 256, 0, s>>>(X + r0 * D, m, D, W1, b1, H, A1);
        count_launch();
        k_mlp_layer<<<gh, 256, 0, s>>>(A1, m, H, W2, b2, H, A2);
        count_launch();
        k_mlp_out_argmax<<<gm, 256, 0, s>>>(A2, m, H, W3, b3, G, pred + r0);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

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
