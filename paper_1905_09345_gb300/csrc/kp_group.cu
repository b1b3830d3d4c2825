// kp_group.cu -- the clustered grouping of the centroids.
//
// The filters of Sec. I test one lower bound per group of centroids; how the
// groups form is the library's reading (the paper does not say).  Besides
// contiguous index ranges, a context can group nearby centroids: plain Lloyd
// over the K initial centroids with G centres seeded by their first G rows,
// `iters` iterations, each centroid then in the group of its nearest centre
// (lowest index on ties); an empty group keeps its centre.  FP32 (chains of
// dependent FP64 operations are slow on these SMs, and the grouping is a
// heuristic: labels of the method never depend on it, only how much the
// filters skip does).
#include "kp_common.cuh"

namespace kp {
namespace {

constexpr int GRP_THREADS = 256;

// grp[k] = argmin_g ||c_k - cen_g||^2 (lowest g on ties).  Warp per
// centroid, lanes over the groups; the centres sit in shared memory with a
// row stride of D + 1 words, so lanes reading different rows at the same d
// hit different banks.  cen_smem: whether the centres fit in shared memory
// (else they are read from global memory).
__global__ void __launch_bounds__(GRP_THREADS) k_grp_assign(const float *__restrict__ C, int K, int D,
                                                            const float *__restrict__ cen, int G, int cen_smem,
                                                            int32_t *__restrict__ grp) {
    extern __shared__ float sm_grp[];  // ck (warps x D) | cen (G x (D + 1)) when cen_smem
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    float *ck = sm_grp + (size_t)warp * D;
    float *cs = sm_grp + (size_t)nw * D;
    const int ld = cen_smem ? D + 1 : D;
    if (cen_smem) {
        for (int i = threadIdx.x; i < G * D; i += blockDim.x) cs[(i / D) * ld + i % D] = cen[i];
        __syncthreads();
    }
    const float *m0 = cen_smem ? cs : cen;
    for (int k = blockIdx.x * nw + warp; k < K; k += gridDim.x * nw) {
        for (int d = lane; d < D; d += 32) ck[d] = C[(size_t)k * D + d];
        __syncwarp();
        float best = INFINITY;
        int bi = 0x7fffffff;
        for (int g = lane; g < G; g += 32) {
            const float *m = m0 + (size_t)g * ld;
            float s = 0.f;
            for (int d = 0; d < D; ++d) {
                const float t = ck[d] - m[d];
                s = fmaf(t, t, s);
            }
            if (s < best) {  // g ascends within a lane: the first minimum stays
                best = s;
                bi = g;
            }
        }
        for (int o = 16; o; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
            if (ob < best || (ob == best && oi < bi)) {
                best = ob;
                bi = oi;
            }
        }
        if (lane == 0) grp[k] = bi < G ? bi : 0;  // bi >= G only if every distance is NaN
        __syncwarp();
    }
}

// cen_g = mean of the centroids in group g, summed in ascending centroid
// order (block per group; members compacted chunk by chunk); a group
// without members keeps its centre.
__global__ void __launch_bounds__(GRP_THREADS) k_grp_update(const float *__restrict__ C, int K, int D,
                                                            const int32_t *__restrict__ grp, float *__restrict__ cen) {
    extern __shared__ float sm_grp[];  // sum (D) | members (blockDim) | warp counts (32)
    float *sum = sm_grp;
    int *mem = reinterpret_cast<int *>(sm_grp + D);
    int *wcnt = mem + blockDim.x;
    const int g = blockIdx.x;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int d = threadIdx.x; d < D; d += blockDim.x) sum[d] = 0.f;
    int n = 0;
    for (int k0 = 0; k0 < K; k0 += blockDim.x) {
        const int k = k0 + threadIdx.x;
        const bool in = k < K && grp[k] == g;
        const unsigned b = __ballot_sync(0xffffffffu, in);
        if (lane == 0) wcnt[warp] = __popc(b);
        __syncthreads();
        int off = 0, tot = 0;
        for (int w = 0; w < nw; ++w) {
            off += w < warp ? wcnt[w] : 0;
            tot += wcnt[w];
        }
        if (in) mem[off + __popc(b & ((1u << lane) - 1u))] = k;
        __syncthreads();
        for (int d = threadIdx.x; d < D; d += blockDim.x) {
            float s = sum[d];
            for (int j = 0; j < tot; ++j) s += C[(size_t)mem[j] * D + d];
            sum[d] = s;
        }
        n += tot;
        __syncthreads();
    }
    if (n == 0) return;
    for (int d = threadIdx.x; d < D; d += blockDim.x) cen[(size_t)g * D + d] = sum[d] / (float)n;
}

__global__ void k_grp_seed(const float *C, int G, int D, float *cen) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < G * D; i += gridDim.x * blockDim.x) cen[i] = C[i];
}

}  // namespace

cudaError_t launch_clustered_groups(const float *C, int K, int D, int G, int iters, int32_t *grp, float *cen,
                                    cudaStream_t s, int num_sms) {
    const int nw = GRP_THREADS / 32;
    const size_t sm_ck = (size_t)nw * D * 4;
    const size_t sm_cen = (size_t)G * (D + 1) * 4;
    const int cen_smem = sm_ck + sm_cen <= 96 * 1024;  // leaves room for two blocks per SM
    const size_t smem_a = sm_ck + (cen_smem ? sm_cen : 0);
    const size_t smem_u = (size_t)D * 4 + (size_t)GRP_THREADS * 4 + 32 * 4;
    if (smem_a > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_grp_assign, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_a);
        if (e != cudaSuccess) return e;
    }
    if (smem_u > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_grp_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_u);
        if (e != cudaSuccess) return e;
    }
    const unsigned ga = (unsigned)std::max(1, std::min((K + nw - 1) / nw, num_sms));
    count_launch();
    k_grp_seed<<<(unsigned)std::max(1, std::min((G * D + 255) / 256, num_sms * 4)), 256, 0, s>>>(C, G, D, cen);
    cudaError_t e = cudaGetLastError();
    for (int it = 0; e == cudaSuccess && it <= iters; ++it) {
        count_launch();
        k_grp_assign<<<ga, GRP_THREADS, smem_a, s>>>(C, K, D, cen, G, cen_smem, grp);
        e = cudaGetLastError();
        if (e != cudaSuccess || it == iters) break;
        count_launch();
        k_grp_update<<<(unsigned)G, GRP_THREADS, smem_u, s>>>(C, K, D, grp, cen);
        e = cudaGetLastError();
    }
    return e;
}

}  // namespace kp
