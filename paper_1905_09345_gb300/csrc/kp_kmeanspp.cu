// kp_kmeanspp.cu -- k-means++ seeding on the GPU.
//
// The paper takes its initial centroids as given; the library also offers the
// D^2 seeding of k-means++ (Arthur and Vassilvitskii, SODA 2007): the first
// centre is a point drawn uniformly, each further one a point drawn with
// probability proportional to D(x)^2, its squared distance to the nearest
// centre chosen so far.  The random numbers are inputs (one uniform in [0, 1)
// per centre) and every decision is exact, so that any implementation given
// the same uniforms picks the same points:
//   D(x)^2   FP64, sum_i (x_i - c_i)^2 with i ascending and no fused
//            multiply-add, minimised over the centres chosen so far;
//   weights  q(x) = floor(D(x)^2 * 2^s) (64-bit integers), 2^s the power of two
//            that puts max_x D(x)^2 in [2^31, 2^32) -- an exact scaling, and
//            integer sums are exact in any order;
//   draw     T = floor(u_j * W), W = sum q (T = W - 1 if the product rounds up
//            to W); the centre is the first point (in index order) whose
//            running sum of q exceeds T; W = 0: floor(u_j * N); first: floor(u_0 * N).
//
// Per centre: k_pp_update (the new centre's FP64 distances, the running
// minimum and its maximum), k_pp_blocksum (integer weights summed per chunk of
// 1024 points), k_pp_pick (one block: the chunk holding T, then the point in
// it; copies the point to the output centroids).
#include "kp_common.cuh"

namespace kp {
namespace {

constexpr int kPPChunk = 1024;  // points per block sum
constexpr int kPPThreads = 256;

struct PPState {
    unsigned long long wmax;  // bit pattern of max D^2 (non-negative doubles order as their bits)
    long long pick;           // the centre chosen last
    long long err;            // nonzero: an index out of range was produced
};

__device__ __forceinline__ long long uniform_index(double u, long long N) {
    long long i = (long long)floor(__dmul_rn(u, (double)N));
    return i < 0 ? 0 : (i >= N ? N - 1 : i);
}

// 2^(32 - e) for wmax = m 2^e, m in [0.5, 1) (wmax normal: a nonzero squared
// distance between FP32 points is at least 2^-298)
__device__ __forceinline__ double weight_scale(unsigned long long wbits) {
    const int e = (int)((wbits >> 52) & 0x7ff) - 1022;
    return __longlong_as_double((long long)(1023 + 32 - e) << 52);
}

__device__ __forceinline__ unsigned long long weight(double d, double scale) {
    return (unsigned long long)floor(__dmul_rn(d, scale));  // exact: a power-of-two scaling
}

__global__ void k_pp_first(const double *u, long long N, PPState *st) {
    st->pick = uniform_index(u[0], N);
    st->wmax = 0ull;
    st->err = 0;
}


// dmin[n] = min(dmin[n], D(x_n, X[pick])^2); wmax = max over n (one atomic per warp)
__global__ void __launch_bounds__(kPPThreads) k_pp_update(const float *X, long long N, int D, double *dmin,
                                                         PPState *st, int first) {
    const long long pick = st->pick;
    const float *c = X + pick * D;
    double m = 0.0;
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const float *x = X + n * D;
        double s = 0.0;
        for (int i = 0; i < D; ++i) {
            const double t = __dsub_rn((double)x[i], (double)c[i]);
            s = __dadd_rn(s, __dmul_rn(t, t));
        }
        const double d = first ? s : fmin(dmin[n], s);
        dmin[n] = d;
        m = fmax(m, d);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0.0) atomicMax(&st->wmax, (unsigned long long)__double_as_longlong(m));
}

// bsum[b] = sum of q over points [b * 1024, (b + 1) * 1024)
__global__ void __launch_bounds__(kPPThreads) k_pp_blocksum(const double *dmin, long long N, const PPState *st,
                                                           unsigned long long *bsum) {
    __shared__ unsigned long long ws[kPPThreads / 32];
    const unsigned long long wbits = st->wmax;
    const double scale = wbits ? weight_scale(wbits) : 0.0;
    const long long n0 = (long long)blockIdx.x * kPPChunk;
    unsigned long long acc = 0;
    if (wbits)
        for (int k = threadIdx.x; k < kPPChunk; k += blockDim.x) {
            const long long n = n0 + k;
            if (n < N) acc += weight(dmin[n], scale);
        }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < kPPThreads / 32; ++w) t += ws[w];
        bsum[blockIdx.x] = t;
    }
}

// inclusive scan of one value per thread across a block of 1024 threads
__device__ __forceinline__ unsigned long long block_scan_incl(unsigned long long v, unsigned long long *sh,
                                                              unsigned long long *total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) sh[w] = v;
    __syncthreads();
    if (w == 0) {
        unsigned long long s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long t = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += t;
        }
        sh[lane] = s;  // inclusive sums of the warp totals
    }
    __syncthreads();
    const unsigned long long out = v + (w > 0 ? sh[w - 1] : 0ull);
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return out;
}

// one block of 1024 threads: the draw of centre j
__global__ void __launch_bounds__(1024) k_pp_pick(const float *X, long long N, int D, const double *dmin,
                                                 const unsigned long long *bsum, long long nb, const double *u,
                                                 int j, PPState *st, float *C, long long *idx) {
    __shared__ unsigned long long sh[32];
    __shared__ long long s_block;
    __shared__ unsigned long long s_before;
    __shared__ long long s_pick;
    const int tid = threadIdx.x;
    // per-thread run of chunk sums, scanned across the block
    const long long per = (nb + 1023) / 1024;
    const long long b0 = tid * per, b1 = min(b0 + per, nb);
    unsigned long long run = 0;
    for (long long b = b0; b < b1; ++b) run += bsum[b];
    unsigned long long W = 0;
    const unsigned long long incl = block_scan_incl(run, sh, &W);
    if (tid == 0) {
        s_block = -1;
        s_pick = N;
    }
    __syncthreads();
    if (W == 0) {  // every weight is zero: a uniform draw
        if (tid == 0) s_pick = uniform_index(u[j], N);
    } else {
        unsigned long long T = (unsigned long long)floor(__dmul_rn(u[j], (double)W));
        if (T >= W) T = W - 1;
        const unsigned long long excl = incl - run;
        if (excl <= T && T < incl) {  // exactly one thread: its run holds T
            unsigned long long acc = excl;
            for (long long b = b0; b < b1; ++b) {
                if (acc + bsum[b] > T) {
                    s_block = b;
                    s_before = acc;
                    break;
                }
                acc += bsum[b];
            }
        }
        __syncthreads();
        const long long b = s_block;
        if (b >= 0) {
            const double scale = weight_scale(st->wmax);
            const long long n = b * kPPChunk + tid;
            const unsigned long long q = n < N ? weight(dmin[n], scale) : 0ull;
            const unsigned long long in = block_scan_incl(q, sh, nullptr);
            if (n < N && s_before + in > T && s_before + in - q <= T) s_pick = n;  // the first run above T
        }
    }
    __syncthreads();
    long long pick = s_pick;
    if (pick < 0 || pick >= N) {  // cannot happen: the chunk sums and the scan agree
        if (tid == 0) st->err = 1;
        pick = 0;
    }
    for (int i = tid; i < D; i += blockDim.x) C[(long long)j * D + i] = X[pick * D + i];
    if (tid == 0) {
        idx[j] = pick;
        st->pick = pick;
        st->wmax = 0ull;  // the update of this centre recomputes it
    }
}

}  // namespace

cudaError_t launch_kmeanspp(const float *X, int64_t N, int D, int K, const double *u, float *C, long long *idx,
                            double *dmin, unsigned long long *bsum, void *state, cudaStream_t s, int num_sms,
                            long long *err_out) {
    PPState *st = static_cast<PPState *>(state);
    const long long nb = (N + kPPChunk - 1) / kPPChunk;
    const unsigned ug = (unsigned)std::min<int64_t>((N + kPPThreads - 1) / kPPThreads, (int64_t)num_sms * 16);
    cudaError_t e;
    count_launch();
    k_pp_first<<<1, 1, 0, s>>>(u, N, st);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // centre 0 is drawn by a pick over all-zero chunk sums (the uniform draw
    // floor(u_0 N)), which also copies its row out
    if ((e = cudaMemsetAsync(bsum, 0, (size_t)nb * 8, s)) != cudaSuccess) return e;
    for (int j = 0; j < K; ++j) {
        if (j > 0) {
            count_launch();
            k_pp_blocksum<<<(unsigned)nb, kPPThreads, 0, s>>>(dmin, N, st, bsum);
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
        }
        count_launch();
        k_pp_pick<<<1, 1024, 0, s>>>(X, N, D, dmin, bsum, nb, u, j, st, C, idx);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        count_launch();
        k_pp_update<<<ug, kPPThreads, 0, s>>>(X, N, D, dmin, st, j == 0 ? 1 : 0);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (err_out) return cudaMemcpyAsync(err_out, &st->err, 8, cudaMemcpyDeviceToHost, s);
    return cudaSuccess;
}

size_t kmeanspp_state_bytes() { return sizeof(PPState); }

}  // namespace kp

using namespace kp;

extern "C" {

KM_API int kmeans_init_kmeanspp(const float *X, int64_t N, int32_t D, int32_t K, const double *u, float *centroids,
                                int64_t *indices, void *stream) {
    auto fail = [](int code, const char *msg) {
        set_thread_error(msg);
        return code;
    };
    if (!X || !u || !centroids) return fail(KM_EINVAL, "a pointer argument is NULL");
    if (N < 1 || N >= ((int64_t)1 << 40) || D < 1 || D > 4096 || K < 1 || (int64_t)K > N)
        return fail(KM_EINVAL, "need 1 <= K <= N < 2^40 and 1 <= D <= 4096");
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, X) != cudaSuccess ||
        (a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(KM_EINVAL, "X must be device memory");
    }
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
        return fail(KM_ECUDA, "device query failed");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t nb = (N + 1023) / 1024;
    double *dmin = nullptr, *ud = nullptr;
    unsigned long long *bsum = nullptr;
    void *st = nullptr;
    float *Cd = nullptr;
    long long *idx = nullptr;
    long long err = 0;
    cudaError_t e = pool_alloc(dev, reinterpret_cast<void **>(&dmin), (size_t)N * 8, s);
    if (e == cudaSuccess) e = pool_alloc(dev, reinterpret_cast<void **>(&bsum), (size_t)nb * 8, s);
    if (e == cudaSuccess) e = pool_alloc(dev, &st, kmeanspp_state_bytes(), s);
    if (e == cudaSuccess) e = pool_alloc(dev, reinterpret_cast<void **>(&ud), (size_t)K * 8, s);
    if (e == cudaSuccess) e = pool_alloc(dev, reinterpret_cast<void **>(&Cd), (size_t)K * D * 4, s);
    if (e == cudaSuccess) e = pool_alloc(dev, reinterpret_cast<void **>(&idx), (size_t)K * 8, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ud, u, (size_t)K * 8, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = launch_kmeanspp(X, N, D, K, ud, Cd, idx, dmin, bsum, st, s, sms, &err);
    if (e == cudaSuccess) e = cudaMemcpyAsync(centroids, Cd, (size_t)K * D * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess && indices) e = cudaMemcpyAsync(indices, idx, (size_t)K * 8, cudaMemcpyDefault, s);
    for (void *p : {(void *)dmin, (void *)bsum, st, (void *)ud, (void *)Cd, (void *)idx})
        if (p) cudaFreeAsync(p, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA, cudaGetErrorString(e));
    }
    if (err) return fail(KM_ECUDA, "the draw produced an index out of range");
    return KM_OK;
}

}  // extern "C"
