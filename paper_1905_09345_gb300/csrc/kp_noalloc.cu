// kp_noalloc.cu -- one plain-Lloyd iteration that allocates nothing.
//
// For callers that may not allocate device memory at all: a host framework
// that owns every byte of device memory through its own pool, a
// latency-critical loop in which cudaMalloc / cudaFree would synchronise the
// device, or a deployment that must reserve all memory at start-up.  They
// pass X, C and the output arrays; every intermediate (FP64 cluster sums,
// counts, a padded centroid copy, the control block) lives in the
// file-scope array below, which each GPU that loads the library holds until
// the process exits.  The paper has no counterpart to this entry point.
#include <cuda.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "kp_common.cuh"

namespace kp {
namespace {

constexpr int kNaMaxK = 1024;  // KM_NOALLOC_MAX_K
constexpr int kNaMaxD = 128;   // KM_NOALLOC_MAX_D
constexpr int kNaMaxDp = 132;  // padded centroid row stride for D <= 128

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffStats = align256(kOffCtrl + sizeof(Ctrl));
constexpr size_t kOffC = align256(kOffStats + sizeof(kmeans_iter_stats));
constexpr size_t kOffS = align256(kOffC + sizeof(float) * kNaMaxK * kNaMaxDp);
constexpr size_t kOffQ = align256(kOffS + sizeof(double) * kNaMaxK * kNaMaxD);
constexpr size_t kOffCnt = align256(kOffQ + sizeof(double) * kNaMaxK);
constexpr size_t kOffJk = align256(kOffCnt + sizeof(unsigned long long) * kNaMaxK);
constexpr size_t kOffDelta = align256(kOffJk + sizeof(double) * kNaMaxK);
constexpr size_t kOffGrp = align256(kOffDelta + sizeof(float) * kNaMaxK);
constexpr size_t kOffGstart = align256(kOffGrp + sizeof(int32_t) * kNaMaxK);
constexpr size_t kOffDc = align256(kOffGstart + sizeof(int32_t) * 4);
constexpr size_t kOffDg = align256(kOffDc + sizeof(float) * 2 * kNaMaxK);
constexpr size_t kOffDm = align256(kOffDg + sizeof(float) * 2 * 4);
constexpr size_t kScratchBytes = align256(kOffDm + sizeof(float) * 2);  // about 1.6 MB

// The scratch itself.  Host code may not use `g_noalloc_scratch` as an
// address: its device address comes from cudaGetSymbolAddress, per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of the array, per device ordinal, with the context it was
// looked up in: a context destroyed and made again (cudaDeviceReset) loads the
// module again, so the address is looked up again when the context differs.
struct ScratchSlot {
    CUcontext ctx;
    void *ptr;
};
std::mutex g_mu;
ScratchSlot g_scratch[256] = {};

// the calling thread's current context (driver entry point, fetched once)
CUcontext current_context() {
    using Fn = CUresult (*)(CUcontext *);
    static std::once_flag once;
    static Fn fn = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<Fn>(f);
    });
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// group table of a single group holding every centroid: gstart = {0, K}
__global__ void k_noalloc_groups(int32_t *gstart, int K) {
    if (threadIdx.x == 0) {
        gstart[0] = 0;
        gstart[1] = K;
    }
}

// the J_t of the iteration (kept in the stats record) to the caller
__global__ void k_noalloc_objective(const kmeans_iter_stats *st, double *out) {
    if (threadIdx.x == 0) *out = st->objective;
}

float up32(double x) {
    float f = (float)x;
    return (double)f < x ? nextafterf(f, INFINITY) : f;
}
float dn32(double x) {
    float f = (float)x;
    return (double)f > x ? nextafterf(f, -INFINITY) : f;
}

bool on_device(const void *ptr, int dev) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

// the message is read back with kmeans_last_error(NULL)
int fail(int code, const char *msg) {
    set_thread_error(msg);
    return code;
}

}  // namespace
}  // namespace kp

using namespace kp;

extern "C" {

KM_API int kmeans_lloyd_step_noalloc(const float *X, int64_t N, int32_t D, const float *C, int32_t K,
                                     int32_t *labels, float *C_new, double *objective, void *stream) {
    if (!X || !C || !labels || !C_new || !objective) return fail(KM_EINVAL, "a pointer argument is NULL");
    if (N < 1 || N >= ((int64_t)1 << 31)) return fail(KM_EINVAL, "N out of range [1, 2^31)");
    if (D < 1 || D > kNaMaxD) return fail(KM_EINVAL, "D out of range [1, 128] for the allocation-free step");
    if (K < 1 || K > kNaMaxK || (int64_t)K > N)
        return fail(KM_EINVAL, "K out of range [1, min(N, 1024)] for the allocation-free step");
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return fail(KM_ECUDA, "cudaGetDevice failed");
    if (!on_device(X, dev) || !on_device(C, dev) || !on_device(labels, dev) || !on_device(C_new, dev) ||
        !on_device(objective, dev))
        return fail(KM_EINVAL, "every array must be device memory of the current device");

    // set-up once per device (and again if its context was made anew): the
    // scratch array's device address, looked up with that device current
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        const CUcontext cur = current_context();
        if (!cur) return fail(KM_ECUDA, "no current CUDA context");
        if (!g_scratch[dev].ptr || g_scratch[dev].ctx != cur) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) return fail(KM_ECUDA, "cudaGetSymbolAddress of the scratch array failed");
            g_scratch[dev].ptr = p;
            g_scratch[dev].ctx = cur;
        }
        base = g_scratch[dev].ptr;
    }
    unsigned char *b = static_cast<unsigned char *>(base);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    int num_sms = 0;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return fail(KM_ECUDA, "cudaDeviceGetAttribute failed");

    Params p;
    memset(&p, 0, sizeof(p));
    p.X = X;
    p.N = N;
    p.D = D;
    p.K = K;
    p.G = 1;
    const int dp = dense_dp(D);
    p.Dp = ((dp / 4) % 2 == 0) ? dp + 4 : dp;
    p.Gp = 4;
    p.tcap = 2;
    p.x_vec4 = (D % 4 == 0) && ((reinterpret_cast<uintptr_t>(X) & 15) == 0);
    p.label = labels;
    p.C = reinterpret_cast<float *>(b + kOffC);
    p.S = reinterpret_cast<double *>(b + kOffS);
    p.Q = reinterpret_cast<double *>(b + kOffQ);
    p.R = p.C;  // reference points = the centroids of this step (the update reads each before writing it)
    p.cnt = reinterpret_cast<unsigned long long *>(b + kOffCnt);
    p.Jk = reinterpret_cast<double *>(b + kOffJk);
    p.delta = reinterpret_cast<float *>(b + kOffDelta);
    p.grp = reinterpret_cast<const int32_t *>(b + kOffGrp);
    p.gstart = reinterpret_cast<const int32_t *>(b + kOffGstart);
    p.Dc = reinterpret_cast<float *>(b + kOffDc);
    p.Dg = reinterpret_cast<float *>(b + kOffDg);
    p.Dm = reinterpret_cast<float *>(b + kOffDm);
    p.ctrl = reinterpret_cast<Ctrl *>(b + kOffCtrl);
    p.stats = reinterpret_cast<kmeans_iter_stats *>(b + kOffStats);
    const double eps = (D + 4) * std::ldexp(1.0, -24) * (1.0 + 1.0 / 1024);
    p.eps_hi = up32(1.0 + 2.0 * eps);
    p.eps_lo = dn32(1.0 - eps);
    p.tiny = std::ldexp((float)(D + 4), -149);
    p.algo = KM_ALGO_LLOYD;

    // the array keeps the previous call's contents: clear everything this
    // step accumulates into or reads before writing
#define NA_CUDA(call)                                                           \
    do {                                                                        \
        cudaError_t e_ = (call);                                                \
        if (e_ != cudaSuccess) return fail(KM_ECUDA, cudaGetErrorString(e_));   \
    } while (0)
    NA_CUDA(cudaMemsetAsync(b, 0, kOffC, s));  // control block + stats record
    NA_CUDA(cudaMemsetAsync(p.C, 0, sizeof(float) * (size_t)K * p.Dp, s));
    NA_CUDA(cudaMemcpy2DAsync(p.C, sizeof(float) * p.Dp, C, sizeof(float) * D, sizeof(float) * D, K,
                              cudaMemcpyDeviceToDevice, s));
    NA_CUDA(cudaMemsetAsync(p.S, 0, sizeof(double) * (size_t)K * D, s));
    NA_CUDA(cudaMemsetAsync(p.Q, 0, sizeof(double) * K, s));
    NA_CUDA(cudaMemsetAsync(p.cnt, 0, sizeof(unsigned long long) * K, s));
    NA_CUDA(cudaMemsetAsync(b + kOffGrp, 0, sizeof(int32_t) * K, s));
    NA_CUDA(cudaMemsetAsync(b + kOffDc, 0, kScratchBytes - kOffDc, s));  // drift rows
    k_noalloc_groups<<<1, 32, 0, s>>>(reinterpret_cast<int32_t *>(b + kOffGstart), K);
    NA_CUDA(cudaGetLastError());
    count_launch();

    // the existing kernels: dense exact assignment, cluster sums, update
    NA_CUDA(launch_dense_assign(p, s, 1, 0, num_sms, 0));
    NA_CUDA(launch_apply_moves(p, s, 1, 0, num_sms, 0));
    NA_CUDA(launch_update(p, s, 0, 0));

    NA_CUDA(cudaMemcpy2DAsync(C_new, sizeof(float) * D, p.C, sizeof(float) * p.Dp, sizeof(float) * D, K,
                              cudaMemcpyDeviceToDevice, s));
    k_noalloc_objective<<<1, 32, 0, s>>>(p.stats, objective);
    NA_CUDA(cudaGetLastError());
    count_launch();
#undef NA_CUDA
    return KM_OK;
}

}  // extern "C"
