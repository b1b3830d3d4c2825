// kp_selftest.cu -- device self-test of the square-root bounds.
//
// Every distance bound of the method (Sec. I: the upper bound u and the
// lower bounds lb of the triangle-inequality filters) passes through sqrt_lo /
// sqrt_hi, which wrap the hardware square-root approximation with a margin of
// two steps of the bit pattern.  This checks the margin on the running device
// for every non-negative float v, exactly: lo >= 0, lo^2 <= v <= hi^2, with
// the squares formed in FP64 (a product of two floats is exact there).
#include "kp_common.cuh"

namespace kp {
namespace {

__global__ void k_selftest_sqrt(unsigned long long *violations) {
    unsigned long long bad = 0;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long u = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; u < 0x80000000ull;
         u += stride) {
        const float v = __uint_as_float((uint32_t)u);
        if (v != v) continue;  // NaN bit patterns
        const float lo = sqrt_lo(v), hi = sqrt_hi(v);
        const double dv = (double)v, dl = (double)lo, dh = (double)hi;
        bad += (lo < 0.f) || (lo != lo) || (hi != hi) || !(dl * dl <= dv) || !(dh * dh >= dv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(violations, bad);
}

// One thread waits, with the bounded mbarrier wait every kernel of the library
// uses, on a barrier that expects one arrival that never comes; when the wait
// gives up it records KM_ETIMEOUT in the control block's error word, the way
// the library's kernels do, and returns.  Nothing is in flight on the barrier.
__global__ void k_selftest_timeout(uint32_t polls, Ctrl *ctrl) {
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    if (!mbar_wait_bounded(&bar, 0, polls)) atomicExch(&ctrl->err, (int)KM_ETIMEOUT);
}

int fail_msg(int code, const char *msg) {
    set_thread_error(msg);
    return code;
}

}  // namespace
}  // namespace kp

using namespace kp;

extern "C" {

KM_API int kmeans_selftest_sqrt(int64_t *violations) {
    if (!violations) return fail_msg(KM_EINVAL, "violations is NULL");
    unsigned long long *d = nullptr;
    if (cudaMalloc(&d, sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(KM_ENOMEM, "cudaMalloc failed");
    }
    unsigned long long h = 0;
    cudaError_t e = cudaMemset(d, 0, sizeof(h));
    int sms = 0, dev = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        k_selftest_sqrt<<<sms * 8, 256>>>(d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(KM_ECUDA, cudaGetErrorString(e));
    }
    *violations = (int64_t)h;
    return KM_OK;
}

}  // extern "C"

extern "C" {

KM_API int kmeans_selftest_timeout(int32_t polls) {
    if (polls < 1 || polls > (1 << 16)) return fail_msg(KM_EINVAL, "polls out of range [1, 65536]");
    Ctrl *d = nullptr;
    if (cudaMalloc(&d, sizeof(Ctrl)) != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(KM_ENOMEM, "cudaMalloc failed");
    }
    Ctrl h;
    cudaError_t e = cudaMemset(d, 0, sizeof(Ctrl));
    if (e == cudaSuccess) {
        k_selftest_timeout<<<1, 32>>>((uint32_t)polls, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail_msg(KM_ECUDA, cudaGetErrorString(e));
    }
    if (h.err == KM_ETIMEOUT) return fail_msg(KM_ETIMEOUT, "a bounded device-side wait gave up");
    return KM_OK;
}

}  // extern "C"
