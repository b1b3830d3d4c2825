// kp_settle.cu -- the exact settle behind the tensor-core dense passes.
//
// The tensor-core passes (kp_dense_tc.cu, kp_dense_tcb.cu) estimate every
// distance with a bounded error; a row whose runner-up lies inside the error
// window of its winner is queued (a per-row request and one bit in a bitmap),
// and the kernels here decide it exactly from FP32 direct differences, with
// FP64 where the FP32 error bound cannot order the two smallest, so that the
// labels are those of the exact argmin (KPynq Sec. I: the distance
// calculator's result).
#include "kp_common.cuh"

namespace kp {
namespace {

// ---------------------------------------------------------------------------
// k_settle: the exact decision for the rows the tensor-core epilogue queued
// (runner-up inside the error window).  A sub-warp of D / 8 lanes per
// request, eight coordinates per lane, candidates one after another so that
// the sub-warp never diverges: FP32 direct-difference distances reduced
// across the sub-warp, the smallest with the lowest index; where FP32 cannot
// separate it from the runner-up, every candidate again in FP64 with the
// summation order of the FP64 definition (lanes over candidates).  The candidates are the centroids
// of the groups whose tensor-core minimum lies in the window (a group mask,
// or -- for the streamed-centroid pass -- the groups whose written bound is
// within the window's edge).  Writes the label, corrects u / lb / lbg when
// the winner is not i1, and appends label changes to the moved-point list
// 32 at a time.
// ---------------------------------------------------------------------------
constexpr int kSettleThreads = 256;
constexpr int kSettleWarps = kSettleThreads / 32;

// The bitmap's set bits, compacted into the settle queue: a warp takes 32
// words, scans their populations and reserves its slots with one atomic.
__global__ void k_settle_gather(Params p, int respect_done) {
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (*(volatile int *)&ctrl->path != KM_PATH_DENSE_TC) return;
    const int lane = threadIdx.x & 31;
    const int64_t nwords = (p.N + 31) / 32;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t w0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane; w0 < nwords; w0 += stride) {
        const int64_t w = w0 + lane;
        const uint32_t bits = w < nwords ? p.sbits[w] : 0u;
        const int c = __popc(bits);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int tot = __shfl_sync(0xffffffffu, incl, 31);
        int base = 0;
        if (lane == 31 && tot) base = atomicAdd(&ctrl->settle_count, tot);
        base = __shfl_sync(0xffffffffu, base, 31);
        int64_t pos = (int64_t)base + incl - c;
        for (uint32_t b = bits; b; b &= b - 1u) {
            const int64_t n = w * 32 + (__ffs(b) - 1);
            if (pos < p.N && n < p.N) p.squeue[pos] = (int32_t)n;
            ++pos;
        }
    }
}

// FP64 squared distance, i ascending, no fused multiply-add
__device__ __forceinline__ double settle_fp64(const float *x, const float *c, int D) {
    double s = 0.0;
    for (int i = 0; i < D; ++i) {
        const double t = __dsub_rn((double)__ldg(x + i), (double)c[i]);
        s = __dadd_rn(s, __dmul_rn(t, t));
    }
    return s;
}

template <int D>
__global__ void __launch_bounds__(kSettleThreads, 1) k_settle(Params p, int first, int respect_done, int staged) {
    // a request per SUB lanes, 8 coordinates per lane
    constexpr int PL = 8, SUB = D / PL, PER = 32 / SUB;
    extern __shared__ __align__(16) float sm_settle[];  // C (K x D) | group starts
    __shared__ int32_t mv_n[kSettleWarps][32], mv_old[kSettleWarps][32];  // moves not yet appended
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    // the requests of this iteration's dense pass, if it ran on the tensor cores
    if (*(volatile int *)&ctrl->path != KM_PATH_DENSE_TC) return;
    int64_t total = *(volatile int *)&ctrl->settle_count;
    if (total < 0 || total > p.N) {  // cannot happen: at most one request per row
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&ctrl->err, kErrQueue);
        total = 0;
    }
    const int warp_in = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int sub = lane / SUB, sl = lane - sub * SUB;  // sub-warp and lane in it
    const unsigned smask = (SUB == 32 ? 0xffffffffu : ((1u << SUB) - 1u)) << (sub * SUB);
    if ((int64_t)blockIdx.x * kSettleWarps * PER >= total) return;  // uniform per block
    const int K = p.K, G = p.G;
    // C in shared memory (row stride D) when it fits, else read from L2
    const int cst = staged ? D : p.Dp;
    const float *Cb = staged ? sm_settle : p.C;
    int32_t *gs_s = reinterpret_cast<int32_t *>(sm_settle + (staged ? (size_t)K * D : 0));
    if (staged)
        for (int i = threadIdx.x; i < K * (D / 4); i += kSettleThreads) {
            const int row = i / (D / 4), q4 = i - row * (D / 4);
            reinterpret_cast<float4 *>(sm_settle + (size_t)row * D)[q4] =
                __ldg(reinterpret_cast<const float4 *>(p.C + (size_t)row * p.Dp) + q4);
        }
    for (int i = threadIdx.x; i <= G; i += kSettleThreads) gs_s[i] = p.gstart[i];
    __syncthreads();
    const bool bounds = p.algo == KM_ALGO_FILTERED;
    unsigned long long c_changed = 0, c_recheck = 0;
    int mcount = 0;  // warp-uniform
    // append the buffered moves (one slot reservation per warp)
    auto flush_moves = [&]() {
        if (mcount) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&ctrl->moved_count, mcount);
            base = __shfl_sync(0xffffffffu, base, 0);
            if (lane < mcount) {
                p.moved[base + lane] = mv_n[warp_in][lane];
                p.moved_old[base + lane] = mv_old[warp_in][lane];
            }
            __syncwarp();
            mcount = 0;
        }
    };
    // dynamic schedule: each warp takes the next kGrab requests from a counter
    // (the requests differ in work; a fixed split leaves SMs idle at the end)
    // and gives them to its sub-warps, PER at a time (warp-uniform trips)
    constexpr int kGrab = 4 * PER;
    int r0 = 0, j = kGrab;  // the warp's current grab and its next unused slot
    for (;;) {
        if (j == kGrab) {
            if (lane == 0) r0 = atomicAdd(&ctrl->settle_next, kGrab);
            r0 = __shfl_sync(0xffffffffu, r0, 0);
            j = 0;
        }
        if (r0 >= total) break;
        const int64_t r = (int64_t)r0 + j + sub;
        j += PER;
        bool moved = false;
        int64_t n = -1;
        int old = -1;
        if (r < total) {
            n = p.squeue[r];
            const SettleReq q = p.sreq[n >= 0 && n < p.N ? n : 0];
            if (n < 0 || n >= p.N || q.n != n || (unsigned)q.i1 >= (unsigned)K) {  // sub-warp-uniform
                if (sl == 0) atomicExch(&ctrl->err, kErrQueue);
            } else {
                old = q.old;
                const float *xg = p.X + n * D;
                float xv[PL];
#pragma unroll
                for (int k4 = 0; k4 < PL / 4; ++k4) {
                    const float4 a = __ldg(reinterpret_cast<const float4 *>(xg + sl * PL) + k4);
                    xv[4 * k4] = a.x;
                    xv[4 * k4 + 1] = a.y;
                    xv[4 * k4 + 2] = a.z;
                    xv[4 * k4 + 3] = a.w;
                }
                // FP32 distance to centroid col, reduced across the sub-warp
                auto part = [&](int col) __attribute__((always_inline)) {
                    const float4 *cp = reinterpret_cast<const float4 *>(Cb + (size_t)col * cst + sl * PL);
                    float a0 = 0.f, a1 = 0.f;
#pragma unroll
                    for (int k4 = 0; k4 < PL / 4; ++k4) {
                        const float4 c = cp[k4];
                        const float d0 = xv[4 * k4] - c.x, d1 = xv[4 * k4 + 1] - c.y;
                        const float d2 = xv[4 * k4 + 2] - c.z, d3 = xv[4 * k4 + 3] - c.w;
                        a0 = fmaf(d0, d0, a0);
                        a1 = fmaf(d1, d1, a1);
                        a0 = fmaf(d2, d2, a0);
                        a1 = fmaf(d3, d3, a1);
                    }
                    return a0 + a1;
                };
                // the candidates in ascending index (a sub-warp-uniform walk)
                auto for_groups = [&](auto &&fn) __attribute__((always_inline)) {
                    if (q.gmask == ~0ull || (q.gmask == 0ull && !p.lb)) {
                        fn(0, K);
                        return;
                    }
                    if (q.gmask == 0ull) {  // the groups whose bound is within the window's edge
                        const float *lbr = p.lb + n * p.Gp;
                        for (int g0 = 0; g0 < G; g0 += SUB) {
                            const bool in = g0 + sl < G && lbr[g0 + sl] <= q.lim;
                            unsigned m = (__ballot_sync(smask, in) >> (sub * SUB)) &
                                         (SUB == 32 ? 0xffffffffu : ((1u << SUB) - 1u));
                            while (m) {
                                const int g = g0 + __ffs(m) - 1;
                                m &= m - 1;
                                fn(gs_s[g], gs_s[g + 1]);
                            }
                        }
                        return;
                    }
                    unsigned long long m = q.gmask;
                    while (m) {
                        const int g = __ffsll((long long)m) - 1;
                        m &= m - 1;
                        if (g >= G) break;
                        fn(gs_s[g], gs_s[g + 1]);
                    }
                };
                float s1 = INFINITY, s2 = INFINITY;
                int bi = q.i1;
                for_groups([&](int c0, int c1) __attribute__((always_inline)) {
                    for (int col = c0; col < c1; col += 2) {  // two at a time: independent chains
                        const bool two = col + 1 < c1;
                        float pa = part(col), pb = part(two ? col + 1 : col);
#pragma unroll
                        for (int o = SUB / 2; o > 0; o >>= 1) {
                            pa += __shfl_xor_sync(smask, pa, o, SUB);
                            pb += __shfl_xor_sync(smask, pb, o, SUB);
                        }
                        if (pa < s1) {
                            s2 = s1;
                            s1 = pa;
                            bi = col;
                        } else {
                            s2 = fminf(s2, pa);
                        }
                        if (two) {
                            if (pb < s1) {
                                s2 = s1;
                                s1 = pb;
                                bi = col + 1;
                            } else {
                                s2 = fminf(s2, pb);
                            }
                        }
                    }
                });
                float bs = s1;
                if (s2 != INFINITY && unresolved(s1, s2, p)) {
                    // FP64 over every candidate, lanes over candidates
                    double bd = INFINITY;
                    int bj = 0x7fffffff;
                    for_groups([&](int c0, int c1) __attribute__((always_inline)) {
                        for (int col = c0 + sl; col < c1; col += SUB) {
                            const double d64 = settle_fp64(xg, Cb + (size_t)col * cst, D);
                            if (d64 < bd || (d64 == bd && tie_key(p, col) < tie_key(p, bj))) {
                                bd = d64;
                                bj = col;
                            }
                        }
                    });
#pragma unroll
                    for (int o = SUB / 2; o > 0; o >>= 1) {
                        const double ov = __shfl_xor_sync(smask, bd, o, SUB);
                        const int oi = __shfl_xor_sync(smask, bj, o, SUB);
                        if (ov < bd || (ov == bd && tie_key(p, oi) < tie_key(p, bj))) {
                            bd = ov;
                            bj = oi;
                        }
                    }
                    if (bj != bi) {  // its FP32 distance, for u
                        float pc = part(bj);
#pragma unroll
                        for (int o = SUB / 2; o > 0; o >>= 1) pc += __shfl_xor_sync(smask, pc, o, SUB);
                        bs = pc;
                    }
                    bi = bj;
                    c_recheck += sl == 0 ? 1 : 0;
                }
                if (sl == 0) {
                    p.label[n] = bi;
                    if (bounds) {
                        p.u[n] = dist_up(bs, p);
                        if (bi != q.i1) {
                            p.lb[n * p.Gp + p.grp[q.i1]] = q.lb_alt;
                            p.lb[n * p.Gp + p.grp[bi]] = q.lb_alt;
                            p.lbg[n] = q.lb_alt;
                        }
                    }
                }
                moved = bi != old;
                c_changed += (moved && sl == 0) ? 1 : 0;
            }
        }
        // label changes: the sub-warp leaders' moves, appended 32 at a time
        __syncwarp();
        if (!first) {
            const unsigned mm = __ballot_sync(0xffffffffu, moved && sl == 0);
            if (mm) {
                const int k = mcount + __popc(mm & ((1u << lane) - 1u));
                if (moved && sl == 0) {
                    mv_n[warp_in][k] = (int32_t)n;
                    mv_old[warp_in][k] = old;
                }
                mcount += __popc(mm);
            }
            __syncwarp();
            if (mcount > 32 - PER) flush_moves();
        }
    }
    if (!first) flush_moves();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_changed += __shfl_xor_sync(0xffffffffu, c_changed, o);
        c_recheck += __shfl_xor_sync(0xffffffffu, c_recheck, o);
    }
    if (lane == 0) {
        if (c_changed) atomicAdd(&ctrl->n_changed, c_changed);
        if (c_recheck) atomicAdd(&ctrl->n_recheck, c_recheck);
    }
}

// The staged variant for short rows (D <= 64, C in shared memory): one
// thread per request with the row in registers.  Its candidate walks diverge
// across the warp, but with C in shared memory that costs less than the
// sub-warp reductions above (measured: about 100 against 135 us per pass on
// the 1M x 64, K = 256 workload).  The rare near-ties that need FP64 are
// settled afterwards by the whole warp, one request at a time.
// FP32 squared distance of the row (packed pairs in registers) to a centroid
// row in shared memory: packed FP32x2 subtract / fused multiply-add (each
// half an ordinary round-to-nearest FP32 operation; four partial sums)
template <int D>
__device__ __forceinline__ float settle_fp32(const ulonglong2 (&xr)[D / 4], const float *c) {
    const ulonglong2 *c2p = reinterpret_cast<const ulonglong2 *>(c);
    unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
    for (int i = 0; i < D / 4; ++i) {
        const ulonglong2 c2 = c2p[i];
        unsigned long long d0, d1;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(xr[i].x), "l"(c2.x));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(xr[i].y), "l"(c2.y));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a0) : "l"(d0));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a1) : "l"(d1));
    }
    float l0, h0, l1, h1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l0), "=f"(h0) : "l"(a0));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l1), "=f"(h1) : "l"(a1));
    return (l0 + h0) + (l1 + h1);
}
// The same FP32 distance with the row read from memory (16-byte aligned, D a
// multiple of 4): the packing and every rounding step of settle_fp32
template <int D>
__device__ __forceinline__ float settle_fp32_mem(const float *x, const float *c) {
    const ulonglong2 *x2p = reinterpret_cast<const ulonglong2 *>(x);
    const ulonglong2 *c2p = reinterpret_cast<const ulonglong2 *>(c);
    unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll 4
    for (int i = 0; i < D / 4; ++i) {
        const ulonglong2 x2 = __ldg(x2p + i);
        const ulonglong2 c2 = c2p[i];
        unsigned long long d0, d1;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(x2.x), "l"(c2.x));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(x2.y), "l"(c2.y));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a0) : "l"(d0));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a1) : "l"(d1));
    }
    float l0, h0, l1, h1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l0), "=f"(h0) : "l"(a0));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(l1), "=f"(h1) : "l"(a1));
    return (l0 + h0) + (l1 + h1);
}

template <int D>
__global__ void __launch_bounds__(kSettleThreads, 2) k_settle_t(Params p, int first, int respect_done, int staged) {
    static_assert(D <= 64 && D % 4 == 0, "the row lives in registers");
    extern __shared__ __align__(16) float sm_settle[];  // C (K rows, stride SD) | group starts
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    // the requests of this iteration's dense pass, if it ran on the tensor cores
    if (*(volatile int *)&ctrl->path != KM_PATH_DENSE_TC) return;
    int64_t total = *(volatile int *)&ctrl->settle_count;
    if (total < 0 || total > p.N) {  // cannot happen: at most one request per row
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&ctrl->err, kErrQueue);
        total = 0;
    }
    const int lane = threadIdx.x & 31;
    if ((int64_t)blockIdx.x * kSettleThreads >= total) return;  // uniform per block
    const int K = p.K, G = p.G;
    // C staged with a row stride of D + 4 floats (16-byte reads of different
    // rows by the threads of a warp spread over the banks), or read from
    // global memory when it does not fit
    const int SD = staged ? D + 4 : p.Dp;
    const float *Cs = staged ? sm_settle : p.C;
    int32_t *gs_s = reinterpret_cast<int32_t *>(sm_settle + (staged ? (size_t)K * SD : 0));
    if (staged)
        for (int i = threadIdx.x; i < K * (D / 4); i += kSettleThreads) {
            const int row = i / (D / 4), q4 = i - row * (D / 4);
            reinterpret_cast<float4 *>(sm_settle + (size_t)row * SD)[q4] =
                __ldg(reinterpret_cast<const float4 *>(p.C + (size_t)row * p.Dp) + q4);
        }
    for (int i = threadIdx.x; i <= G; i += kSettleThreads) gs_s[i] = p.gstart[i];
    __syncthreads();
    const bool bounds = p.algo == KM_ALGO_FILTERED;
    unsigned long long c_changed = 0, c_recheck = 0;
    // the candidates of a request: the centroids of the masked groups; all K
    // when the mask holds every group
    auto all_of = [&](const SettleReq &q) { return q.gmask == ~0ull || (q.gmask == 0ull && !p.lb); };
    // dynamic schedule: each warp takes the next 32 requests (one per lane)
    // from a counter; the requests differ in work, and a fixed split left
    // many SMs idle while a few finished their share
    for (;;) {
        int r0 = 0;
        if (lane == 0) r0 = atomicAdd(&ctrl->settle_next, 32);
        r0 = __shfl_sync(0xffffffffu, r0, 0);
        if (r0 >= total) break;
        const int64_t r = (int64_t)r0 + lane;
        bool act = r < total;
        int64_t n = 0;
        SettleReq q;
        q.n = -1;
        q.old = -1;
        q.i1 = 0;
        q.lb_alt = 0.f;
        q.gmask = 0ull;
        q.lim = 0.f;
        if (act) {
            n = p.squeue[r];
            if (n < 0 || n >= p.N) {
                atomicExch(&ctrl->err, kErrQueue);
                act = false;
            }
        }
        if (act) {
            q = p.sreq[n];
            if (q.n != n || (unsigned)q.i1 >= (unsigned)K) {
                atomicExch(&ctrl->err, kErrQueue);
                act = false;
            }
        }
        float s1 = INFINITY, s2 = INFINITY;
        int bi = q.i1;
        if (act) {
            // the row in registers
            ulonglong2 xr[D / 4];
            {
                const ulonglong2 *xp = reinterpret_cast<const ulonglong2 *>(p.X + n * D);
#pragma unroll
                for (int i = 0; i < D / 4; ++i) xr[i] = __ldg(xp + i);
            }
            // smallest (first in ascending order on ties) and runner-up over the
            // candidates in ascending index
            auto visit = [&](int col) {
                const float sx = settle_fp32<D>(xr, Cs + (size_t)col * SD);
                if (sx < s1) {
                    s2 = s1;
                    s1 = sx;
                    bi = col;
                } else {
                    s2 = fminf(s2, sx);
                }
            };
            if (all_of(q)) {
                for (int col = 0; col < K; ++col) visit(col);
            } else if (q.gmask == 0ull) {  // the groups whose bound is within the window's edge
                const float *lbr = p.lb + n * p.Gp;
                for (int g = 0; g < G; ++g)
                    if (lbr[g] <= q.lim)
                        for (int col = gs_s[g]; col < gs_s[g + 1]; ++col) visit(col);
            } else {
                unsigned long long m = q.gmask;
                while (m) {
                    const int g = __ffsll((long long)m) - 1;
                    m &= m - 1;
                    if (g >= G) break;
                    for (int col = gs_s[g]; col < gs_s[g + 1]; ++col) visit(col);
                }
            }
        }
        float bs = s1;
        // near-ties (FP32 cannot order the two smallest): the smallest FP64
        // distance among the candidates that FP32 cannot separate from s1,
        // lowest index on equal distances; settled one request at a time by the
        // whole warp, lanes over the centroids, so that one lane's FP64 work
        // does not hold up the warp's other requests
        const bool rc = act && s2 != INFINITY && unresolved(s1, s2, p);
        unsigned rm = __ballot_sync(0xffffffffu, rc);
        while (rm) {
            const int src = __ffs(rm) - 1;
            rm &= rm - 1;
            const int64_t nr = __shfl_sync(0xffffffffu, n, src);
            const float s1r = __shfl_sync(0xffffffffu, s1, src);
            const int bir = __shfl_sync(0xffffffffu, bi, src);
            SettleReq qr;
            qr.gmask = __shfl_sync(0xffffffffu, q.gmask, src);
            qr.lim = __shfl_sync(0xffffffffu, q.lim, src);
            const bool all = all_of(qr);
            const float *xg = p.X + nr * D;
            const float *lbr = p.lb + nr * p.Gp;
            double bd = INFINITY;
            int bj = 0x7fffffff;
            for (int c = lane; c < K; c += 32) {  // ascending: the first of equal distances stays
                bool cand = all;
                if (!cand) {
                    const int g = p.grp[c];
                    cand = qr.gmask == 0ull ? lbr[g] <= qr.lim : (g < 64 && ((qr.gmask >> g) & 1ull));
                }
                if (!cand || !unresolved(s1r, settle_fp32_mem<D>(xg, Cs + (size_t)c * SD), p)) continue;
                const double d64 = settle_fp64(xg, Cs + (size_t)c * SD, D);
                if (d64 < bd || (d64 == bd && tie_key(p, c) < tie_key(p, bj))) {
                    bd = d64;
                    bj = c;
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bd, o);
                const int oi = __shfl_xor_sync(0xffffffffu, bj, o);
                if (ov < bd || (ov == bd && tie_key(p, oi) < tie_key(p, bj))) {
                    bd = ov;
                    bj = oi;
                }
            }
            // bir is among them (its own FP32 distance is s1r)
            if (bj == 0x7fffffff) bj = bir;
            const float bsr = bj != bir ? settle_fp32_mem<D>(xg, Cs + (size_t)bj * SD) : s1r;
            if (lane == src) {
                bi = bj;
                bs = bsr;
                c_recheck += 1;
            }
        }
        bool moved = false;
        if (act) {
            p.label[n] = bi;
            if (bounds) {
                p.u[n] = dist_up(bs, p);
                if (bi != q.i1) {
                    p.lb[n * p.Gp + p.grp[q.i1]] = q.lb_alt;
                    p.lb[n * p.Gp + p.grp[bi]] = q.lb_alt;
                    p.lbg[n] = q.lb_alt;
                }
            }
            moved = bi != q.old;
            c_changed += moved ? 1 : 0;
        }
        // label changes: one slot reservation per warp
        if (!first) {
            const unsigned mm = __ballot_sync(0xffffffffu, moved);
            if (mm) {
                int base = 0;
                if (lane == 0) base = atomicAdd(&ctrl->moved_count, __popc(mm));
                base = __shfl_sync(0xffffffffu, base, 0);
                if (moved) {
                    const int slot = base + __popc(mm & ((1u << lane) - 1u));
                    p.moved[slot] = (int32_t)n;
                    p.moved_old[slot] = q.old;
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_changed += __shfl_xor_sync(0xffffffffu, c_changed, o);
        c_recheck += __shfl_xor_sync(0xffffffffu, c_recheck, o);
    }
    if (lane == 0) {
        if (c_changed) atomicAdd(&ctrl->n_changed, c_changed);
        if (c_recheck) atomicAdd(&ctrl->n_recheck, c_recheck);
    }
}

}  // namespace

cudaError_t launch_settle(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms) {
    if (p.D != 32 && p.D != 64 && p.D != 128) return cudaErrorInvalidValue;
    // compact the request bitmap (one warp per 32 words), then one thread per request
    const int64_t words = (p.N + 31) / 32;
    const int64_t gblocks = std::max<int64_t>(1, std::min<int64_t>((words + 255) / 256, (int64_t)num_sms * 8));
    count_launch();
    k_settle_gather<<<(unsigned)gblocks, 256, 0, s>>>(p, respect_done);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // C in shared memory when it fits (up to 160 KB), else read from L2; short
    // rows with C in shared memory: thread per request (C rows padded by 4
    // floats), else sub-warps (C rows unpadded)
    const int staged = (size_t)p.K * (p.D + 4) * 4 <= ((size_t)160 << 10);
    const bool per_thread = staged && p.D <= 64;
    const size_t cbytes = staged ? (size_t)p.K * (p.D + (per_thread ? 4 : 0)) * 4 : 0;
    const size_t smem = cbytes + (size_t)(p.G + 1) * 4;
    auto kern = per_thread ? (p.D == 32 ? k_settle_t<32> : k_settle_t<64>)
                           : (p.D == 32 ? k_settle<32> : (p.D == 64 ? k_settle<64> : k_settle<128>));
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSettleThreads, smem);
    if (e != cudaSuccess) return e;
    count_launch();
    kern<<<(unsigned)(num_sms * std::max(per_sm, 1)), kSettleThreads, smem, s>>>(p, first, respect_done, staged);
    return cudaGetLastError();
}

}  // namespace kp
