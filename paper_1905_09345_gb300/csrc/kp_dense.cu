// kp_dense.cu -- dense assignment (every point against every centroid) and
// the cluster-statistics update for the points it moved.
//
// Used for iteration 0 of the filtered method, where every bound is created
// (KPynq Sec. I: the distance calculator evaluates whatever the filters have
// not removed, and at t = 0 nothing is removed yet), and for every iteration
// of plain Lloyd, the comparison baseline.
//
// One thread per point: x lives in registers, centroid tiles are staged in
// shared memory and read by all threads at the same address (broadcast).  The
// distance is the direct difference sum (x_i - c_i)^2 in FP32; its rounding
// error is bounded (Params::eps_hi/eps_lo), and when the two nearest FP32
// values cannot be ordered by that bound the point is settled in FP64 with the
// summation order of the FP64 definition, so labels are exact.
#include "kp_common.cuh"

namespace kp {

constexpr int kDenseThreads = 128;
constexpr int kDenseTileBytes = 64 * 1024;

template <int DP>
struct XRow {
    float v[DP];
};

// squared distance of x (registers) to centroid row c (shared, DP floats)
template <int DP>
__device__ __forceinline__ float sqdist_reg(const XRow<DP> &x, const float *__restrict__ c) {
    float a0 = 0.f, a1 = 0.f;
#pragma unroll
    for (int i = 0; i < DP; i += 8) {
        float4 c0 = *reinterpret_cast<const float4 *>(c + i);
        float t0 = x.v[i + 0] - c0.x, t1 = x.v[i + 1] - c0.y;
        float t2 = x.v[i + 2] - c0.z, t3 = x.v[i + 3] - c0.w;
        a0 = fmaf(t0, t0, a0);
        a0 = fmaf(t1, t1, a0);
        a0 = fmaf(t2, t2, a0);
        a0 = fmaf(t3, t3, a0);
        if (i + 4 < DP) {
            float4 c1 = *reinterpret_cast<const float4 *>(c + i + 4);
            float u0 = x.v[i + 4] - c1.x, u1 = x.v[i + 5] - c1.y;
            float u2 = x.v[i + 6] - c1.z, u3 = x.v[i + 7] - c1.w;
            a1 = fmaf(u0, u0, a1);
            a1 = fmaf(u1, u1, a1);
            a1 = fmaf(u2, u2, a1);
            a1 = fmaf(u3, u3, a1);
        }
    }
    return a0 + a1;
}

// generic D: x and c in global memory (c with stride Dp)
__device__ __forceinline__ float sqdist_gen(const float *__restrict__ x, const float *__restrict__ c, int D) {
    float a0 = 0.f, a1 = 0.f;
    int i = 0;
    for (; i + 1 < D; i += 2) {
        float t0 = x[i] - c[i], t1 = x[i + 1] - c[i + 1];
        a0 = fmaf(t0, t0, a0);
        a1 = fmaf(t1, t1, a1);
    }
    if (i < D) {
        float t0 = x[i] - c[i];
        a0 = fmaf(t0, t0, a0);
    }
    return a0 + a1;
}

template <int DP>
__device__ __forceinline__ void load_x(XRow<DP> &x, const Params &p, int64_t n) {
    const float *row = p.X + n * p.D;
    if (p.x_vec4 && DP == p.D) {
#pragma unroll
        for (int i = 0; i < DP; i += 4) {
            float4 t = __ldg(reinterpret_cast<const float4 *>(row + i));
            x.v[i] = t.x;
            x.v[i + 1] = t.y;
            x.v[i + 2] = t.z;
            x.v[i + 3] = t.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < DP; ++i) x.v[i] = i < p.D ? __ldg(row + i) : 0.f;
    }
}

// The FP32 value of the distance from point n to centroid c, computed exactly
// as in the main loop (global-memory operands; same arithmetic, same order).
template <int DP>
__device__ __forceinline__ float sqdist_again(const Params &p, const XRow<(DP > 0 ? DP : 1)> &x, int64_t n, int c) {
    if constexpr (DP > 0) {
        return sqdist_reg<DP>(x, p.C + (size_t)c * p.Dp);
    } else {
        return sqdist_gen(p.X + n * p.D, p.C + (size_t)c * p.Dp, p.D);
    }
}

// Dense assignment.  first: iteration 0 of this context (all points count as
// moved and are added to the sums by the caller).  Writes labels; for the
// filtered method also u, lbg, lb and stamps (exact at the current version).
template <int DP>
__global__ void __launch_bounds__(kDenseThreads) k_dense_assign(Params p, int first, int respect_done, int if_dense) {
    extern __shared__ __align__(128) float smem[];
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (if_dense && !*(volatile int *)&ctrl->dense_mode) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->path = KM_PATH_DENSE_FP32;
    const int v = ctrl->v;
    const int K = p.K;
    const int G = p.G;
    const bool bounds = p.algo == KM_ALGO_FILTERED;
    constexpr int DPs = DP > 0 ? DP : 4;  // shared row stride (unused for DP = 0)
    const int KT = DP > 0 ? min(K, kDenseTileBytes / (DPs * 4)) : 0;
    float *cs = smem;
    const int lbs_stride = p.Gp + 1;
    const bool stage_lb = bounds && (size_t)lbs_stride * kDenseThreads * 4 <= 48 * 1024;
    float *lbs = smem + (size_t)KT * DPs;
    const bool c_resident = DP > 0 && KT == K;

    if (c_resident) {  // whole centroid set fits: stage once for all point tiles
        for (int idx = threadIdx.x; idx < K * (DPs / 4); idx += blockDim.x) {
            int r = idx / (DPs / 4), q = idx % (DPs / 4);
            reinterpret_cast<float4 *>(cs)[idx] = *reinterpret_cast<const float4 *>(p.C + (size_t)r * p.Dp + q * 4);
        }
        __syncthreads();
    }

    unsigned long long my_changed = 0, my_recheck = 0;
    for (int64_t base = (int64_t)blockIdx.x * kDenseThreads; base < p.N; base += (int64_t)gridDim.x * kDenseThreads) {
        const int64_t n = base + threadIdx.x;
        const bool active = n < p.N;
        XRow<(DP > 0 ? DP : 1)> x;
        if constexpr (DP > 0) {
            if (active) load_x<DP>(x, p, n);
            else {
#pragma unroll
                for (int i = 0; i < DP; ++i) x.v[i] = 0.f;
            }
        }
        int best = 0;
        float s1 = INFINITY, s2 = INFINITY;   // best / second-best over all centroids
        int cur_g = 0;
        float gm1 = INFINITY, gm2 = INFINITY;  // two smallest in the current group
        float bg_m2 = INFINITY;                // second smallest of the best's group
        bool best_in_cur = false;

        auto close_group = [&](int g) {
            if (bounds && active) {
                float d = gm1 == INFINITY ? INFINITY : dist_dn(gm1, p);
                if (stage_lb) lbs[threadIdx.x * lbs_stride + g] = d;
                else p.lb[n * p.Gp + g] = d;
            }
            if (best_in_cur) bg_m2 = gm2;
            best_in_cur = false;
            gm1 = gm2 = INFINITY;
        };
        auto visit = [&](int c, float s) {
            int g = p.grp[c];
            if (g != cur_g) {
                close_group(cur_g);
                cur_g = g;
            }
            if (s < gm1) { gm2 = gm1; gm1 = s; }
            else if (s < gm2) gm2 = s;
            if (s < s1) {
                s2 = s1;
                s1 = s;
                best = c;
                best_in_cur = true;
            } else if (s < s2) {
                s2 = s;
            }
        };

        if constexpr (DP > 0) {
            for (int c0 = 0; c0 < K; c0 += KT) {
                const int kt = min(KT, K - c0);
                if (!c_resident) {
                    __syncthreads();
                    for (int idx = threadIdx.x; idx < kt * (DP / 4); idx += blockDim.x) {
                        int r = idx / (DP / 4), q = idx % (DP / 4);
                        reinterpret_cast<float4 *>(cs)[idx] =
                            *reinterpret_cast<const float4 *>(p.C + (size_t)(c0 + r) * p.Dp + q * 4);
                    }
                    __syncthreads();
                }
                int j = 0;
                for (; j + 1 < kt; j += 2) {
                    float sa = sqdist_reg<DP>(x, cs + (size_t)j * DP);
                    float sb = sqdist_reg<DP>(x, cs + (size_t)(j + 1) * DP);
                    visit(c0 + j, sa);
                    visit(c0 + j + 1, sb);
                }
                if (j < kt) visit(c0 + j, sqdist_reg<DP>(x, cs + (size_t)j * DP));
            }
        } else {
            if (active) {
                const float *xr = p.X + n * p.D;
                for (int c = 0; c < K; ++c) visit(c, sqdist_gen(xr, p.C + (size_t)c * p.Dp, p.D));
            }
        }
        close_group(cur_g);

        if (active) {
            // near-tie: settle in FP64 among every centroid the FP32 error
            // bound cannot separate from the FP32 best
            if (s2 != INFINITY && unresolved(s1, s2, p)) {
                const float s1_ref = s1;
                double bd = INFINITY;
                int bi = best;
                float bs = s1;
                for (int c = 0; c < K; ++c) {
                    float s = sqdist_again<DP>(p, x, n, c);
                    if (!unresolved(s1_ref, s, p)) continue;
                    double d64 = dist2_f64(p.X + n * p.D, p.C + (size_t)c * p.Dp, p.D);
                    if (d64 < bd || (d64 == bd && tie_key(p, c) < tie_key(p, bi))) { bd = d64; bi = c; bs = s; }
                }
                my_recheck += 1;
                if (bi != best) {
                    best = bi;
                    s1 = bs;
                    if (bounds) {  // group bounds must now exclude the new best
                        for (int g = 0; g < G; ++g) {
                            float m = INFINITY;
                            for (int c = p.gstart[g]; c < p.gstart[g + 1]; ++c)
                                if (c != best) m = fminf(m, sqdist_again<DP>(p, x, n, c));
                            float d = m == INFINITY ? INFINITY : dist_dn(m, p);
                            if (stage_lb) lbs[threadIdx.x * lbs_stride + g] = d;
                            else p.lb[n * p.Gp + g] = d;
                        }
                        bg_m2 = -1.f;  // already written
                    }
                }
            }
            if (bounds && bg_m2 >= 0.f) {
                int g = p.grp[best];
                float d = bg_m2 == INFINITY ? INFINITY : dist_dn(bg_m2, p);
                if (stage_lb) lbs[threadIdx.x * lbs_stride + g] = d;
                else p.lb[n * p.Gp + g] = d;
            }
            const int old = first ? -1 : p.label[n];
            p.label[n] = best;
            if (bounds) {
                p.u[n] = dist_up(s1, p);
                p.stamp[n] = make_stamp(v, v);
            }
            if (old != best) {
                my_changed += 1;
                if (!first) {
                    int slot = atomicAdd(&ctrl->moved_count, 1);
                    p.moved[slot] = (int)n;
                    p.moved_old[slot] = old;
                }
            }
        }
        if (bounds) {
            if (stage_lb) {
                __syncthreads();
                // lbg = min over the row, then a coalesced copy of the rows
                if (active) {
                    float m = INFINITY;
                    for (int g = 0; g < G; ++g) m = fminf(m, lbs[threadIdx.x * lbs_stride + g]);
                    p.lbg[n] = m;
                }
                const int64_t rows = min((int64_t)kDenseThreads, p.N - base);
                for (int64_t idx = threadIdx.x; idx < rows * p.Gp; idx += blockDim.x) {
                    int64_t r = idx / p.Gp;
                    int g = (int)(idx % p.Gp);
                    p.lb[(base + r) * p.Gp + g] = g < G ? lbs[r * lbs_stride + g] : 0.f;
                }
                __syncthreads();
            } else if (active) {
                float m = INFINITY;
                for (int g = 0; g < G; ++g) m = fminf(m, p.lb[n * p.Gp + g]);
                p.lbg[n] = m;
            }
        }
    }
    // counters: one atomic per warp
    unsigned long long ch = my_changed, rc = my_recheck;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        ch += __shfl_xor_sync(0xffffffffu, ch, o);
        rc += __shfl_xor_sync(0xffffffffu, rc, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (ch) atomicAdd(&ctrl->n_changed, ch);
        if (rc) atomicAdd(&ctrl->n_recheck, rc);
        int64_t lo = (int64_t)blockIdx.x * kDenseThreads + (threadIdx.x & ~31);
        (void)lo;
    }
    if (threadIdx.x == 0) {
        // points this block assigned, times K distances each
        int64_t pts = 0;
        for (int64_t base = (int64_t)blockIdx.x * kDenseThreads; base < p.N; base += (int64_t)gridDim.x * kDenseThreads)
            pts += min((int64_t)kDenseThreads, p.N - base);
        atomicAdd(&ctrl->n_dist, (unsigned long long)(pts * K));
    }
}

// Cluster statistics for moved points: S[new] += x, S[old] -= x (FP64),
// Q (sum of ||x||^2) and counts likewise.  One warp per point, lanes over the
// coordinates, so each point's atomics are coalesced.
__global__ void __launch_bounds__(256) k_apply_moves(Params p, int all_points, int respect_done, int if_dense) {
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (if_dense && !*(volatile int *)&ctrl->dense_mode) return;
    if (*(volatile int *)&ctrl->stats_full) return;  // recomputed in full instead
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int64_t count = all_points ? p.N : (int64_t)ctrl->moved_count;
    for (int64_t it = warp; it < count; it += nwarps) {
        int64_t n;
        int old;
        if (all_points) { n = it; old = -1; }
        else { n = p.moved[it]; old = p.moved_old[it]; }
        const int nw = checked_label(p, n);
        if (nw < 0) continue;  // warp-uniform: one point per warp
        const float *x = p.X + n * p.D;
        // ||x - R_k||^2 for the new and the old cluster as FP32 pairs (exact
        // squares, compensated sums): FP64 arithmetic is slow on these SMs;
        // only the atomics are FP64
        float qh = 0.f, ql = 0.f, oh = 0.f, ol = 0.f;
        auto two_sum = [](float a, float b, float &s, float &e) {  // s + e == a + b exactly
            s = __fadd_rn(a, b);
            const float bb = __fsub_rn(s, a);
            e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
        };
        // (x - r)^2 into the pair (h, l): x - r as the exact pair dh + dl, its
        // square as sq + sqe (exact) plus 2 dh dl + dl^2 (below 2^-47 of it)
        auto acc = [&](float &h, float &l, float xv, float r) {
            float dh, dl, s, e;
            two_sum(xv, -r, dh, dl);
            const float sq = __fmul_rn(dh, dh);
            const float sqe = __fmaf_rn(dh, dh, -sq);
            const float cross = __fmaf_rn(__fmul_rn(2.f, dh), dl, __fmul_rn(dl, dl));
            two_sum(h, sq, s, e);
            h = s;
            l = __fadd_rn(l, __fadd_rn(e, __fadd_rn(sqe, cross)));
        };
        for (int i = lane; i < p.D; i += 32) {
            const float xf = __ldg(x + i);
            acc(qh, ql, xf, p.R[(size_t)nw * p.Dp + i]);
            if (old >= 0) acc(oh, ol, xf, p.R[(size_t)old * p.Dp + i]);
            const double xi = (double)xf;
            atomicAdd(&p.S[(size_t)nw * p.D + i], xi);
            if (old >= 0) atomicAdd(&p.S[(size_t)old * p.D + i], -xi);
        }
        const double q = warp_sum_d((double)qh + (double)ql);
        const double qo = warp_sum_d((double)oh + (double)ol);
        if (lane == 0) {
            atomicAdd(&p.Q[nw], q);
            atomicAdd(&p.cnt[nw], 1ull);
            if (old >= 0) {
                atomicAdd(&p.Q[old], -qo);
                atomicAdd(&p.cnt[old], ~0ull);  // -1
            }
        }
    }
}

int dense_dp(int D) {
    if (D <= 4) return 4;
    if (D <= 8) return 8;
    if (D <= 16) return 16;
    if (D <= 32) return 32;
    if (D <= 64) return 64;
    if (D <= 128) return 128;
    return 0;
}

template <int DP>
static cudaError_t launch_dense_t(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms,
                                  int if_dense) {
    constexpr int DPs = DP > 0 ? DP : 4;
    const int KT = DP > 0 ? std::min(p.K, kDenseTileBytes / (DPs * 4)) : 0;
    size_t smem = (size_t)KT * DPs * 4;
    const bool bounds = p.algo == KM_ALGO_FILTERED;
    if (bounds && (size_t)(p.Gp + 1) * kDenseThreads * 4 <= 48 * 1024) smem += (size_t)(p.Gp + 1) * kDenseThreads * 4;
    cudaError_t e = cudaFuncSetAttribute(k_dense_assign<DP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dense_assign<DP>, kDenseThreads, smem);
    if (e != cudaSuccess) return e;
    int64_t tiles = (p.N + kDenseThreads - 1) / kDenseThreads;
    int64_t grid = std::min<int64_t>(tiles, (int64_t)num_sms * std::max(per_sm, 1));
    count_launch();
    k_dense_assign<DP><<<(unsigned)grid, kDenseThreads, smem, s>>>(p, first, respect_done, if_dense);
    return cudaGetLastError();
}

cudaError_t launch_dense_assign(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms,
                                int if_dense) {
    switch (dense_dp(p.D)) {
    case 4: return launch_dense_t<4>(p, s, first, respect_done, num_sms, if_dense);
    case 8: return launch_dense_t<8>(p, s, first, respect_done, num_sms, if_dense);
    case 16: return launch_dense_t<16>(p, s, first, respect_done, num_sms, if_dense);
    case 32: return launch_dense_t<32>(p, s, first, respect_done, num_sms, if_dense);
    case 64: return launch_dense_t<64>(p, s, first, respect_done, num_sms, if_dense);
    case 128: return launch_dense_t<128>(p, s, first, respect_done, num_sms, if_dense);
    default: return launch_dense_t<0>(p, s, first, respect_done, num_sms, if_dense);
    }
}

cudaError_t launch_apply_moves(const Params &p, cudaStream_t s, int all_points, int respect_done, int num_sms,
                               int if_dense) {
    int64_t items = all_points ? p.N : p.N;  // moved count is only known on the device
    int64_t grid = std::min<int64_t>((items + 7) / 8, (int64_t)num_sms * 8);
    grid = std::max<int64_t>(grid, 1);
    count_launch();
    k_apply_moves<<<(unsigned)grid, 256, 0, s>>>(p, all_points, respect_done, if_dense);
    return cudaGetLastError();
}

}  // namespace kp
