// kp_survivor_tp.cu -- the filtered assignment of the survivors, one thread
// per point (D <= 128).
//
// The survivors of the global filter (KPynq Sec. I: the "Multi-level Filters"
// in front of the "Distance Calculator") mostly need very little work: the
// tightened own distance, one group-bound test per group, and on average
// fewer than one further distance.  A warp per point leaves that work
// latency-bound on shuffles and dependent loads, so here each thread owns one
// queued point:
//
//   * the point's coordinates live in registers (D/4 float4 loads);
//   * the centroids (K x Dp FP32) are staged in shared memory by TMA bulk
//     copies when they fit, else read through the read-only path;
//   * the stored group bounds are read and rewritten in place, one row per
//     thread (the row's cache lines stay in L1 between the reads);
//   * groups are visited in index order with a running best, so the group
//     filter and the point filter test against the best distance found so
//     far (a valid upper bound of the final best);
//   * each group's refreshed bound is the smallest lower value of its
//     centroids other than the final best: every centroid contributes either
//     its computed distance (rounded down) or its point-filter bound, and the
//     group that holds the running best keeps both the value that excludes
//     the best and the value that includes it, in case the best moves on;
//   * a point whose FP32 best and runner-up cannot be separated by the FP32
//     error bound is settled over all K centroids, in FP64 where needed, and
//     its bounds are rebuilt from that full scan -- by the whole warp, after
//     the batch's points are done, so that one lane does not hold up the
//     other 31 (and the SM) for the length of a K-centroid scan;
//   * label changes go to the moved-point list; the cluster sums are updated
//     by the moves kernel afterwards.
#include "kp_common.cuh"

namespace kp {
namespace {

constexpr int kTpThreads = 256;

// x is kept as packed pairs of FP32 values: xr[q] holds coordinates
// 4q .. 4q+3 as two 64-bit registers (low half = lower coordinate)
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack2(unsigned long long v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ float hsum2(unsigned long long v) {
    float lo, hi;
    unpack2(v, lo, hi);
    return lo + hi;
}

// Direct-difference squared distance sum_i (x_i - c_i)^2 with packed FP32x2
// subtract and fused multiply-add (each lane of a pair is an ordinary
// round-to-nearest FP32 operation): four partial sums of D/4 terms each, so
// the FP32 error bound of a D-term sum covers it.  Padding coordinates are
// zero on both sides; c is a 16-byte-aligned row.
template <int DP>
__device__ __forceinline__ float sqdist_xr(const ulonglong2 (&xr)[DP / 4], const float *__restrict__ c) {
    unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
    for (int q = 0; q < DP / 4; ++q) {
        const ulonglong2 c2 = *reinterpret_cast<const ulonglong2 *>(c + 4 * q);
        unsigned long long d0, d1;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(xr[q].x), "l"(c2.x));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(xr[q].y), "l"(c2.y));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a0) : "l"(d0));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a1) : "l"(d1));
    }
    return hsum2(a0) + hsum2(a1);
}

template <int DP>
__device__ __forceinline__ void load_x(const Params &p, int64_t n, ulonglong2 (&xr)[DP / 4]) {
    const int D = p.D;
    const float *xg = p.X + n * D;
    if (p.x_vec4) {
#pragma unroll
        for (int q = 0; q < DP / 4; ++q)
            xr[q] = 4 * q < D ? __ldg(reinterpret_cast<const ulonglong2 *>(xg) + q) : make_ulonglong2(0ull, 0ull);
    } else {
#pragma unroll
        for (int q = 0; q < DP / 4; ++q) {
            const float x0 = 4 * q + 0 < D ? __ldg(xg + 4 * q + 0) : 0.f;
            const float x1 = 4 * q + 1 < D ? __ldg(xg + 4 * q + 1) : 0.f;
            const float x2 = 4 * q + 2 < D ? __ldg(xg + 4 * q + 2) : 0.f;
            const float x3 = 4 * q + 3 < D ? __ldg(xg + 4 * q + 3) : 0.f;
            xr[q] = make_ulonglong2(pack2(x0, x1), pack2(x2, x3));
        }
    }
}

// Distances with the point read from memory instead of registers (the warp's
// settle below keeps no copy of the row, which keeps the survivor kernel free
// of spills): coordinates are loaded and packed exactly as load_x does, four
// at a time, so sqdist_mem rounds every step as sqdist_xr does on load_x's
// result.  dist2_f64_mem is the FP64 squared distance, coordinates ascending,
// no fused multiply-add (the summation order of the FP64 definition).
template <int DP>
__device__ __forceinline__ ulonglong2 x_quad(const Params &p, const float *xg, int q) {
    const int D = p.D;
    if (p.x_vec4) return 4 * q < D ? __ldg(reinterpret_cast<const ulonglong2 *>(xg) + q) : make_ulonglong2(0ull, 0ull);
    const float x0 = 4 * q + 0 < D ? __ldg(xg + 4 * q + 0) : 0.f;
    const float x1 = 4 * q + 1 < D ? __ldg(xg + 4 * q + 1) : 0.f;
    const float x2 = 4 * q + 2 < D ? __ldg(xg + 4 * q + 2) : 0.f;
    const float x3 = 4 * q + 3 < D ? __ldg(xg + 4 * q + 3) : 0.f;
    return make_ulonglong2(pack2(x0, x1), pack2(x2, x3));
}
template <int DP>
__device__ __forceinline__ float sqdist_mem(const Params &p, const float *xg, const float *__restrict__ c) {
    unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll 4
    for (int q = 0; q < DP / 4; ++q) {
        const ulonglong2 x2 = x_quad<DP>(p, xg, q);
        const ulonglong2 c2 = *reinterpret_cast<const ulonglong2 *>(c + 4 * q);
        unsigned long long d0, d1;
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d0) : "l"(x2.x), "l"(c2.x));
        asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d1) : "l"(x2.y), "l"(c2.y));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a0) : "l"(d0));
        asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(a1) : "l"(d1));
    }
    return hsum2(a0) + hsum2(a1);
}
template <int DP>
__device__ __forceinline__ double dist2_f64_mem(const Params &p, const float *xg, const float *__restrict__ c) {
    const int D = p.D;
    double s = 0.0;
    for (int q = 0; q < DP / 4; ++q) {
        const ulonglong2 x2 = x_quad<DP>(p, xg, q);
        float xv[4];
        unpack2(x2.x, xv[0], xv[1]);
        unpack2(x2.y, xv[2], xv[3]);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (4 * q + j < D) {
                const double t = __dsub_rn((double)xv[j], (double)c[4 * q + j]);
                s = __dadd_rn(s, __dmul_rn(t, t));
            }
        }
    }
    return s;
}

// Rare path, taken by the whole warp for one point: the FP32 results do not
// separate the best (FP32 value s1, index i1) from the runner-up.  The lanes
// take the centroids lane, lane + 32, ...; every centroid whose FP32 distance
// the error bound cannot separate from s1 is settled in FP64, and the warp
// keeps the smallest FP64 distance (lowest index on equal distances).  When
// that winner is not i1, every group bound is rebuilt from FP32 distances,
// one lane per group (the bounds written by the filtered scan assumed i1),
// and *lbg_out receives their minimum.  All lanes return the winner; *s_win
// is its FP32 squared distance.  (One lane alone took about 125 us for this
// at K = 256, D = 64, against about 28 us for a whole batch of 32 points.)
template <int DP>
__device__ __forceinline__ int settle_warp(const Params &p, const float *Cs, const int32_t *gs, int64_t n, float s1,
                                        int i1, float *s_win, float *lbg_out) {
    const int K = p.K, G = p.G, D = p.D;
    const int lane = threadIdx.x & 31;
    const float *xg = p.X + n * D;
    double bd = INFINITY;
    int bi = 0x7fffffff;
    for (int c = lane; c < K; c += 32) {  // ascending: the first of equal distances stays
        const float s = sqdist_mem<DP>(p, xg, Cs + (size_t)c * p.Dp);
        if (!unresolved(s1, s, p)) continue;
        const double d = dist2_f64_mem<DP>(p, xg, Cs + (size_t)c * p.Dp);
        if (d < bd || (d == bd && tie_key(p, c) < tie_key(p, bi))) {
            bd = d;
            bi = c;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double od = __shfl_xor_sync(0xffffffffu, bd, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (od < bd || (od == bd && tie_key(p, oi) < tie_key(p, bi))) {
            bd = od;
            bi = oi;
        }
    }
    // i1 is always among the unresolved centroids (its own distance is s1)
    if (bi == 0x7fffffff || bi == i1) {
        *s_win = s1;
        return i1;
    }
    float lmin = INFINITY;
    float *lbrow = p.lb + n * p.Gp;
    for (int g = lane; g < G; g += 32) {
        float m = INFINITY;
        for (int c = gs[g]; c < gs[g + 1]; ++c) {
            if (c == bi) continue;
            m = fminf(m, dist_dn(sqdist_mem<DP>(p, xg, Cs + (size_t)c * p.Dp), p));
        }
        lbrow[g] = m;
        lmin = fminf(lmin, m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    *s_win = sqdist_mem<DP>(p, xg, Cs + (size_t)bi * p.Dp);
    *lbg_out = lmin;
    return bi;
}

// shared-memory layout (in 4-byte words, each part 16-byte aligned):
// [C, K x Dp, when staged] | Dc[v] (K) | Dg[v] (Gp) | gstart (G + 1) | grp (K)
struct TpLayout {
    size_t dcv, dgv, gs, grp, total;
    __host__ __device__ static size_t up4(size_t x) { return (x + 3) & ~(size_t)3; }
    __host__ __device__ TpLayout(const Params &p, bool stage_c) {
        dcv = stage_c ? (size_t)p.K * p.Dp : 0;
        dgv = up4(dcv + p.K);
        gs = up4(dgv + p.Gp);
        grp = up4(gs + p.G + 1);
        total = grp + p.K;
    }
};

// two blocks per SM up to 64 coordinates; at 128 the point's registers (64
// for x alone) leave room for one
template <int DP, bool STAGE>
__global__ void __launch_bounds__(kTpThreads, DP > 64 ? 1 : 2) k_survivor_tp(Params p, int respect_done) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (*(volatile int *)&ctrl->dense_mode) return;  // this iteration runs the dense pass
    const int count = *(volatile int *)&ctrl->queue_count;
    if ((int64_t)blockIdx.x * kTpThreads >= count) return;  // no work for this block (uniform)
    const int v = ctrl->v;
    const int K = p.K, G = p.G, Gp = p.Gp;

    const TpLayout L(p, STAGE);
    const float *Cs = p.C;
    if constexpr (STAGE) {
        if (!stage_to_smem(smem, p.C, (uint32_t)((size_t)K * p.Dp * 4), &bar, ctrl)) return;
        Cs = smem;
    }
    float *dcv = smem + L.dcv;
    float *dgv = smem + L.dgv;
    int32_t *gs = reinterpret_cast<int32_t *>(smem + L.gs);
    int32_t *sgrp = reinterpret_cast<int32_t *>(smem + L.grp);
    for (int i = threadIdx.x; i < K; i += kTpThreads) sgrp[i] = p.grp[i];
    for (int i = threadIdx.x; i < K; i += kTpThreads) dcv[i] = p.Dc[(size_t)v * K + i];
    for (int i = threadIdx.x; i < Gp; i += kTpThreads) dgv[i] = p.Dg[(size_t)v * Gp + i];
    for (int i = threadIdx.x; i <= G; i += kTpThreads) gs[i] = p.gstart[i];
    __syncthreads();

    unsigned long long c_scanned = 0, c_dist = 0, c_recheck = 0, c_changed = 0;
    const int lane = threadIdx.x & 31;

    // dynamic schedule: each warp claims the next `grab` queue entries from a
    // global counter (points differ a lot in work; a static split leaves
    // SMs idle at the end) and works through them 32 at a time, one per lane
    const int grab = p.surv_grab > 0 ? p.surv_grab : 32;
    int claim = 0, claim_end = 0;
    for (;;) {
        if (claim >= claim_end) {
            int b0 = 0;
            if (lane == 0) b0 = atomicAdd(&ctrl->surv_next, grab);
            claim = __shfl_sync(0xffffffffu, b0, 0);
            claim_end = claim + grab;
        }
        const int base = claim;
        claim += 32;
        if (base >= count) break;
        const int64_t it = (int64_t)base + lane;
        const bool active = it < count;
        bool moved = false;
        int64_t n = 0;
        int a = 0;
        // a point deferred to the warp's settle: its FP32 best, index and global bound
        bool rc = false;
        float rc_s = 0.f, rc_lbg = 0.f;
        int rc_best = 0;
        const unsigned long long c_dist0 = c_dist;  // this lane's count before its point
        if (active) {
            n = p.queue[it];
            if (Gp * 4 * (DP > 64 ? 256 : 512) <= 128 * 1024) {
                // the point's stored bound row into L1 now (it is read after the
                // coordinates, the tightening and the global test): its 128-byte
                // lines (lb is 128-byte aligned).  Only when the rows of all the
                // threads an SM holds (512, or 256 at 128 coordinates) fit in
                // 128 KB of L1; longer rows would evict one another.
                const uintptr_t r0 = reinterpret_cast<uintptr_t>(p.lb + n * Gp);
                const uintptr_t r1 = r0 + (uintptr_t)Gp * 4 - 1;
                for (uintptr_t q = r0 & ~(uintptr_t)127; q <= r1; q += 128)
                    asm volatile("prefetch.global.L1 [%0];" ::"l"(q));
            }
            a = p.label[n];
            const uint32_t st = p.stamp[n];
            const int wl = (int)stamp_l(st);
            const float lbg_e = __fsub_rd(p.lbg[n], drift_m(p, v, wl));
            float *lbrow = p.lb + n * Gp;

            ulonglong2 xr[DP / 4];
            load_x<DP>(p, n, xr);

            // tighten: exact distance to the own centroid, then the global test again
            const float sa = sqdist_xr<DP>(xr, Cs + (size_t)a * p.Dp);
            const float ut = dist_up(sa, p);
            c_dist += 1;
            if (ut <= lbg_e) {
                p.u[n] = ut;
                p.stamp[n] = make_stamp(v, wl);
            } else {
                c_scanned += 1;
                const float da_dn = dist_dn(sa, p);
                const float *dcw = p.Dc + (size_t)wl * K;
                const float *dgw = p.Dg + (size_t)wl * Gp;

                float s_best = sa, s_sec = INFINITY, bd_up = ut;
                int best = a;
                int bg = -1;                      // group holding the running best, once visited
                float bg_val = INFINITY, bg_m1 = INFINITY;  // its bound without / with the best
                float lmin = INFINITY;            // minimum over the other groups' new bounds

                // one group: group filter, then point filter + distances over its
                // centroids; writes the group's new bound
                auto visit_group = [&](const int g) {
                    const float lr = lbrow[g];
                    const float le = wl == v ? lr : __fsub_rd(lr, __fsub_ru(dgv[g], __ldg(dgw + g)));
                    const int c_lo = gs[g], c_hi = gs[g + 1];
                    const bool has_a = a >= c_lo && a < c_hi;
                    float val, val_leave;
                    bool here = false;  // the best is in this group when it is done
                    if (!(le < bd_up)) {
                        // group filter: no centroid of g can beat the running best
                        if (has_a) {
                            val = best == a ? le : fminf(le, da_dn);
                            val_leave = fminf(le, da_dn);
                            here = best == a;
                        } else {
                            val = le;
                            val_leave = le;
                        }
                    } else {
                        // point filter + distance calculator over the group.  Two
                        // pools of lower values: computed squared distances (the two
                        // smallest, with the index of the smallest; the own centroid
                        // enters with its exact value) and point-filter bounds (the
                        // smallest); dist_dn is monotone, so it is applied once at the end.
                        float sm1 = INFINITY, sm2 = INFINITY, pm1 = INFINITY;
                        int sm1i = -1;
                        if (has_a) {
                            sm1 = sa;
                            sm1i = a;
                        }
                        bool best_moved = false;
                        // windows of up to 32 centroids: first the point-filter test of
                        // each (independent loads, no branches), then the distances of
                        // those that pass, in index order
                        for (int w0 = c_lo; w0 < c_hi; w0 += 32) {
                            const int wn = min(32, c_hi - w0);
                            uint32_t pass = 0;
#pragma unroll 4
                            for (int j = 0; j < wn; ++j) {
                                const int c = w0 + j;
                                const float pb = wl == v ? lr : __fsub_rd(lr, __fsub_ru(dcv[c], __ldg(dcw + c)));
                                const bool ok = c != a && pb < bd_up;
                                pass |= ok ? (1u << j) : 0u;
                                pm1 = (c != a && !ok) ? fminf(pm1, pb) : pm1;
                            }
                            while (pass) {
                                const int j = __ffs(pass) - 1;
                                pass &= pass - 1;
                                const int c = w0 + j;
                                const float s = sqdist_xr<DP>(xr, Cs + (size_t)c * p.Dp);
                                c_dist += 1;
                                if (s < s_best || (s == s_best && c < best)) {
                                    s_sec = fminf(s_sec, s_best);
                                    s_best = s;
                                    best = c;
                                    best_moved = true;
                                    bd_up = fminf(bd_up, dist_up(s, p));
                                } else {
                                    s_sec = fminf(s_sec, s);
                                }
                                if (s < sm1) {
                                    sm2 = sm1;
                                    sm1 = s;
                                    sm1i = c;
                                } else {
                                    sm2 = fminf(sm2, s);
                                }
                            }
                        }
                        here = best_moved || (has_a && best == a);
                        val_leave = fminf(pm1, dist_dn(sm1, p));
                        val = (here && sm1i == best) ? fminf(pm1, dist_dn(sm2, p)) : val_leave;
                    }
                    if (here) {
                        if (bg >= 0 && bg != g) {
                            // the best left group bg: its bound takes the value with the old best
                            lbrow[bg] = bg_m1;
                            lmin = fminf(lmin, bg_m1);
                        }
                        bg = g;
                        bg_val = val;
                        bg_m1 = val_leave;
                    } else {
                        lmin = fminf(lmin, val);
                    }
                    lbrow[g] = val;
                };
                const int ga = sgrp[a];
                for (int g0 = 0; g0 < G; g0 += 4) {
                    // four groups at a time: when none of them survives the group
                    // filter and none holds the own centroid, their new bounds are
                    // the drift-adjusted stored ones (one vector load and store)
                    const float4 lr4 = *reinterpret_cast<const float4 *>(lbrow + g0);
                    float4 le4 = lr4;
                    if (wl != v) {
                        const float4 dv4 = *reinterpret_cast<const float4 *>(dgv + g0);
                        const float4 dw4 = __ldg(reinterpret_cast<const float4 *>(dgw + g0));
                        le4.x = __fsub_rd(lr4.x, __fsub_ru(dv4.x, dw4.x));
                        le4.y = __fsub_rd(lr4.y, __fsub_ru(dv4.y, dw4.y));
                        le4.z = __fsub_rd(lr4.z, __fsub_ru(dv4.z, dw4.z));
                        le4.w = __fsub_rd(lr4.w, __fsub_ru(dv4.w, dw4.w));
                    }
                    if (g0 + 1 >= G) le4.y = INFINITY;  // padding groups
                    if (g0 + 2 >= G) le4.z = INFINITY;
                    if (g0 + 3 >= G) le4.w = INFINITY;
                    const bool scan = le4.x < bd_up || le4.y < bd_up || le4.z < bd_up || le4.w < bd_up;
                    if (!scan && (ga < g0 || ga >= g0 + 4)) {
                        lmin = fminf(lmin, fminf(fminf(le4.x, le4.y), fminf(le4.z, le4.w)));
                        *reinterpret_cast<float4 *>(lbrow + g0) = le4;
                    } else {
                        const int g1 = min(g0 + 4, G);
                        for (int g = g0; g < g1; ++g) visit_group(g);
                    }
                }
                float lbg_new = bg >= 0 ? fminf(lmin, bg_val) : lmin;

                if (s_sec != INFINITY && unresolved(s_best, s_sec, p)) {
                    rc = true;  // settled by the warp below
                    rc_s = s_best;
                    rc_best = best;
                    rc_lbg = lbg_new;
                } else {
                    p.lbg[n] = lbg_new;
                    p.u[n] = dist_up(s_best, p);
                    p.label[n] = best;
                    p.stamp[n] = make_stamp(v, v);
                    moved = best != a;
                }
            }
        }
        // the batch's unresolved points, one at a time by the whole warp (its
        // lanes' bound-row stores above are ordered before the rebuild's)
        __syncwarp();
        unsigned rm = __ballot_sync(0xffffffffu, rc);
        while (rm) {
            const int src = __ffs(rm) - 1;
            rm &= rm - 1;
            const int64_t nr = __shfl_sync(0xffffffffu, n, src);
            const float s1 = __shfl_sync(0xffffffffu, rc_s, src);
            const int i1 = __shfl_sync(0xffffffffu, rc_best, src);
            float sw = s1, lg = __shfl_sync(0xffffffffu, rc_lbg, src);
            const int w = settle_warp<DP>(p, Cs, gs, nr, s1, i1, &sw, &lg);
            if (lane == src) {
                rc_best = w;
                rc_s = sw;
                rc_lbg = lg;
            }
        }
        if (rc) {
            p.lbg[n] = rc_lbg;
            p.u[n] = dist_up(rc_s, p);
            p.label[n] = rc_best;
            p.stamp[n] = make_stamp(v, v);
            moved = rc_best != a;
            c_dist = c_dist0 + (unsigned long long)K;  // evaluated against all K: K, not scan + K
            c_recheck += 1;
        }
        // moved points: one atomic per warp for the list slots
        const unsigned mm = __ballot_sync(0xffffffffu, moved);
        if (mm) {
            int base = 0;
            if (lane == 0) base = atomicAdd(&ctrl->moved_count, __popc(mm));
            base = __shfl_sync(0xffffffffu, base, 0);
            if (moved) {
                const int slot = base + __popc(mm & ((1u << lane) - 1u));
                p.moved[slot] = (int32_t)n;
                p.moved_old[slot] = a;
            }
            c_changed += moved ? 1 : 0;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c_scanned += __shfl_xor_sync(0xffffffffu, c_scanned, o);
        c_dist += __shfl_xor_sync(0xffffffffu, c_dist, o);
        c_recheck += __shfl_xor_sync(0xffffffffu, c_recheck, o);
        c_changed += __shfl_xor_sync(0xffffffffu, c_changed, o);
    }
    if (lane == 0) {
        if (c_scanned) atomicAdd(&ctrl->n_scanned, c_scanned);
        if (c_dist) atomicAdd(&ctrl->n_dist, c_dist);
        if (c_recheck) atomicAdd(&ctrl->n_recheck, c_recheck);
        if (c_changed) atomicAdd(&ctrl->n_changed, c_changed);
    }
}

template <int DP, bool STAGE>
cudaError_t launch_tp2(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem) {
    auto kern = k_survivor_tp<DP, STAGE>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTpThreads, smem);
    if (e != cudaSuccess) return e;
    const int64_t blocks = ((int64_t)p.N + kTpThreads - 1) / kTpThreads;
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms * std::max(per_sm, 1)));
    count_launch();
    kern<<<(unsigned)grid, kTpThreads, smem, s>>>(p, respect_done);
    return cudaGetLastError();
}

template <int DP>
cudaError_t launch_tp(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem_limit) {
    // stage the centroids in shared memory when they fit
    const size_t cbytes = (size_t)p.K * p.Dp * 4;
    const bool stage = TpLayout(p, true).total * 4 <= smem_limit && cbytes < (1u << 31);
    const size_t smem = TpLayout(p, stage).total * 4;
    if (smem > smem_limit) return cudaErrorInvalidConfiguration;
    return stage ? launch_tp2<DP, true>(p, s, respect_done, num_sms, smem)
                 : launch_tp2<DP, false>(p, s, respect_done, num_sms, smem);
}

}  // namespace

bool survivor_tp_eligible(const Params &p) {
    const int dp = dense_dp(p.D);
    return dp > 0 && dp <= 128 && p.K < 0x7fffffff;
}

cudaError_t launch_survivor_tp(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem_limit) {
    smem_limit -= 64;  // static shared (mbarrier)
    switch (dense_dp(p.D)) {
    case 4: return launch_tp<4>(p, s, respect_done, num_sms, smem_limit);
    case 8: return launch_tp<8>(p, s, respect_done, num_sms, smem_limit);
    case 16: return launch_tp<16>(p, s, respect_done, num_sms, smem_limit);
    case 32: return launch_tp<32>(p, s, respect_done, num_sms, smem_limit);
    case 64: return launch_tp<64>(p, s, respect_done, num_sms, smem_limit);
    case 128: return launch_tp<128>(p, s, respect_done, num_sms, smem_limit);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace kp
