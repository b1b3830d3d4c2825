// kp_filter.cu -- the filtered assignment of iterations t >= 1.
//
// KPynq (Sec. I) splits the assignment into "Multi-level Filters" (a
// group-level and a point-level filter) and a "Distance Calculator" that
// evaluates only what the filters could not remove.  Here:
//
//   k_filter    all N points, one thread per 4 points, coalesced 16-byte
//               loads of label/u/lbg/stamp: applies the drift since each
//               point's stamp (bound update) and the global test
//               u <= lbg, and counts the points that fail per label bucket;
//   k_filter_scatter  repeats the test and writes the survivors to a work
//               queue grouped by label (a counting sort: shared-memory
//               counts per tile, one global atomic per bucket and tile).
//   k_survivor  one warp per queued point, centroids staged in shared memory
//               by TMA bulk copies: tightens u to the exact distance and
//               retests; then the group-level filter (lanes over groups, one
//               coalesced read of the point's lb row), the point-level filter
//               (lb_g at the stamp minus the centroid's own drift since then)
//               and the distance calculator over the surviving centroids
//               (lanes over centroids); refreshes u, lb, lbg and the label,
//               settles near-ties in FP64, and appends the point to the
//               moved-point list when its label changes.  Used for D > 128;
//               smaller D takes the thread-per-point kernel of
//               kp_survivor_tp.cu.
#include "kp_common.cuh"

namespace kp {

// ---------------------------------------------------------------------------
// global filter + compaction
// ---------------------------------------------------------------------------
constexpr int kFilterThreads = 256;

// The global test of up to four consecutive points: bit j of the result is
// set when point n0 + j fails it (a survivor); a[] receives the labels.
__device__ __forceinline__ unsigned global_test4(const Params &p, int v, int64_t n0, int (&a)[4]) {
    float u[4], lg[4];
    uint32_t st[4];
    if (n0 + 3 < p.N) {
        int4 a4 = *reinterpret_cast<const int4 *>(p.label + n0);
        float4 u4 = *reinterpret_cast<const float4 *>(p.u + n0);
        float4 l4 = *reinterpret_cast<const float4 *>(p.lbg + n0);
        uint4 s4 = *reinterpret_cast<const uint4 *>(p.stamp + n0);
        a[0] = a4.x; a[1] = a4.y; a[2] = a4.z; a[3] = a4.w;
        u[0] = u4.x; u[1] = u4.y; u[2] = u4.z; u[3] = u4.w;
        lg[0] = l4.x; lg[1] = l4.y; lg[2] = l4.z; lg[3] = l4.w;
        st[0] = s4.x; st[1] = s4.y; st[2] = s4.z; st[3] = s4.w;
    } else {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (n0 + j < p.N) {
                a[j] = p.label[n0 + j]; u[j] = p.u[n0 + j];
                lg[j] = p.lbg[n0 + j]; st[j] = p.stamp[n0 + j];
            } else {
                a[j] = 0; u[j] = 0.f; lg[j] = INFINITY; st[j] = make_stamp(v, v);
            }
        }
    }
    unsigned m = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        // bound update after drift, then the global filter
        float ue = __fadd_ru(u[j], drift_c(p, v, (int)stamp_u(st[j]), a[j]));
        float le = __fsub_rd(lg[j], drift_m(p, v, (int)stamp_l(st[j])));
        if (!(ue <= le)) m |= 1u << j;
    }
    return m;
}

// Pass 1 of the compaction: counts the survivors per label bucket (label >>
// bshift) into bcount and their total into queue_count.  The last block to
// finish decides whether this iteration runs the dense pass and, if not,
// turns the counts into the start offsets (bcursor) of each bucket's segment
// of the queue.
__global__ void __launch_bounds__(kFilterThreads) k_filter(Params p, int respect_done) {
    extern __shared__ int hist[];  // nbucket counters
    __shared__ int last;
    __shared__ unsigned long long blk_total;
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    const int v = ctrl->v;
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < p.nbucket; i += kFilterThreads) hist[i] = 0;
    if (threadIdx.x == 0) blk_total = 0;
    __syncthreads();
    const int64_t warp = ((int64_t)blockIdx.x * kFilterThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kFilterThreads) >> 5;
    unsigned long long my_surv = 0;
    // each warp handles 128 consecutive points per step (4 per lane)
    for (int64_t wb = warp * 128; wb < p.N; wb += nwarps * 128) {
        int a[4];
        const unsigned m = global_test4(p, v, wb + lane * 4, a);
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (m & (1u << j)) atomicAdd(&hist[a[j] >> p.bshift], 1);
        my_surv += __popc(m);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) my_surv += __shfl_xor_sync(0xffffffffu, my_surv, o);
    if (lane == 0 && my_surv) atomicAdd(&blk_total, my_surv);
    __syncthreads();
    for (int i = threadIdx.x; i < p.nbucket; i += kFilterThreads)
        if (hist[i]) atomicAdd(&p.bcount[i], hist[i]);
    if (threadIdx.x == 0 && blk_total) {
        atomicAdd(&ctrl->queue_count, (int)blk_total);
        atomicAdd(&ctrl->n_survivors, blk_total);
    }
    // the last block to finish decides dense versus filtered and lays out the queue
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctrl->filter_ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // dense when the survivors exceed dense_frac * N: the survivor kernel's
    // cost grows with the survivors, the dense pass costs the same for any
    // and leaves every bound exact (tight bounds make the next iterations'
    // global filter effective again)
    const int q = *(volatile int *)&ctrl->queue_count;
    const int dense = p.dense_frac < 1.0f && (double)q > (double)p.dense_frac * (double)p.N;
    if (threadIdx.x == 0) {
        ctrl->dense_mode = dense;
        ctrl->filter_ticket = 0;
    }
    if (dense) return;
    // exclusive scan of the bucket counts: each thread sums a contiguous run
    const int per = (p.nbucket + kFilterThreads - 1) / kFilterThreads;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, p.nbucket);
    int run = 0;
    for (int b = b0; b < b1; ++b) run += __ldcg(p.bcount + b);
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    __shared__ int wsum[kFilterThreads / 32];
    if (lane == 31) wsum[threadIdx.x >> 5] = incl;
    __syncthreads();
    int off = incl - run;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) off += wsum[w];
    for (int b = b0; b < b1; ++b) {
        p.bcursor[b] = off;
        off += __ldcg(p.bcount + b);
    }
}

// Pass 2: the same global test again (the inputs are unchanged, so the
// decisions are the same), and each survivor is written to its bucket's
// segment of the queue: per tile of 1024 points a block counts its survivors
// per bucket in shared memory, reserves each bucket's range with one global
// atomic, and places the points.  The queue then holds the survivors grouped
// by label, so that neighbouring threads of the survivor kernel tend to visit
// the same groups and centroids.  Also clears bcount for the next iteration.
__global__ void __launch_bounds__(kFilterThreads) k_filter_scatter(Params p, int respect_done) {
    extern __shared__ int sh[];  // nbucket counters | nbucket bases
    int *cnt = sh;
    int *base = sh + p.nbucket;
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    for (int64_t i = (int64_t)blockIdx.x * kFilterThreads + threadIdx.x; i < p.nbucket;
         i += (int64_t)gridDim.x * kFilterThreads)
        p.bcount[i] = 0;
    if (*(volatile int *)&ctrl->dense_mode) return;
    const int v = ctrl->v;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int kTile = kFilterThreads * 4;
    for (int i = threadIdx.x; i < p.nbucket; i += kFilterThreads) cnt[i] = 0;
    __syncthreads();
    for (int64_t t0 = (int64_t)blockIdx.x * kTile; t0 < p.N; t0 += (int64_t)gridDim.x * kTile) {
        const int64_t n0 = t0 + warp * 128 + lane * 4;
        int a[4];
        const unsigned m = n0 < p.N ? global_test4(p, v, n0, a) : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (m & (1u << j)) atomicAdd(&cnt[a[j] >> p.bshift], 1);
        __syncthreads();
        for (int i = threadIdx.x; i < p.nbucket; i += kFilterThreads) {
            const int c = cnt[i];
            base[i] = c ? atomicAdd(&p.bcursor[i], c) : 0;
            cnt[i] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (m & (1u << j)) {
                const int b = a[j] >> p.bshift;
                p.queue[base[b] + atomicAdd(&cnt[b], 1)] = (int32_t)(n0 + j);
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < p.nbucket; i += kFilterThreads) cnt[i] = 0;
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// survivor kernel
// ---------------------------------------------------------------------------
// Per-warp shared scratch (floats / ints), sizes in 4-byte words:
//   xs   [DPa]   the point
//   sq   [K]     FP32 squared distance of each evaluated centroid, -1 if the
//                point filter skipped it
//   lbr  [Gp]    stored group bounds of the point
//   lbe  [Gp]    drift-adjusted group bounds
//   sg   [Gp]    surviving groups, compacted
//   off  [Gp+1]  prefix sums of their sizes
struct WarpScratch {
    int DPa, K, Gp;
    // rounded to 4 words so that every warp's xs stays 16-byte aligned
    __host__ __device__ int words() const { return (DPa + K + 4 * Gp + 1 + 3) & ~3; }
};

template <int DP>
__device__ __forceinline__ float sqdist_lane(const float *__restrict__ xs, const float *__restrict__ c, int D) {
    if constexpr (DP > 0) {
        // packed FP32x2 subtract / fused multiply-add (each half an ordinary
        // round-to-nearest FP32 operation): half the instructions of the
        // scalar form; four partial sums of DP/4 terms
        unsigned long long a0 = 0ull, a1 = 0ull;
#pragma unroll
        for (int i = 0; i < DP; i += 4) {
            const ulonglong2 x2 = *reinterpret_cast<const ulonglong2 *>(xs + i);
            const ulonglong2 c2 = *reinterpret_cast<const ulonglong2 *>(c + i);
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
    } else {
        float a0 = 0.f, a1 = 0.f;
        int i = 0;
        for (; i + 1 < D; i += 2) {
            float t0 = xs[i] - c[i], t1 = xs[i + 1] - c[i + 1];
            a0 = fmaf(t0, t0, a0);
            a1 = fmaf(t1, t1, a1);
        }
        if (i < D) {
            float t0 = xs[i] - c[i];
            a0 = fmaf(t0, t0, a0);
        }
        return a0 + a1;
    }
}

// point-filter bound of centroid c (group g) for a point stamped at version w
__device__ __forceinline__ float point_bound(const Params &p, float lb_stored, int v, int w, int c) {
    return __fsub_rd(lb_stored, drift_c(p, v, w, c));
}

template <int DP, bool STAGE>
__global__ void __launch_bounds__(512, 2) k_survivor(Params p, int respect_done, int warps_per_block) {
    extern __shared__ __align__(128) float smem[];
    __shared__ __align__(8) uint64_t bar;
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (*(volatile int *)&ctrl->dense_mode) return;  // this iteration runs the dense pass
    const int count = *(volatile int *)&ctrl->queue_count;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * warps_per_block + warp;
    const int nwarps = gridDim.x * warps_per_block;
    if (blockIdx.x * warps_per_block >= count) return;  // no work for this block (uniform)
    const int v = ctrl->v;
    const int K = p.K, G = p.G, D = p.D;
    const int DPa = DP > 0 ? DP : ((D + 3) & ~3);

    const float *Cs = p.C;
    float *scratch = smem;
    if constexpr (STAGE) {
        const uint32_t cbytes = (uint32_t)((size_t)K * p.Dp * 4);
        if (!stage_to_smem(smem, p.C, cbytes, &bar, ctrl)) return;
        Cs = smem;
        scratch = smem + (size_t)K * p.Dp;
    }
    WarpScratch ws{DPa, K, p.Gp};
    float *xs = scratch + (size_t)warp * ws.words();
    float *sq = xs + DPa;
    float *lbr = sq + K;
    float *lbe = lbr + p.Gp;
    int *sg = reinterpret_cast<int *>(lbe + p.Gp);
    int *off = sg + p.Gp;

    unsigned long long c_scanned = 0, c_dist = 0, c_recheck = 0, c_changed = 0, c_dist_lane = 0;

    // The next point's id, label, stamp, global bound, coordinates and (up
    // to 128 groups) bound row are loaded while the current one is processed:
    // each point's loads otherwise form a chain of dependent global reads.
    constexpr int XPL = DP > 0 ? (DP + 31) / 32 : 1;  // coordinates per lane
    constexpr int LPL = 4;                           // bound-row entries per lane
    const bool pf_lb = DP > 0 && G <= 32 * LPL;
    int64_t pn = 0;
    int pa = 0;
    uint32_t pst = 0;
    float plbg = 0.f, px[XPL], plb[LPL];
    auto prefetch = [&](int idx) {
        if (idx >= count) return;  // warp-uniform
        pn = p.queue[idx];
        pa = p.label[pn];
        pst = p.stamp[pn];
        plbg = p.lbg[pn];
        if constexpr (DP > 0) {
#pragma unroll
            for (int k = 0; k < XPL; ++k) {
                const int i = lane + 32 * k;
                px[k] = i < D ? __ldg(p.X + pn * D + i) : 0.f;
            }
        }
        if (pf_lb) {
#pragma unroll
            for (int k = 0; k < LPL; ++k) {
                const int g = lane + 32 * k;
                plb[k] = g < G ? p.lb[pn * p.Gp + g] : 0.f;
            }
        }
    };
    prefetch(gwarp);

    for (int it = gwarp; it < count; it += nwarps) {
        const int64_t n = pn;
        const int a = pa;
        const uint32_t st = pst;
        const int wu = (int)stamp_u(st), wl = (int)stamp_l(st);
        const float lbg_e = __fsub_rd(plbg, drift_m(p, v, wl));
        float clb[LPL];
#pragma unroll
        for (int k = 0; k < LPL; ++k) clb[k] = plb[k];

        // the point
        if constexpr (DP > 0) {
#pragma unroll
            for (int k = 0; k < XPL; ++k)
                if (lane + 32 * k < DPa) xs[lane + 32 * k] = px[k];
        } else {
            const float *xg = p.X + n * D;
            for (int i = lane; i < DPa; i += 32) xs[i] = i < D ? __ldg(xg + i) : 0.f;
        }
        __syncwarp();
        prefetch(it + nwarps);

        // tighten: exact distance to the own centroid (lanes split the
        // coordinates; any summation order is covered by the error bound)
        const float *ca = Cs + (size_t)a * p.Dp;
        float part = 0.f;
        for (int i = lane; i < D; i += 32) {
            float t = xs[i] - ca[i];
            part = fmaf(t, t, part);
        }
        const float sa = warp_sum(part);
        const float ut = dist_up(sa, p);
        c_dist += 1;
        if (ut <= lbg_e) {  // the global filter holds after tightening
            if (lane == 0) {
                p.u[n] = ut;
                p.stamp[n] = make_stamp(v, wl);
            }
            __syncwarp();
            continue;
        }
        c_scanned += 1;

        // group-level filter: lanes over groups, surviving groups compacted
        int nsg = 0, total = 0;
        for (int g0 = 0; g0 < G; g0 += 32) {
            const int g = g0 + lane;
            bool surv = false;
            int size = 0;
            if (g < G) {
                float lr;
                if (pf_lb) {  // prefetched: entry g0 / 32 of this lane
                    lr = clb[0];
#pragma unroll
                    for (int k = 1; k < LPL; ++k)
                        if ((g0 >> 5) == k) lr = clb[k];
                } else {
                    lr = p.lb[n * p.Gp + g];
                }
                float le = __fsub_rd(lr, drift_g(p, v, wl, g));
                lbr[g] = lr;
                lbe[g] = le;
                surv = le < ut;
                size = surv ? p.gstart[g + 1] - p.gstart[g] : 0;
            }
            unsigned bal = __ballot_sync(0xffffffffu, surv);
            int incl = size;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (surv) {
                int r = nsg + __popc(bal & ((1u << lane) - 1u));
                sg[r] = g;
                off[r] = total + incl - size;
            }
            nsg += __popc(bal);
            total += __shfl_sync(0xffffffffu, incl, 31);
        }
        if (lane == 0) off[nsg] = total;
        if (lane == 0) sq[a] = sa;
        __syncwarp();

        // point-level filter + distance calculator over the surviving
        // centroids, 32 at a time; running best decides the point filter
        float s_best = sa, s_sec = INFINITY;
        int best = a;
        float bd_up = ut;
        for (int b0 = 0; b0 < total; b0 += 32) {
            const int q = b0 + lane;
            float s = INFINITY;
            int c = 0x7fffffff;
            if (q < total) {
                int lo = 0, hi = nsg - 1;  // last j with off[j] <= q
                while (lo < hi) {
                    int mid = (lo + hi + 1) >> 1;
                    if (off[mid] <= q) lo = mid; else hi = mid - 1;
                }
                const int g = sg[lo];
                c = p.gstart[g] + (q - off[lo]);
                if (c != a) {
                    float bnd = point_bound(p, lbr[g], v, wl, c);
                    if (bnd >= bd_up) {
                        sq[c] = -1.f;  // point filter: cannot beat the best
                    } else {
                        s = sqdist_lane<DP>(xs, Cs + (size_t)c * p.Dp, D);
                        sq[c] = s;
                        c_dist_lane += 1;
                    }
                }
                if (c == a) c = 0x7fffffff;
            }
            // batch minimum and second minimum, then merge
            float s1 = s;
            int i1 = c;
            warp_argmin(s1, i1);
            float s2 = (c == i1) ? INFINITY : s;
            s2 = warp_min(s2);
            if (s1 < s_best || (s1 == s_best && i1 < best)) {
                s_sec = fminf(fminf(s_best, s2), s_sec);
                s_best = s1;
                best = i1;
            } else {
                s_sec = fminf(s_sec, s1);
            }
            bd_up = fminf(bd_up, dist_up(s_best, p));
        }
        __syncwarp();

        // near-tie: settle in FP64 among all evaluated centroids that the
        // FP32 error bound cannot separate from the FP32 best
        if (s_sec != INFINITY && unresolved(s_best, s_sec, p)) {
            double bd64 = INFINITY;
            int bi = 0x7fffffff;
            for (int b0 = 0; b0 <= total; b0 += 32) {
                const int q = b0 + lane;
                int c = -1;
                if (q < total) {
                    int lo = 0, hi = nsg - 1;
                    while (lo < hi) {
                        int mid = (lo + hi + 1) >> 1;
                        if (off[mid] <= q) lo = mid; else hi = mid - 1;
                    }
                    c = p.gstart[sg[lo]] + (q - off[lo]);
                } else if (q == total) {
                    c = a;  // the own centroid may be outside the surviving groups
                }
                if (c >= 0 && (q == total || c != a)) {
                    float s = sq[c];
                    if (s >= 0.f && unresolved(s_best, s, p)) {
                        double d64 = dist2_f64(xs, Cs + (size_t)c * p.Dp, D);
                        if (d64 < bd64 || (d64 == bd64 && tie_key(p, c) < tie_key(p, bi))) { bd64 = d64; bi = c; }
                    }
                }
            }
            warp_argmin_d_key(bd64, bi, p);
            best = bi;
            s_best = sq[bi];
            c_recheck += 1;
        }

        // bound refresh: lanes over groups
        const int ga = p.grp[a];
        const float da_dn = dist_dn(sa, p);
        float gmin = INFINITY;
        for (int g0 = 0; g0 < G; g0 += 32) {
            const int g = g0 + lane;
            if (g < G) {
                const bool surv = lbe[g] < ut;
                float m;
                if (surv) {
                    m = INFINITY;
                    for (int c = p.gstart[g]; c < p.gstart[g + 1]; ++c) {
                        if (c == best) continue;
                        float s = sq[c];
                        float val = s >= 0.f ? dist_dn(s, p) : point_bound(p, lbr[g], v, wl, c);
                        m = fminf(m, val);
                    }
                } else {
                    m = lbe[g];
                    if (g == ga && best != a) m = fminf(m, da_dn);
                }
                p.lb[n * p.Gp + g] = m;
                gmin = fminf(gmin, m);
            }
        }
        gmin = warp_min(gmin);
        if (lane == 0) {
            p.lbg[n] = gmin;
            p.u[n] = dist_up(s_best, p);
            p.label[n] = best;
            p.stamp[n] = make_stamp(v, v);
        }
        if (best != a) {
            // the moves kernel moves x between the cluster sums afterwards
            if (lane == 0) {
                const int slot = atomicAdd(&ctrl->moved_count, 1);
                p.moved[slot] = (int32_t)n;
                p.moved_old[slot] = a;
            }
            c_changed += 1;
        }
        __syncwarp();
    }
    // c_dist counts per lane (the lanes split the candidates); the other
    // counters are per point and identical in every lane
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c_dist_lane += __shfl_xor_sync(0xffffffffu, c_dist_lane, o);
    c_dist += c_dist_lane;
    if (lane == 0) {
        if (c_scanned) atomicAdd(&ctrl->n_scanned, c_scanned);
        if (c_dist) atomicAdd(&ctrl->n_dist, c_dist);
        if (c_recheck) atomicAdd(&ctrl->n_recheck, c_recheck);
        if (c_changed) atomicAdd(&ctrl->n_changed, c_changed);
    }
}

cudaError_t launch_filter(const Params &p, cudaStream_t s, int respect_done, int num_sms) {
    // two blocks per SM: each block adds its bucket counts to the global ones
    // (and reserves queue ranges), so fewer blocks mean fewer contended atomics
    int64_t warps = (p.N + 127) / 128;
    int64_t grid = std::min<int64_t>((warps + 7) / 8, (int64_t)num_sms * 2);
    grid = std::max<int64_t>(grid, 1);
    const size_t smem1 = (size_t)p.nbucket * 4, smem2 = 2 * smem1;
    cudaError_t e = cudaFuncSetAttribute(k_filter_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
    if (e != cudaSuccess) return e;
    count_launch();
    k_filter<<<(unsigned)grid, kFilterThreads, smem1, s>>>(p, respect_done);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    count_launch();
    k_filter_scatter<<<(unsigned)grid, kFilterThreads, smem2, s>>>(p, respect_done);
    return cudaGetLastError();
}

template <int DP, bool STAGE>
static cudaError_t launch_surv_t(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem_limit) {
    const int DPa = DP > 0 ? DP : ((p.D + 3) & ~3);
    WarpScratch ws{DPa, p.K, p.Gp};
    size_t per_warp = (size_t)ws.words() * 4;
    size_t cbytes = STAGE ? (size_t)p.K * p.Dp * 4 : 0;
    int wpb = 16;
    while (wpb > 1 && cbytes + per_warp * wpb > smem_limit) wpb >>= 1;
    size_t smem = cbytes + per_warp * wpb;
    if (smem > smem_limit) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_survivor<DP, STAGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_survivor<DP, STAGE>, wpb * 32, smem);
    if (e != cudaSuccess) return e;
    int grid = num_sms * std::max(per_sm, 1);
    count_launch();
    k_survivor<DP, STAGE><<<grid, wpb * 32, smem, s>>>(p, respect_done, wpb);
    return cudaGetLastError();
}

template <int DP>
static cudaError_t launch_surv_dp(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem_limit) {
    const int DPa = DP > 0 ? DP : ((p.D + 3) & ~3);
    WarpScratch ws{DPa, p.K, p.Gp};
    size_t per_warp = (size_t)ws.words() * 4;
    size_t cbytes = (size_t)p.K * p.Dp * 4;
    // stage the centroids when they fit next to at least 4 warps of scratch
    if (cbytes + 4 * per_warp <= smem_limit && cbytes < (1u << 31))
        return launch_surv_t<DP, true>(p, s, respect_done, num_sms, smem_limit);
    return launch_surv_t<DP, false>(p, s, respect_done, num_sms, smem_limit);
}

cudaError_t launch_survivor(const Params &p, cudaStream_t s, int respect_done, int num_sms, size_t smem_limit) {
    if (survivor_tp_eligible(p)) return launch_survivor_tp(p, s, respect_done, num_sms, smem_limit);
    smem_limit -= 64;  // static shared (mbarrier)
    switch (dense_dp(p.D)) {
    case 4: return launch_surv_dp<4>(p, s, respect_done, num_sms, smem_limit);
    case 8: return launch_surv_dp<8>(p, s, respect_done, num_sms, smem_limit);
    case 16: return launch_surv_dp<16>(p, s, respect_done, num_sms, smem_limit);
    case 32: return launch_surv_dp<32>(p, s, respect_done, num_sms, smem_limit);
    case 64: return launch_surv_dp<64>(p, s, respect_done, num_sms, smem_limit);
    case 128: return launch_surv_dp<128>(p, s, respect_done, num_sms, smem_limit);
    default: return launch_surv_dp<0>(p, s, respect_done, num_sms, smem_limit);
    }
}

}  // namespace kp
