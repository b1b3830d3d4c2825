// kp_dense_tcb.cu -- dense assignment on the tensor cores when the centroids
// do not fit one accumulator (K > 256).
//
// The same contraction as kp_dense_tc.cu (Sec. I: the distance calculator on
// the pairs the filters leave, here all of them): t_k = ||c_k||^2 - 2 x.c_k
// from BF16x3 tcgen05.mma, exact decisions through the settle queue.  The
// centroids stream through shared memory in blocks of 128 (both bfloat16
// halves, loaded by TMA from a split copy made at the start of each pass),
// and each row's scan -- group minima, winner, runner-up -- carries across
// the blocks.  Group minima are converted to lower bounds and written to lb
// after every 64 columns, so shared memory holds only the groups those
// columns close.
//
// Persistent CTA per SM, 320 threads: warp 0 issues TMA, one thread of warp 1
// the MMAs, warps 2..9 are two epilogue groups of four.  Tiles of 128 points
// go in pairs to the two groups; both tiles of a pair use each centroid block
// while it is in shared memory.  Each group owns two TMEM buffers of 128
// columns, so the MMAs of block j+1 run while the group scans block j.
#include "kp_tc.cuh"

namespace kp {
namespace {

constexpr int kNB = 128;                       // centroids per block (MMA N)
constexpr int kBAtom = kNB * 128;              // one 64-element column block of a centroid block
constexpr int kEpiWarps = 4;
constexpr int kPairs = 2;                      // epilogue groups = tiles in flight
constexpr int kThreads = 64 + kPairs * kEpiWarps * 32;
constexpr int kMaxKp = 4096;

struct TcbCfg {
    int Kp;          // K padded to a multiple of kNB
    int nb;          // centroid blocks
    int bst;         // centroid-block stages (1 or 2)
    int srow;        // staging floats per row (odd, >= groups 64 columns can close + 1)
    uint32_t off_A, off_B, off_cn, off_bm, off_stage, off_bar;
    int num_tiles;
    float e_lin, e_c2, xn_lo, xn_hi;
};

// uses of accumulator buffer `buf` (blocks j with j % 2 == buf) before block j of pair pr
__device__ __forceinline__ uint32_t acc_uses(int pr, int j, int buf, int nb) {
    return (uint32_t)(pr * ((nb + 1 - buf) >> 1) + (j >> 1));
}

template <int D>
__global__ void __launch_bounds__(kThreads, 1)
    k_dense_tcb(const __grid_constant__ CUtensorMap tmh, const __grid_constant__ CUtensorMap tml,
                const __grid_constant__ CUtensorMap tmch, const __grid_constant__ CUtensorMap tmcl, Params p,
                TcbCfg cfg, int first, int respect_done, int if_dense) {
    extern __shared__ uint8_t raw[];
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (if_dense && !*(volatile int *)&ctrl->dense_mode) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->path = KM_PATH_DENSE_TC;
    constexpr int NA = D / 64;
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    const int Kp = cfg.Kp, nb = cfg.nb, BS = cfg.bst;
    uint8_t *sA = sm + cfg.off_A;  // 2 stages: [NA atoms x_h][NA atoms x_l]
    uint8_t *sB = sm + cfg.off_B;  // BS stages: [NA atoms c_h][NA atoms c_l]
    float *cn = reinterpret_cast<float *>(sm + cfg.off_cn);  // [Kp] ||c||^2 (+inf: padding)
    float *pen = cn + Kp;                                    // [Kp] +inf where a group opens
    uint32_t *bm = reinterpret_cast<uint32_t *>(sm + cfg.off_bm);  // [Kp / 32] group-start masks
    float *stage = reinterpret_cast<float *>(sm + cfg.off_stage);  // [8 warps x 32 rows][srow]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + cfg.off_bar);
    uint64_t *full_a = bars;                 // [2]
    uint64_t *empty_a = bars + 2;            // [2]
    uint64_t *full_b = bars + 4;             // [BS]
    uint64_t *empty_b = bars + 4 + BS;       // [BS]
    uint64_t *acc_full = bars + 4 + 2 * BS;  // [2 groups][2 buffers]
    uint64_t *acc_empty = acc_full + 4;      // [2][2]
    uint64_t *mma_done = acc_empty + 4;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mma_done + 1);
    float *c2max_s = reinterpret_cast<float *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = ctrl->v;
    const int K = p.K, G = p.G;
    // this CTA's tiles: blockIdx.x + i * gridDim.x; pairs (2pr, 2pr + 1)
    const int ntile = cfg.num_tiles > (int)blockIdx.x
                          ? (cfg.num_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                          : 0;
    const int npair = (ntile + 1) >> 1;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            bar_init(&full_a[i], 1);
            bar_init(&empty_a[i], 1 + kEpiWarps);  // the MMAs' commit and the norm reads
        }
        for (int i = 0; i < BS; ++i) {
            bar_init(&full_b[i], 1);
            bar_init(&empty_b[i], 1);
        }
        for (int i = 0; i < 4; ++i) {
            bar_init(&acc_full[i], 1);
            bar_init(&acc_empty[i], kEpiWarps);
        }
        bar_init(mma_done, 1);
        *c2max_s = 0.f;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    // norms (from the pass's split copy), penalties, group-start masks
    for (int c = threadIdx.x; c < Kp / 32; c += blockDim.x) bm[c] = 0u;
    {
        float cm = 0.f;
        for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
            const float s2 = k < K ? p.cnorm[k] : INFINITY;
            if (k < K) cm = fmaxf(cm, s2);
            cn[k] = s2;
            pen[k] = 0.f;
        }
        cm = warp_max(cm);
        __syncthreads();  // c2max_s, the masks and the penalties initialised
        if (lane == 0 && cm > 0.f) atomicMax(reinterpret_cast<int *>(c2max_s), __float_as_int(cm));
        for (int g = 1 + threadIdx.x; g < G; g += blockDim.x) {
            const int col = p.gstart[g];
            if ((unsigned)col < (unsigned)Kp) {
                atomicOr(&bm[col >> 5], 1u << (col & 31));
                pen[col] = INFINITY;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmh) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tml) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmch) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmcl) : "memory");
            bool ok = true;
            int nbl = 0;           // centroid blocks issued
            int ia[2] = {0, 0};    // tiles issued into each A stage
            for (int pr = 0; pr < npair && ok; ++pr) {
                for (int g = 0; g < 2 && ok; ++g) {
                    const int i = 2 * pr + g;
                    if (i >= ntile) break;
                    if (pr > 0 && !(ok = bar_wait(&empty_a[g], (pr - 1) & 1, ctrl))) break;
                    ++ia[g];
                    const int tile = (int)blockIdx.x + i * (int)gridDim.x;
                    uint8_t *st = sA + (size_t)g * 2 * NA * kAtomBytes;
                    mbar_arrive_expect_tx(&full_a[g], (uint32_t)(2 * NA * kAtomBytes));
                    for (int a = 0; a < NA; ++a) {
                        tma_2d(st + a * kAtomBytes, &tmh, 64 * a, tile * kTM, &full_a[g]);
                        tma_2d(st + (NA + a) * kAtomBytes, &tml, 64 * a, tile * kTM, &full_a[g]);
                    }
                }
                for (int j = 0; j < nb && ok; ++j) {
                    const int bs = nbl % BS, fb = nbl / BS;
                    if (fb > 0 && !(ok = bar_wait(&empty_b[bs], (fb - 1) & 1, ctrl))) break;
                    ++nbl;
                    uint8_t *sb = sB + (size_t)bs * 2 * NA * kBAtom;
                    mbar_arrive_expect_tx(&full_b[bs], (uint32_t)(2 * NA * kBAtom));
                    for (int a = 0; a < NA; ++a) {
                        tma_2d(sb + a * kBAtom, &tmch, 64 * a, j * kNB, &full_b[bs]);
                        tma_2d(sb + (NA + a) * kBAtom, &tmcl, 64 * a, j * kNB, &full_b[bs]);
                    }
                }
            }
            // drain: the last loads of each barrier have landed before the block exits
            for (int g = 0; g < 2; ++g)
                if (ia[g] > 0) bar_wait(&full_a[g], (ia[g] - 1) & 1, ctrl);
            for (int b = 0; b < BS; ++b) {
                const int uses = nbl > b ? (nbl - b + BS - 1) / BS : 0;
                if (uses > 0) bar_wait(&full_b[b], (uses - 1) & 1, ctrl);
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            // kind::f16: F32 accumulate, BF16 A and B, K-major, N = 128, M = 128
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNB >> 3) << 17) |
                                   ((uint32_t)(kTM >> 4) << 24);
            bool ok = true;
            int nbl = 0;
            for (int pr = 0; pr < npair && ok; ++pr) {
                const int ng = 2 * pr + 1 < ntile ? 2 : 1;
                for (int g = 0; g < ng && ok; ++g) ok = bar_wait(&full_a[g], pr & 1, ctrl);
                if (!ok) break;
                tc_fence_after();
                for (int j = 0; j < nb && ok; ++j, ++nbl) {
                    const int bs = nbl % BS, fb = nbl / BS;
                    if (!(ok = bar_wait(&full_b[bs], fb & 1, ctrl))) break;
                    tc_fence_after();
                    const uint8_t *sb = sB + (size_t)bs * 2 * NA * kBAtom;
                    const int buf = j & 1;
                    for (int g = 0; g < ng; ++g) {
                        const uint32_t uses = acc_uses(pr, j, buf, nb);
                        if (uses > 0 && !(ok = bar_wait(&acc_empty[g * 2 + buf], (uses - 1) & 1, ctrl))) break;
                        tc_fence_after();
                        const uint32_t d_tmem = tmem + (uint32_t)(g * 2 * kNB + buf * kNB);
                        const uint8_t *st = sA + (size_t)g * 2 * NA * kAtomBytes;
#pragma unroll
                        for (int ks = 0; ks < D / 16; ++ks) {
                            const int a = ks >> 2, jj = ks & 3;
                            const uint64_t dah = desc_sw128(smem_u32(st + a * kAtomBytes + jj * 32));
                            const uint64_t dal = desc_sw128(smem_u32(st + (NA + a) * kAtomBytes + jj * 32));
                            const uint64_t dbh = desc_sw128(smem_u32(sb + a * kBAtom + jj * 32));
                            const uint64_t dbl = desc_sw128(smem_u32(sb + (NA + a) * kBAtom + jj * 32));
                            const uint32_t acc = ks > 0;
                            asm volatile(
                                "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.eq.b32 q, %4, %4;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %5, %3, q;\n\t"
                                "tcgen05.mma.cta_group::1.kind::f16 [%0], %6, %2, %3, q;\n\t}" ::"r"(d_tmem),
                                "l"(dah), "l"(dbh), "r"(idesc), "r"(acc), "l"(dbl), "l"(dal)
                                : "memory");
                        }
                        asm volatile(
                            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                smem_u32(&acc_full[g * 2 + buf]))
                            : "memory");
                    }
                    if (!ok) break;
                    // the block's stage is free once these MMAs have read it
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty_b[bs]))
                                 : "memory");
                }
                if (!ok) break;
                for (int g = 0; g < ng; ++g)
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                     smem_u32(&empty_a[g]))
                                 : "memory");
            }
            // every MMA of this thread is complete before TMEM is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(mma_done))
                         : "memory");
            bar_wait(mma_done, 0, ctrl);
        }
    } else {
        // ------------------------------------------------------- epilogue
        const int g = (warp - 2) / kEpiWarps;  // epilogue group = tile of the pair
        const int q = warp & 3;                // TMEM lane quadrant of this warp
        const int r = q * 32 + lane;
        const float c2max = __fmul_ru(*c2max_s, 1.0f + 1.0f / 1024);
        const float cmax = sqrt_hi(c2max);
        const float ec2 = __fmul_ru(cfg.e_c2, c2max);
        // the filtered method keeps every bound; plain Lloyd keeps only the
        // group bounds, for the exact settle's candidate groups
        const bool bounds = p.algo == KM_ALGO_FILTERED;
        const bool has_lb = p.lb != nullptr;
        const int wrow = (warp - 2) * 32;      // this warp's rows in the staging area
        float *row = stage + (size_t)(wrow + lane) * cfg.srow;
        const uint32_t row_addr = smem_u32(row);
        unsigned long long c_changed = 0, c_dist = 0;
        for (int pr = 0; pr < npair; ++pr) {
            const int i = 2 * pr + g;
            if (i >= ntile) break;
            const int tile = (int)blockIdx.x + i * (int)gridDim.x;
            if (!__all_sync(0xffffffffu, bar_wait(&full_a[g], pr & 1, ctrl))) break;
            const uint8_t *st = sA + (size_t)g * 2 * NA * kAtomBytes;
            const int64_t n = (int64_t)tile * kTM + r;
            const bool valid = n < p.N;
            const int old = valid ? (first ? -1 : p.label[n]) : -1;
            const float xn = valid ? p.xnorm[n] : 0.f;
            __syncwarp();
            if (lane == 0) bar_arrive(&empty_a[g]);
            const float xlo = __fmul_rd(xn, cfg.xn_lo), xup = __fmul_ru(xn, cfg.xn_hi);
            const float R = __fadd_ru(sqrt_hi(xup), cmax);  // bounds ||x - mu|| + ||c - mu||
            const float E = __fmaf_ru(p.e_cen, __fmul_ru(R, R), __fmaf_ru(cfg.e_lin, __fmul_ru(sqrt_hi(xup), cmax), ec2));
            const float twoE = __fmul_ru(2.f, E);
            const int64_t n0 = (int64_t)tile * kTM + q * 32;
            const int rows = (int)max((int64_t)0, min((int64_t)32, p.N - n0));

            // converts this thread's staged minima [0, cnt) in place, then the
            // warp writes them to lb as groups gfirst.. of its 32 rows
            int gfirst = 0;
            auto flush = [&](int cnt) {
                for (int s = 0; s < cnt; ++s) {
                    const float tg = row[s];
                    row[s] = tg == INFINITY ? INFINITY : sqrt_lo(__fsub_rd(__fadd_rd(xlo, tg), E));
                }
                __syncwarp();
                const float *st0 = stage + (size_t)wrow * cfg.srow;
                for (int e = lane; e < rows * cnt; e += 32) {
                    const int rw = e / cnt, s = e - rw * cnt;
                    if (has_lb && gfirst + s < G) p.lb[(n0 + rw) * p.Gp + gfirst + s] = st0[rw * cfg.srow + s];
                }
                __syncwarp();
                gfirst += cnt;
            };

            RowScan sc;
            sc.init(row);
            for (int j = 0; j < nb; ++j) {
                const int buf = j & 1;
                const uint32_t uses = acc_uses(pr, j, buf, nb);
                if (!__all_sync(0xffffffffu, bar_wait(&acc_full[g * 2 + buf], uses & 1, ctrl))) {
                    gfirst = -1;
                    break;
                }
                tc_fence_after();
                const uint32_t tb = tmem + (uint32_t)(g * 2 * kNB + buf * kNB) + ((uint32_t)(q * 32) << 16);
                {
                    uint32_t ra[32], rb[32];
                    tmem_ld32_async(tb, ra);
#pragma unroll 1
                    for (int c0 = 0; c0 < kNB; c0 += 64) {
                        tmem_wait32(ra);
                        tmem_ld32_async(tb + c0 + 32, rb);
                        scan_one(sc, ra, j * kNB + c0, cn, pen);
                        tmem_wait32(rb);
                        if (c0 + 64 < kNB) {
                            tmem_ld32_async(tb + c0 + 64, ra);
                        } else {  // the accumulators are read: release them
                            tc_fence_before();
                            __syncwarp();
                            if (lane == 0) bar_arrive(&acc_empty[g * 2 + buf]);
                        }
                        scan_one(sc, rb, j * kNB + c0 + 32, cn, pen);
                        // groups closed in these 64 columns: slots [0, (rp - row) / 4)
                        flush((int)((sc.rp - row_addr) >> 2));
                        sc.rp = row_addr;
                    }
                }
            }
            if (gfirst < 0) break;  // a wait timed out (error recorded)
            sc.close();
            flush(1);  // the last group
            float b1, b2;
            int i1;
            sc.result(b1, i1, b2);
            const float thr = __fadd_ru(b1, twoE);
            const bool need = valid && b2 <= thr;
            const unsigned nm = __ballot_sync(0xffffffffu, need);
            if (need) {
                // candidates of the exact settle: the groups whose bound does not
                // exceed the bound of the window's edge (lb is written by now)
                SettleReq rq;
                rq.n = (int32_t)n;
                rq.old = old;
                rq.i1 = i1;
                rq.lb_alt = sqrt_lo(__fsub_rd(__fadd_rd(xlo, b1), E));
                rq.gmask = 0ull;
                rq.lim = sqrt_hi(__fsub_ru(__fadd_ru(xup, thr), E));
                p.sreq[n] = rq;
            }
            if (lane == 0) p.sbits[(int64_t)tile * (kTM / 32) + q] = nm;
            const int best = i1;
            if (valid) {
                c_dist += (unsigned long long)K;
                if (!need) p.label[n] = best;
                // the winner's group excludes the winner: every other column is
                // at least the runner-up; the smallest group bound is that bound
                const float lw = b2 == INFINITY ? INFINITY : sqrt_lo(__fsub_rd(__fadd_rd(xlo, b2), E));
                if (has_lb) p.lb[n * p.Gp + group_of(bm, best)] = lw;
                if (bounds) {
                    p.lbg[n] = lw;
                    p.u[n] = sqrt_hi(__fadd_ru(__fadd_ru(xup, b1), E));
                    p.stamp[n] = make_stamp(v, v);
                }
            }
            {
                const bool moved = valid && !need && old != best;
                const unsigned mm = __ballot_sync(0xffffffffu, moved);
                c_changed += moved ? 1 : 0;
                if (mm && !first) {
                    int base = 0;
                    if (lane == 0) base = atomicAdd(&ctrl->moved_count, __popc(mm));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (moved) {
                        const int slot = base + __popc(mm & ((1u << lane) - 1u));
                        p.moved[slot] = (int)n;
                        p.moved_old[slot] = old;
                    }
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c_changed += __shfl_xor_sync(0xffffffffu, c_changed, o);
            c_dist += __shfl_xor_sync(0xffffffffu, c_dist, o);
        }
        if (lane == 0) {
            if (c_changed) atomicAdd(&ctrl->n_changed, c_changed);
            if (c_dist) atomicAdd(&ctrl->n_dist, c_dist);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
    }
}

// C -> (c_h, c_l) bfloat16 copies (K padded to Kp with zero rows) and the
// FP32 norms, as the kernel above reads them; gated like the dense pass
__global__ void k_split_c(Params p, int Kp, int respect_done, int if_dense) {
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (if_dense && !*(volatile int *)&ctrl->dense_mode) return;
    const int D = p.D, Dt = tc_dim(p.D);
    const int64_t total = (int64_t)Kp * Dt;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(i / Dt), d = (int)(i - (int64_t)k * Dt);
        float x = (k < p.K && d < D) ? p.C[(size_t)k * p.Dp + d] : 0.f;  // zero padding
        if (p.mu && k < p.K && d < D) x = __fsub_rn(x, p.mu[d]);  // c - mu
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
        p.Ch[i] = __bfloat16_as_ushort(h);
        p.Cl[i] = __bfloat16_as_ushort(l);
    }
    // norms: one warp per centroid, the same two-accumulator FP32 sum as the
    // single-block kernel (even / odd coordinates, then added)
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t k = wid; k < p.K; k += nw) {
        if (lane == 0) {
            const float *c = p.C + (size_t)k * p.Dp;
            float a0 = 0.f, a1 = 0.f;
            for (int d = 0; d + 1 < D; d += 2) {  // ||c - mu||^2, the values split above
                const float v0 = p.mu ? __fsub_rn(c[d], p.mu[d]) : c[d];
                const float v1 = p.mu ? __fsub_rn(c[d + 1], p.mu[d + 1]) : c[d + 1];
                a0 = fmaf(v0, v0, a0);
                a1 = fmaf(v1, v1, a1);
            }
            p.cnorm[k] = a0 + a1;
        }
    }
}

bool plan_b(const Params &p, size_t smem_limit, TcbCfg &cfg, size_t &smem) {
    const int Dt = tc_dim(p.D);
    if (!Dt || p.K <= 256) return false;
    cfg.Kp = ((p.K + kNB - 1) / kNB) * kNB;
    if (cfg.Kp > kMaxKp) return false;
    cfg.nb = cfg.Kp / kNB;
    // groups that 64 columns (the span between two flushes of the staged
    // minima) can close under the contiguous grouping j -> j G / K, plus the
    // one still open
    int most = 0;
    for (int j = 0; j < cfg.Kp / 64; ++j) {
        const int64_t c0 = (int64_t)j * 64, c1 = std::min<int64_t>((int64_t)(j + 1) * 64, p.K) - 1;
        if (c0 >= p.K) break;
        const int g0 = (int)(c0 * p.G / p.K), g1 = (int)(c1 * p.G / p.K);
        most = std::max(most, g1 - g0 + 1);
    }
    cfg.srow = (most + 2) | 1;
    const size_t NA = Dt / 64;
    const size_t a_stage = 2 * NA * (size_t)kAtomBytes;
    const size_t b_stage = 2 * NA * (size_t)kBAtom;
    const size_t tables = (size_t)cfg.Kp * 8 + (size_t)cfg.Kp / 32 * 4;
    const size_t stage_bytes = (size_t)kPairs * kEpiWarps * 32 * cfg.srow * 4;
    const size_t bars = (4 + 2 * 2 + 8 + 1) * 8 + 16;
    auto need = [&](int bst) { return 1024 + 2 * a_stage + bst * b_stage + tables + 16 + stage_bytes + bars + 16; };
    cfg.bst = need(2) <= smem_limit ? 2 : 1;
    if (need(cfg.bst) > smem_limit) return false;
    size_t off = 0;
    cfg.off_A = (uint32_t)off;
    off += 2 * a_stage;
    cfg.off_B = (uint32_t)off;
    off += cfg.bst * b_stage;
    cfg.off_cn = (uint32_t)off;
    off += (size_t)cfg.Kp * 8;
    cfg.off_bm = (uint32_t)off;
    off += ((size_t)cfg.Kp / 32 * 4 + 15) & ~size_t(15);
    cfg.off_stage = (uint32_t)off;
    off += stage_bytes;
    off = (off + 7) & ~size_t(7);
    cfg.off_bar = (uint32_t)off;
    off += (4 + 2 * cfg.bst + 8 + 1) * 8 + 16;
    smem = 1024 + off;
    if (smem > smem_limit) return false;
    cfg.num_tiles = (int)((p.N + kTM - 1) / kTM);
    const double D = Dt;  // the padded width (zero products add nothing)
    cfg.e_lin = (float)(1.25 * (6.1 * std::ldexp(1.0, -16) + (6 * D + 1) * std::ldexp(1.0, -23)) * (1 + 1e-6));
    cfg.e_c2 = (float)(1.25 * (D + 3) * std::ldexp(1.0, -24) * (1 + 1e-6));
    // ||x - mu||^2 from k_split_x: an FP32 sum of non-negative terms in which
    // each term meets at most 4 + log2(Dt / 4) <= 9 roundings, so the relative
    // error is below 9.01 2^-24 < 2^-20
    const double rel = std::ldexp(1.0, -20);
    cfg.xn_lo = (float)(1.0 - rel);
    cfg.xn_hi = (float)(1.0 + rel);
    return true;
}

template <int D>
cudaError_t launch_b(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms, size_t smem_limit,
                     int if_dense) {
    TcbCfg cfg;
    size_t smem;
    if (!plan_b(p, smem_limit, cfg, smem) || !p.Xh || !p.Xl || !p.xnorm || !p.Ch || !p.Cl || !p.cnorm)
        return cudaErrorNotSupported;
    auto enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tmh, tml, tmch, tmcl;
    const int Dt = tc_dim(p.D);
    cuuint64_t gx[2] = {(cuuint64_t)Dt, (cuuint64_t)p.N}, sx[1] = {(cuuint64_t)Dt * 2};
    cuuint64_t gc[2] = {(cuuint64_t)Dt, (cuuint64_t)cfg.Kp};
    cuuint32_t bx[2] = {64, (cuuint32_t)kTM}, bc[2] = {64, (cuuint32_t)kNB}, es[2] = {1, 1};
    struct M {
        CUtensorMap *m;
        const uint16_t *src;
        cuuint64_t *g;
        cuuint32_t *b;
    } maps[4] = {{&tmh, p.Xh, gx, bx}, {&tml, p.Xl, gx, bx}, {&tmch, p.Ch, gc, bc}, {&tmcl, p.Cl, gc, bc}};
    for (auto &m : maps)
        if (enc(m.m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(m.src), m.g, sx, m.b, es,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return cudaErrorInvalidValue;
    {
        const int64_t total = (int64_t)cfg.Kp * Dt;
        const int64_t grid = std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, (int64_t)num_sms * 4));
        count_launch();
        k_split_c<<<(unsigned)grid, 256, 0, s>>>(p, cfg.Kp, respect_done, if_dense);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaFuncSetAttribute(k_dense_tcb<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(cfg.num_tiles, num_sms);
    count_launch();
    k_dense_tcb<D><<<grid, kThreads, smem, s>>>(tmh, tml, tmch, tmcl, p, cfg, first, respect_done, if_dense);
    return cudaGetLastError();
}

}  // namespace

bool dense_tcb_eligible(const Params &p, size_t smem_limit) {
    TcbCfg cfg;
    size_t smem;
    return encoder() != nullptr && plan_b(p, smem_limit, cfg, smem);
}

int dense_tcb_kp(const Params &p) { return ((p.K + kNB - 1) / kNB) * kNB; }

cudaError_t launch_dense_tcb(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms,
                             size_t smem_limit, int if_dense) {
    switch (tc_dim(p.D)) {
    case 64: return launch_b<64>(p, s, first, respect_done, num_sms, smem_limit, if_dense);
    case 128: return launch_b<128>(p, s, first, respect_done, num_sms, smem_limit, if_dense);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace kp
