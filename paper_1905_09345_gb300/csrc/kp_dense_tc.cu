// kp_dense_tc.cu -- dense assignment on the 5th-generation tensor cores.
//
// The distance calculator of KPynq (Sec. I) evaluates every pair the filters
// leave; when that is (nearly) every pair -- iteration 0, plain Lloyd, or a
// filtered iteration in which most points survive -- the evaluation is a
// dense contraction, ||x||^2 - 2 x.c + ||c||^2, and belongs on the tensor
// cores.
//
// Mixed precision with a bounded error ("BF16x3"): every FP32 value v is
// split into two bfloat16 numbers, v_h = bf16(v) and v_l = bf16(v - v_h), and
//     x.c ~ x_h.c_h + x_h.c_l + x_l.c_h
// is accumulated in FP32 by tcgen05.mma (kind::f16, M=128 points x N<=256
// centroids, K=16 per instruction, three instructions per K step).  X is
// split once per context into two bfloat16 copies that TMA loads with
// 128-byte swizzle; the centroid block is split into shared memory by the
// CTA itself.  Accumulators live in TMEM, double-buffered across two
// epilogue warp groups.
//
// Persistent CTA per SM: warp 0 issues TMA, one thread of warp 1 issues the
// MMAs, warps 2..17 (two groups of eight, two warps per TMEM lane quadrant,
// each scanning half of the columns) read the accumulators back with
// tcgen05.ld, one TMEM lane (= point) per thread, and turn
// t_k = ||c_k||^2 - 2 x.c_k into the winner, the runner-up and the per-group
// minima.  Lower bounds are t-based with the error E(x) subtracted, the upper
// bound adds it; when the runner-up lies within 2E of the winner the point is
// settled exactly by kp_settle.cu (FP32 direct differences, then FP64 if the
// FP32 error bound cannot decide), so labels are exact.
//
// Error model of t_k (per point; c_max = max ||c_k||, c2_max = max ||c_k||^2):
//   the split leaves |v - v_h - v_l| <= 2^-16 |v| (bfloat16 unit roundoff
//   2^-8, twice), so the three products miss at most 3.05 2^-16 |x_i c_i|;
//   products are exact in FP32 and the accumulation of 3D of them adds at
//   most 3D 2^-23 (Cauchy-Schwarz bounds sum |x_i c_i| by ||x|| ||c||);
//   ||c||^2 is an FP32 sum of squares and the final fma rounds once:
//     |t~ - t| <= (6.1 2^-16 + (6D+1) 2^-23) ||x|| ||c|| + (D+3) 2^-24 ||c||^2,
//   used with a 1.25x margin as E(x).
#include "kp_tc.cuh"

namespace kp {

namespace {

constexpr int kEpiWarps = 8;      // warps per epilogue group: two per TMEM lane quadrant
constexpr int kGroups = 2;        // epilogue groups = TMEM buffers
constexpr int kTcThreads = 64 + kGroups * kEpiWarps * 32;

// the two warps of a quadrant (named barrier `id`, 64 threads): every thread
// contributes v, every thread gets the AND
__device__ __forceinline__ bool pair_and(bool v, int id) {
    int out;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\tbar.red.and.pred q, %2, 64, p;\n\t"
        "selp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(out)
        : "r"((int)v), "r"(id)
        : "memory");
    return out != 0;
}
__device__ __forceinline__ void pair_sync(int id) { asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory"); }

struct TcCfg {
    int Kp;        // centroid rows in shared memory (multiple of 32, <= 256)
    int stages;    // A pipeline depth
    int tmem_cols; // allocated TMEM columns (2 buffers)
    int buf_cols;  // columns per buffer (>= Kp, power of two)
    uint32_t off_A, off_cn, off_gs, off_stage, off_bar;
    int num_tiles;
    float e_lin;   // 1.25 (6.1 2^-16 + (6D+1) 2^-23), rounded up
    float e_c2;    // 1.25 (D+3) 2^-24, rounded up
    float xn_lo, xn_hi;  // relative error of the precomputed ||x - mu||^2
};

template <int D>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_dense_tc(const __grid_constant__ CUtensorMap tmh, const __grid_constant__ CUtensorMap tml, Params p, TcCfg cfg,
               int first, int respect_done, int if_dense) {
    extern __shared__ uint8_t raw[];
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    if (if_dense && !*(volatile int *)&ctrl->dense_mode) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->path = KM_PATH_DENSE_TC;
    constexpr int NA = D / 64;  // 64-element atoms per row
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    const int Kp = cfg.Kp;
    const int b_atom = Kp * 128;
    uint8_t *sBh = sm;
    uint8_t *sBl = sm + NA * b_atom;
    uint8_t *sA = sm + cfg.off_A;  // stage s: [NA atoms of x_h][NA atoms of x_l]
    float *cn = reinterpret_cast<float *>(sm + cfg.off_cn);  // [Kp] ||c||^2 (+inf: padding)
    float *pen = cn + Kp;  // [Kp] +inf where a group opens, else 0
    uint32_t *bm = reinterpret_cast<uint32_t *>(sm + cfg.off_gs);  // [Kp / 32] group-start masks
    float *stage = reinterpret_cast<float *>(sm + cfg.off_stage);  // [2 groups x 128 rows][Gp + 1]
    float4 *mrg = reinterpret_cast<float4 *>(stage + (size_t)kGroups * kTM * (p.Gp + 1));  // [2 x 128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + cfg.off_bar);
    const int S = cfg.stages;
    uint64_t *full_a = bars;
    uint64_t *empty_a = bars + S;
    uint64_t *acc_full = bars + 2 * S;  // [kGroups]
    uint64_t *acc_empty = bars + 2 * S + kGroups;
    uint64_t *mma_done = bars + 2 * S + 2 * kGroups;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * S + 2 * kGroups + 1);
    float *c2max_s = reinterpret_cast<float *>(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int v = ctrl->v;
    const int K = p.K, G = p.G;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            bar_init(&full_a[i], 1);
            bar_init(&empty_a[i], 1);  // the commit of the MMAs that read the stage
        }
        for (int g = 0; g < kGroups; ++g) {
            bar_init(&acc_full[g], 1);
            bar_init(&acc_empty[g], kEpiWarps);
        }
        bar_init(mma_done, 1);
        *c2max_s = 0.f;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(cfg.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    for (int c = threadIdx.x; c < Kp / 32; c += blockDim.x) bm[c] = 0u;
    // the centroid block, split into x_h / x_l bfloat16 tiles (128-byte swizzle),
    // and the exact FP32 norms (padding rows: zero tiles, norm +inf)
    for (int idx = threadIdx.x; idx < Kp * (D / 8); idx += blockDim.x) {
        const int row = idx / (D / 8), q = idx - row * (D / 8);
        float vals[8];
        if (row < K && q * 8 < p.D) {  // coordinates beyond D: zero padding
            const float4 a = *reinterpret_cast<const float4 *>(p.C + (size_t)row * p.Dp + q * 8);
            const float4 b = *reinterpret_cast<const float4 *>(p.C + (size_t)row * p.Dp + q * 8 + 4);
            vals[0] = a.x; vals[1] = a.y; vals[2] = a.z; vals[3] = a.w;
            vals[4] = b.x; vals[5] = b.y; vals[6] = b.z; vals[7] = b.w;
            if (p.mu)  // c - mu (mu's padding columns are zero)
#pragma unroll
                for (int i = 0; i < 8; ++i) vals[i] = __fsub_rn(vals[i], p.mu[q * 8 + i]);
        } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) vals[i] = 0.f;
        }
        uint4 h, l;
        split8(vals, h, l);
        *reinterpret_cast<uint4 *>(sBh + swz_chunk(row, q, b_atom)) = h;
        *reinterpret_cast<uint4 *>(sBl + swz_chunk(row, q, b_atom)) = l;
    }
    {
        float cm = 0.f;
        for (int k = threadIdx.x; k < Kp; k += blockDim.x) {
            float s2 = INFINITY;
            if (k < K) {
                const float *c = p.C + (size_t)k * p.Dp;
                float a0 = 0.f, a1 = 0.f;
                for (int d = 0; d + 1 < p.D; d += 2) {  // ||c - mu||^2, the values split above
                    const float v0 = p.mu ? __fsub_rn(c[d], p.mu[d]) : c[d];
                    const float v1 = p.mu ? __fsub_rn(c[d + 1], p.mu[d + 1]) : c[d + 1];
                    a0 = fmaf(v0, v0, a0);
                    a1 = fmaf(v1, v1, a1);
                }
                s2 = a0 + a1;
                cm = fmaxf(cm, s2);
            }
            cn[k] = s2;
            pen[k] = 0.f;
        }
        cm = warp_max(cm);
        __syncthreads();  // c2max_s and the masks initialised
        if (lane == 0 && cm > 0.f) atomicMax(reinterpret_cast<int *>(c2max_s), __float_as_int(cm));
        // group g >= 1 starts at column gstart[g] (< K <= Kp)
        for (int g = 1 + threadIdx.x; g < G; g += blockDim.x) {
            const int col = p.gstart[g];
            if ((unsigned)col < (unsigned)Kp) {
                atomicOr(&bm[col >> 5], 1u << (col & 31));
                pen[col] = INFINITY;
            }
        }
    }
    // generic-proxy writes of the B tiles must be visible to the tensor cores
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmh) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tml) : "memory");
            int i = 0;
            bool ok = true;
            for (int tile = blockIdx.x; tile < cfg.num_tiles && ok; tile += gridDim.x, ++i) {
                const int s = i % S, f = i / S;
                if (f > 0) ok = bar_wait(&empty_a[s], (f - 1) & 1, ctrl);
                if (!ok) break;
                uint8_t *st = sA + (size_t)s * 2 * NA * kAtomBytes;
                mbar_arrive_expect_tx(&full_a[s], (uint32_t)(2 * NA * kAtomBytes));
                for (int a = 0; a < NA; ++a) {
                    tma_2d(st + a * kAtomBytes, &tmh, 64 * a, tile * kTM, &full_a[s]);
                    tma_2d(st + (NA + a) * kAtomBytes, &tml, 64 * a, tile * kTM, &full_a[s]);
                }
            }
            // drain: every issued copy has landed before the block can exit
            const int issued = i;
            for (int j = issued - S < 0 ? 0 : issued - S; j < issued; ++j)
                bar_wait(&full_a[j % S], (j / S) & 1, ctrl);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            // kind::f16: F32 accumulate, BF16 A and B, K-major, N = Kp, M = 128
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(Kp >> 3) << 17) |
                                   ((uint32_t)(kTM >> 4) << 24);
            bool ok = true;
            int i = 0;
            for (int tile = blockIdx.x; tile < cfg.num_tiles && ok; tile += gridDim.x, ++i) {
                const int s = i % S, f = i / S;
                const int buf = i % kGroups, u = i / kGroups;
                if (u > 0 && !(ok = bar_wait(&acc_empty[buf], (u - 1) & 1, ctrl))) break;
                if (!(ok = bar_wait(&full_a[s], f & 1, ctrl))) break;
                tc_fence_after();
                const uint32_t d_tmem = tmem + (uint32_t)(buf * cfg.buf_cols);
                const uint8_t *st = sA + (size_t)s * 2 * NA * kAtomBytes;
#pragma unroll
                for (int ks = 0; ks < D / 16; ++ks) {
                    const int a = ks >> 2, j = ks & 3;
                    const uint64_t dah = desc_sw128(smem_u32(st + a * kAtomBytes + j * 32));
                    const uint64_t dal = desc_sw128(smem_u32(st + (NA + a) * kAtomBytes + j * 32));
                    const uint64_t dbh = desc_sw128(smem_u32(sBh + a * b_atom + j * 32));
                    const uint64_t dbl = desc_sw128(smem_u32(sBl + a * b_atom + j * 32));
                    const uint32_t acc = ks > 0;
                    asm volatile(
                        "{\n\t.reg .pred p, q;\n\tsetp.ne.b32 p, %4, 0;\n\tsetp.eq.b32 q, %4, %4;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %5, %3, q;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %6, %2, %3, q;\n\t}" ::"r"(d_tmem),
                        "l"(dah), "l"(dbh), "r"(idesc), "r"(acc), "l"(dbl), "l"(dal)
                        : "memory");
                }
                // the A stage is free once these MMAs have read it
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty_a[s]))
                             : "memory");
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&acc_full[buf]))
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
        // Two warps per TMEM lane quadrant and group: half 0 scans the first
        // half of the accumulator columns and finishes the rows, half 1 scans
        // the second half; the pair meets at a 64-thread named barrier (1..8).
        const int e = warp - 2;
        const int grp_id = e / kEpiWarps;
        const int half = (e % kEpiWarps) / 4;
        const int pid = 1 + grp_id * 4 + ((e % kEpiWarps) & 3);
        const int q = warp & 3;  // TMEM lane quadrant of this warp
        const int r = q * 32 + lane;
        const bool bounds = p.algo == KM_ALGO_FILTERED;
        const float c2max = __fmul_ru(*c2max_s, 1.0f + 1.0f / 1024);
        const float cmax = sqrt_hi(c2max);
        const float ec2 = __fmul_ru(cfg.e_c2, c2max);
        float *row = stage + (size_t)(grp_id * kTM + r) * (p.Gp + 1);  // shared by the pair
        float4 *mrow = mrg + grp_id * kTM + r;                       // half 1's result for half 0
        // column chunks of 32: half 0 takes [0, ha), half 1 [ha, nch); half 1's
        // first store lands in the slot of the group open at its first column's
        // left neighbour, which half 0 merges with its own last minimum
        const int nch = Kp >> 5, ha = (nch + 1) >> 1;
        const int k0 = half ? ha : 0, k1 = half ? nch : ha;
        const int gsplit = nch > 1 ? group_of(bm, 32 * ha - 1) : 0;
        unsigned long long c_changed = 0, c_recheck = 0, c_dist = 0;
        auto write_req = [&](int64_t n, int old, int i1, float xlo, float b1, float E, unsigned long long gmask) {
            SettleReq rq;
            rq.n = (int32_t)n;
            rq.old = old;
            rq.i1 = i1;
            // every column is at least b1: when i1 loses, this bounds both i1's
            // group (which now keeps i1) and the winner's group
            rq.lb_alt = sqrt_lo(__fsub_rd(__fadd_rd(xlo, b1), E));
            rq.gmask = gmask;
            rq.lim = 0.f;
            p.sreq[n] = rq;
        };
        // the lb-row store: this lane's first float4 of a 16-row block and the
        // step of 32 float4s, as (row, column) pairs
        const int st_q4 = p.Gp >> 2;
        const int st_r0 = lane / st_q4, st_g0 = lane - st_r0 * st_q4;
        const int st_dr = 32 / st_q4, st_dg = 32 - st_dr * st_q4;
        int i = grp_id;
        for (int tile = blockIdx.x + grp_id * gridDim.x; tile < cfg.num_tiles;
             tile += kGroups * gridDim.x, i += kGroups) {
            const int u = i / kGroups;
            // waits are warp-uniform (the TMEM loads below are warp-collective)
            // and pair-uniform (the named barriers need both warps)
            const bool ok = __all_sync(0xffffffffu, bar_wait(&acc_full[grp_id], u & 1, ctrl));
            if (!pair_and(ok, pid)) break;
            tc_fence_after();
            const int64_t n = (int64_t)tile * kTM + r;
            const bool valid = n < p.N;
            int old = -1;
            float xlo = 0.f, xup = 0.f, E = 0.f, xn = 0.f;
            bool need_row = false;  // half 0: this row's settle request, written after the conversion
            int best_row = 0;
            float b1_row = 0.f;
            if (half == 0) {
                // the previous label and the row norm, read now so that their
                // latency hides behind the scan (the error window that needs the
                // norm is formed after it)
                old = valid ? (first ? -1 : p.label[n]) : -1;
                xn = valid ? p.xnorm[n] : 0.f;
            }
            const uint32_t tb = tmem + (uint32_t)(grp_id * cfg.buf_cols) + ((uint32_t)(q * 32) << 16);

            // pass 1: group minima (staged), winner (lowest index on ties), runner-up
            // over this half's columns; the next 32 columns are read from TMEM
            // while the current ones are scanned
            RowScan A;
            A.init(half ? row + gsplit : row);
            if (k0 < k1) {  // 16 columns at a time, the next 16 in flight
                const int c0 = 32 * k0, c1 = 32 * k1;
                uint32_t ra[16], rb[16];
                tmem_ld16_async(tb + c0, ra);
                for (int c = c0; c < c1; c += 32) {  // warp-uniform; c1 - c0 is a multiple of 32
                    tmem_wait16(ra);
                    tmem_ld16_async(tb + c + 16, rb);
                    scan_one<16>(A, ra, c, cn, pen);
                    tmem_wait16(rb);
                    if (c + 32 < c1) tmem_ld16_async(tb + c + 32, ra);
                    scan_one<16>(A, rb, c + 16, cn, pen);
                }
            }
            // accumulators no longer needed
            tc_fence_before();
            __syncwarp();
            if (lane == 0) bar_arrive(&acc_empty[grp_id]);
            if (half) {
                if (nch > 1) A.close();
                float c1, c2;
                int ci;
                A.result(c1, ci, c2);
                *mrow = make_float4(c1, c2, __int_as_float(ci), 0.f);
            }
            pair_sync(pid);  // half 1's minima and result are in shared memory
            if (half == 0) {
                float b1, b2;
                int i1;
                {
                    if (nch > 1) {
                        const float gmA = A.gm;
                        row[gsplit] = fminf(row[gsplit], gmA);
                    } else {
                        A.close();
                    }
                    float a1, a2;
                    int ai;
                    A.result(a1, ai, a2);
                    const float4 m = *mrow;
                    const float c1 = m.x, c2 = m.y;
                    const int ci = __float_as_int(m.z);
                    // half 0 holds the lower indices: it wins ties
                    const bool bw = c1 < a1;
                    b1 = bw ? c1 : a1;
                    i1 = bw ? ci : ai;
                    b2 = fminf(fminf(a2, c2), fmaxf(a1, c1));
                }
                xlo = __fmul_rd(xn, cfg.xn_lo);
                xup = __fmul_ru(xn, cfg.xn_hi);
                E = __fmaf_ru(cfg.e_lin, __fmul_ru(sqrt_hi(xup), cmax), ec2);
                const float R = __fadd_ru(sqrt_hi(xup), cmax);  // bounds ||x - mu|| + ||c - mu||
                E = __fmaf_ru(p.e_cen, __fmul_ru(R, R), E);
                const float twoE = __fmul_ru(2.f, E);
                const float thr = __fadd_ru(b1, twoE);

                // Rows whose runner-up is inside the error window go to the settle
                // queue: k_settle decides them exactly afterwards from FP32 (and
                // FP64) distances to the centroids of the groups whose minimum lies
                // in the window (every other centroid is strictly farther than the
                // tensor-core winner i1, which is among them).  The epilogue writes
                // such a row's bounds as if the tensor-core winner i1 won; k_settle
                // corrects them when it does not.
                const bool need = valid && b2 <= thr;
                need_row = bounds && need;
                best_row = i1;
                b1_row = b1;
                {
                    const unsigned nm = __ballot_sync(0xffffffffu, need);
                    // The groups that can hold a window column: group minimum
                    // within the window (at most 64 groups; more: all of them).
                    // With bounds, the pair tests its halves of the groups while
                    // converting them, and half 0 writes the request afterwards.
                    if (nm && !bounds) {
                        unsigned long long gmask = ~0ull;
                        if (G <= 64) {
                            gmask = 0ull;
                            for (int g = 0; g < G; ++g) gmask |= (row[g] <= thr) ? (1ull << g) : 0ull;
                        }
                        if (need) write_req(n, old, i1, xlo, b1, E, gmask);
                    }
                    // the warp's 32 rows in the request bitmap (every word is written
                    // by every dense pass, so the bitmap needs no clearing)
                    if (lane == 0) p.sbits[(int64_t)tile * (kTM / 32) + q] = nm;
                }

                const int best = i1;
                if (valid) {
                    c_dist += (unsigned long long)K;
                    if (!need) p.label[n] = best;
                    if (bounds) {
                        // the winner's group must exclude the winner: every other
                        // column is at least the runner-up b2 (at least b1 when the
                        // exact winner is not the tensor-core winner); staged in t
                        // and converted with the other groups below
                        const float tw = best == i1 ? b2 : b1;
                        const float lw = tw == INFINITY ? INFINITY : sqrt_lo(__fsub_rd(__fadd_rd(xlo, tw), E));
                        row[group_of(bm, best)] = tw;
                        // the bound is monotone in t, so the smallest group bound is
                        // the bound of the smallest column other than the winner
                        p.lbg[n] = lw;
                        p.u[n] = sqrt_hi(__fadd_ru(__fadd_ru(xup, b1), E));
                        p.stamp[n] = make_stamp(v, v);
                    }
                }
                *mrow = make_float4(xlo, E, thr, 0.f);  // for half 1's share of the conversion
                {
                    // label changes: one slot reservation per warp
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
            pair_sync(pid);  // half 0's winner fixes and (x_lo, E) are in shared memory
            if (bounds) {
                // s_c >= xn_lo + t_c - E for every column c: the pair converts the
                // row's group minima, half 0 the first half of the groups
                // and each half marks its groups whose minimum is within the
                // window (bit g - g0; the winner's group holds tw = b2 <= thr)
                const int gh = (G + 1) >> 1;
                uint32_t gbits = 0u;
                if (valid) {
                    const float4 xe = *mrow;
                    const int g0 = half ? gh : 0, g1 = half ? G : gh;
                    if (G <= 64) {  // gh <= 32: one 32-bit word per half
#pragma unroll 4
                        for (int g = g0; g < g1; ++g) {
                            const float tg = row[g];
                            gbits |= (tg <= xe.z ? 1u : 0u) << (g - g0);
                            row[g] = tg == INFINITY ? INFINITY : sqrt_lo(__fsub_rd(__fadd_rd(xe.x, tg), xe.y));
                        }
                    } else {
#pragma unroll 4
                        for (int g = g0; g < g1; ++g) {
                            const float tg = row[g];
                            row[g] = tg == INFINITY ? INFINITY : sqrt_lo(__fsub_rd(__fadd_rd(xe.x, tg), xe.y));
                        }
                    }
                    if (half) row[p.Gp] = __uint_as_float(gbits);  // the slot past the groups
                }
                pair_sync(pid);  // the rows' bounds and half 1's group bits are complete
                if (half == 0 && need_row) {
                    const unsigned long long gmask =
                        G <= 64 ? ((unsigned long long)gbits | ((unsigned long long)__float_as_uint(row[p.Gp]) << gh))
                                : ~0ull;
                    write_req(n, old, best_row, xlo, b1_row, E, gmask);
                }
                // the quadrant's 32 rows (consecutive points) as one contiguous
                // block, half 0 the first 16 rows, half 1 the rest
                const int64_t n0 = (int64_t)tile * kTM + q * 32;
                const int rows = (int)min((int64_t)32, p.N - n0);
                const int r0 = half * 16, r1 = min(rows, r0 + 16);
                if (r1 > r0) {
                    // rows x Gp floats, contiguous in lb: 16-byte stores (Gp is a
                    // multiple of 4, so no vector crosses a row); lane-strided
                    // element e = rw * q4 + gq, (rw, gq) stepped without division
                    const int Gp = p.Gp;
                    const float *st0 = stage + (size_t)(grp_id * kTM + q * 32) * (Gp + 1);
                    float4 *dst = reinterpret_cast<float4 *>(p.lb + n0 * Gp);
                    for (int rw = r0 + st_r0, gq = st_g0; rw < r1;) {
                        const int g = gq * 4;
                        const float *src = st0 + rw * (Gp + 1) + g;
                        float4 v4;
                        v4.x = g < G ? src[0] : 0.f;
                        v4.y = g + 1 < G ? src[1] : 0.f;
                        v4.z = g + 2 < G ? src[2] : 0.f;
                        v4.w = g + 3 < G ? src[3] : 0.f;
                        dst[rw * st_q4 + gq] = v4;
                        rw += st_dr;
                        gq += st_dg;
                        if (gq >= st_q4) {
                            gq -= st_q4;
                            ++rw;
                        }
                    }
                }
            }
            pair_sync(pid);  // the row slots are free for the pair's next tile
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            c_changed += __shfl_xor_sync(0xffffffffu, c_changed, o);
            c_recheck += __shfl_xor_sync(0xffffffffu, c_recheck, o);
            c_dist += __shfl_xor_sync(0xffffffffu, c_dist, o);
        }
        if (lane == 0) {
            if (c_changed) atomicAdd(&ctrl->n_changed, c_changed);
            if (c_recheck) atomicAdd(&ctrl->n_recheck, c_recheck);
            if (c_dist) atomicAdd(&ctrl->n_dist, c_dist);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cfg.tmem_cols)
                     : "memory");
    }
}

// X -> (x_h, x_l) bfloat16 copies with rows of Dt >= D coordinates (zero
// padding), four elements per thread, and each row's ||x - mu||^2 (FP32 sum of
// the squares of the values split, reduced over the Dt / 4 lanes of the row).
// Dt / 4 is 16 or 32 and the loop steps by whole warps, so a row's lanes are
// one aligned half-warp or warp and all of them run every iteration.
__global__ void k_split_x(const float *X, int64_t N, int D, int Dt, uint2 *Xh, uint2 *Xl, float4 *Xcopy,
                          const float *mu, float *xnorm) {
    const int q4n = Dt / 4;
    const int64_t n4 = N * q4n;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n4; base += stride) {
        const int64_t i = base + lane;
        const bool act = i < n4;
        const int64_t row = i / q4n;
        const int q4 = (int)(i - row * q4n);
        float ss = 0.f;
        if (act) {
            const float4 a =
                q4 * 4 < D ? *reinterpret_cast<const float4 *>(X + row * D + q4 * 4) : make_float4(0, 0, 0, 0);
            if (Xcopy && q4 * 4 < D) Xcopy[(row * D + q4 * 4) / 4] = a;  // the device copy, in the same pass
            // x - mu, rounded once to FP32 (the padding stays exactly zero)
            const float4 m =
                (mu && q4 * 4 < D) ? *reinterpret_cast<const float4 *>(mu + q4 * 4) : make_float4(0, 0, 0, 0);
            const float vv[4] = {__fsub_rn(a.x, m.x), __fsub_rn(a.y, m.y), __fsub_rn(a.z, m.z), __fsub_rn(a.w, m.w)};
            uint32_t hw[2], lw[2];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                __nv_bfloat16 h0 = __float2bfloat16_rn(vv[2 * k]), h1 = __float2bfloat16_rn(vv[2 * k + 1]);
                __nv_bfloat16 l0 = __float2bfloat16_rn(vv[2 * k] - __bfloat162float(h0));
                __nv_bfloat16 l1 = __float2bfloat16_rn(vv[2 * k + 1] - __bfloat162float(h1));
                hw[k] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
                lw[k] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
            }
            Xh[i] = make_uint2(hw[0], hw[1]);
            Xl[i] = make_uint2(lw[0], lw[1]);
#pragma unroll
            for (int k = 0; k < 4; ++k) ss = fmaf(vv[k], vv[k], ss);
        }
        for (int o = q4n >> 1; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
        if (act && q4 == 0 && xnorm) xnorm[row] = ss;
    }
}

int pow2_at_least(int x) {
    int p2 = 32;
    while (p2 < x) p2 <<= 1;
    return p2;
}

bool plan(const Params &p, size_t smem_limit, TcCfg &cfg, size_t &smem) {
    const int Dt = tc_dim(p.D);
    if (!Dt || p.K > 256) return false;
    cfg.Kp = ((p.K + 31) / 32) * 32;
    cfg.buf_cols = pow2_at_least(cfg.Kp);
    cfg.tmem_cols = kGroups * cfg.buf_cols;
    if (cfg.tmem_cols > 512) return false;
    const size_t NA = Dt / 64;
    const size_t b_bytes = 2 * NA * (size_t)cfg.Kp * 128;
    const size_t a_stage = 2 * NA * (size_t)kAtomBytes;
    const size_t cn_bytes = (size_t)cfg.Kp * 8;  // norms and group-opening penalties
    const size_t gs_bytes = (((size_t)cfg.Kp / 32) * 4 + 15) & ~size_t(15);  // group-start masks
    const size_t stage_bytes = (size_t)kGroups * kTM * (p.Gp + 1) * 4 + (size_t)kGroups * kTM * 16;
    const size_t fixed = 1024 + b_bytes + cn_bytes + gs_bytes + stage_bytes + 64 * 8 + 64;
    if (fixed + 2 * a_stage > smem_limit) return false;
    cfg.stages = (int)std::min<size_t>(6, (smem_limit - fixed) / a_stage);
    size_t off = b_bytes;
    cfg.off_A = (uint32_t)off;
    off += cfg.stages * a_stage;
    cfg.off_cn = (uint32_t)off;
    off += cn_bytes;
    cfg.off_gs = (uint32_t)off;
    off += gs_bytes;
    cfg.off_stage = (uint32_t)off;
    off += stage_bytes;
    off = (off + 7) & ~size_t(7);
    cfg.off_bar = (uint32_t)off;
    off += (2 * cfg.stages + 2 * kGroups + 1) * 8 + 16;
    smem = 1024 + off;
    if (smem > smem_limit) return false;
    cfg.num_tiles = (int)((p.N + kTM - 1) / kTM);
    const double D = Dt;  // the padded width: its zero products add nothing, the bound stays valid
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
cudaError_t launch_t(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms, size_t smem_limit,
                     int if_dense) {
    TcCfg cfg;
    size_t smem;
    if (!plan(p, smem_limit, cfg, smem) || !p.Xh || !p.Xl || !p.xnorm) return cudaErrorNotSupported;
    auto enc = encoder();
    if (!enc) return cudaErrorNotSupported;
    CUtensorMap tmh, tml;
    const int Dt = tc_dim(p.D);
    cuuint64_t gx[2] = {(cuuint64_t)Dt, (cuuint64_t)p.N}, sx[1] = {(cuuint64_t)Dt * 2};
    cuuint32_t bx[2] = {64, (cuuint32_t)kTM}, es[2] = {1, 1};
    if (enc(&tmh, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(p.Xh), gx, sx, bx, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    if (enc(&tml, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(p.Xl), gx, sx, bx, es,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_dense_tc<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int grid = std::min(cfg.num_tiles, num_sms);
    count_launch();
    k_dense_tc<D><<<grid, kTcThreads, smem, s>>>(tmh, tml, p, cfg, first, respect_done, if_dense);
    return cudaGetLastError();
}

}  // namespace

bool dense_tc_eligible(const Params &p, size_t smem_limit) {
    TcCfg cfg;
    size_t smem;
    return encoder() != nullptr && plan(p, smem_limit, cfg, smem);
}

cudaError_t launch_split_x(const float *X, int64_t N, int D, int Dt, uint16_t *Xh, uint16_t *Xl, cudaStream_t s,
                           int num_sms, float *Xcopy, const float *mu, float *xnorm) {
    if (Dt != 64 && Dt != 128) return cudaErrorInvalidValue;  // a row's lanes: one half-warp or warp
    const int64_t n4 = N * Dt / 4;  // D and Dt are multiples of 4
    const int64_t grid = std::min<int64_t>((n4 + 255) / 256, (int64_t)num_sms * 16);
    count_launch();
    k_split_x<<<(unsigned)std::max<int64_t>(grid, 1), 256, 0, s>>>(X, N, D, Dt, reinterpret_cast<uint2 *>(Xh),
                                                                    reinterpret_cast<uint2 *>(Xl),
                                                                    reinterpret_cast<float4 *>(Xcopy), mu, xnorm);
    return cudaGetLastError();
}

cudaError_t launch_dense_tc(const Params &p, cudaStream_t s, int first, int respect_done, int num_sms,
                            size_t smem_limit, int if_dense) {
    if (p.K > 256) return launch_dense_tcb(p, s, first, respect_done, num_sms, smem_limit, if_dense);
    switch (tc_dim(p.D)) {
    case 64: return launch_t<64>(p, s, first, respect_done, num_sms, smem_limit, if_dense);
    case 128: return launch_t<128>(p, s, first, respect_done, num_sms, smem_limit, if_dense);
    default: return cudaErrorNotSupported;
    }
}

}  // namespace kp
