// kp_stats.cu -- cluster statistics (S_k = sum x in FP64, Q_k = sum
// ||x - R_k||^2 about a reference point R_k, n_k) for the centroid update.
//
// Two ways, chosen on the device after each assignment, both on the same
// three kernels: a counting sort of entries by cluster (k_stats_hist counts
// and lays out the segments, k_stats_scatter places the entries), then each
// warp sums a run of sorted entries (64; 16 when few points moved)
// coordinate-parallel and adds one partial per cluster it met to the global
// FP64 sums.  Global atomics then
// touch each cluster a few times instead of once per point.
//   * full recompute (iteration 0, or more than N/2 labels changed): one
//     entry per point, under its label; S, Q and the counts start from zero;
//   * incremental (few labels changed): two entries per relabelled point,
//     +x under its new label and -x under its old one (the sign in bit 31 of
//     the entry's id), added to the sums as they stand; the counts change by
//     the entries' signs.
#include "kp_common.cuh"

namespace kp {

constexpr int kStatsThreads = 256;
constexpr int kStatsTile = kStatsThreads * 4;  // points per block step of the scatter
constexpr int kSumRun = 64;                    // sorted entries per warp in k_stats_sum (full mode)
constexpr int kSumRunMoved = 16;               // the same for at most N/8 moved points' entries
                                               // (few, so shorter runs put more warps on them)
constexpr int kSumMaxPer = 8;                  // coordinates per lane (D <= 256)

// full when the moved points' entries (two each) would outnumber the points
__device__ __forceinline__ bool stats_full_rule(const Params &p, int all_points) {
    return all_points || (int64_t)p.ctrl->moved_count * 2 > p.N;
}

constexpr uint32_t kNegEntry = 0x80000000u;  // entry id bit: subtract the point

// Entries of the sort: full mode, point e under its label; incremental mode,
// moved point e under its new label (e < m) or, subtracted, under its old
// label (m <= e < 2m).  Returns the cluster (-1: none) and the entry's id.
__device__ __forceinline__ int stats_entry(const Params &p, bool full, int64_t m, int64_t e, uint32_t &id) {
    if (full) {
        id = (uint32_t)e;
        return checked_label(p, e);
    }
    if (e < m) {
        const int64_t n = p.moved[e];
        id = (uint32_t)n;
        return checked_label(p, n);
    }
    const int64_t n = p.moved[e - m];
    const int old = p.moved_old[e - m];
    id = (uint32_t)n | kNegEntry;
    if (old < 0) return -1;  // the point had no cluster
    if (old >= p.K) {
        atomicExch(&p.ctrl->err, kErrLabel);
        return -1;
    }
    return old;
}
__device__ __forceinline__ int64_t stats_entries(const Params &p, bool full) {
    return full ? p.N : 2 * (int64_t)p.ctrl->moved_count;
}

// Decide the mode; in full mode zero S and Q; count the entries per cluster
// (shared-memory histogram when K fits), and let the last block turn the
// counts into segment offsets (hcur) and, in full mode, the new cluster sizes
// (cnt).
__global__ void __launch_bounds__(kStatsThreads) k_stats_hist(Params p, int all_points, int respect_done) {
    extern __shared__ int hist[];
    __shared__ int last;
    __shared__ int wsum[kStatsThreads / 32];
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    const bool full = stats_full_rule(p, all_points);
    if (blockIdx.x == 0 && threadIdx.x == 0) ctrl->stats_full = full ? 1 : 0;
    const int K = p.K, D = p.D;
    const bool local = K <= p.hist_smem_k;
    const int64_t m = full ? 0 : (int64_t)ctrl->moved_count;
    const int64_t ne = stats_entries(p, full);
    // blocks taking part: one per tile of entries (the others leave at once;
    // few moved points need few blocks)
    const unsigned used = (unsigned)max((int64_t)1, min((int64_t)gridDim.x, (ne + kStatsTile - 1) / kStatsTile));
    if (blockIdx.x >= used) return;
    const int64_t tid = (int64_t)blockIdx.x * kStatsThreads + threadIdx.x;
    const int64_t nthr = (int64_t)used * kStatsThreads;
    if (full) {
        for (int64_t i = tid; i < (int64_t)K * D; i += nthr) p.S[i] = 0.0;
        for (int64_t i = tid; i < K; i += nthr) p.Q[i] = 0.0;
        // the sums start from zero: each cluster's reference point becomes its
        // current centroid (the one the update subtracts), so that Q_k holds the
        // objective term itself and the update cancels nothing large
        for (int64_t i = tid; i < (int64_t)K * p.Dp; i += nthr) p.R[i] = p.C[i];
    }
    if (local) {
        for (int i = threadIdx.x; i < K; i += kStatsThreads) hist[i] = 0;
        __syncthreads();
    }
    for (int64_t e = tid; e < ne; e += nthr) {
        uint32_t id;
        const int k = stats_entry(p, full, m, e, id);
        if (k < 0) continue;
        if (local) atomicAdd(&hist[k], 1);
        else atomicAdd(&p.hcount[k], 1);
    }
    if (local) {
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += kStatsThreads)
            if (hist[i]) atomicAdd(&p.hcount[i], hist[i]);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&ctrl->stats_ticket, 1u) == used - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    // exclusive scan of the counts: each thread a contiguous run
    const int lane = threadIdx.x & 31;
    const int per = (K + kStatsThreads - 1) / kStatsThreads;
    const int b0 = threadIdx.x * per, b1 = min(b0 + per, K);
    int run = 0;
    for (int b = b0; b < b1; ++b) run += __ldcg(p.hcount + b);
    int incl = run;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) wsum[threadIdx.x >> 5] = incl;
    __syncthreads();
    int off = incl - run;
    for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) off += wsum[w];
    for (int b = b0; b < b1; ++b) {
        const int c = __ldcg(p.hcount + b);
        p.hcur[b] = off;
        if (full) p.cnt[b] = (unsigned long long)c;
        p.hcount[b] = 0;  // ready for the next sort
        off += c;
    }
    if (threadIdx.x == 0) ctrl->stats_ticket = 0;
}

// Place every entry in its cluster's segment (per tile of 1024 entries:
// shared-memory counts, one global atomic per cluster and tile).
__global__ void __launch_bounds__(kStatsThreads) k_stats_scatter(Params p, int respect_done) {
    extern __shared__ int sh[];  // K counters | K bases
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    const bool full = *(volatile int *)&ctrl->stats_full;
    const int64_t m = full ? 0 : (int64_t)ctrl->moved_count;
    const int64_t ne = stats_entries(p, full);
    const int K = p.K;
    const bool local = K <= p.hist_smem_k;
    if (!local) {  // large K: one global atomic per entry
        for (int64_t e = (int64_t)blockIdx.x * kStatsThreads + threadIdx.x; e < ne;
             e += (int64_t)gridDim.x * kStatsThreads) {
            uint32_t id;
            const int k = stats_entry(p, full, m, e, id);
            if (k < 0) continue;
            const int pos = atomicAdd(&p.hcur[k], 1);
            p.perm[pos] = (int32_t)id;
            p.slab[pos] = k;
        }
        return;
    }
    if ((int64_t)blockIdx.x * kStatsTile >= ne) return;  // no tile for this block (block-uniform)
    int *cnt = sh;
    int *base = sh + K;
    for (int i = threadIdx.x; i < K; i += kStatsThreads) cnt[i] = 0;
    __syncthreads();
    for (int64_t t0 = (int64_t)blockIdx.x * kStatsTile; t0 < ne; t0 += (int64_t)gridDim.x * kStatsTile) {
        int k[4];
        uint32_t id[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t e = t0 + j * kStatsThreads + threadIdx.x;
            k[j] = e < ne ? stats_entry(p, full, m, e, id[j]) : -1;
            if (k[j] >= 0) atomicAdd(&cnt[k[j]], 1);
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += kStatsThreads) {
            const int c = cnt[i];
            base[i] = c ? atomicAdd(&p.hcur[i], c) : 0;
            cnt[i] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (k[j] >= 0) {
                const int pos = base[k[j]] + atomicAdd(&cnt[k[j]], 1);
                p.perm[pos] = (int32_t)id[j];
                p.slab[pos] = k[j];
            }
        }
        __syncthreads();
        for (int i = threadIdx.x; i < K; i += kStatsThreads) cnt[i] = 0;
        __syncthreads();
    }
}

// Error-free transformation of a sum (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Each warp sums a run of consecutive sorted entries, lanes over the
// coordinates, eight entries' loads in flight at a time, and adds its partial
// sums to S and Q (and, in incremental mode, the count change to cnt) whenever
// the cluster changes along the run (and at its end).  A subtracted entry
// adds -x and -||x - R_k||^2 (exact negations).
// Q_k sums ||x - R_k||^2 (R_k = the cluster's reference point, set to its
// centroid by k_stats_hist).  FP64 arithmetic is slow on the SMs of this GPU,
// so the run sums are kept as unevaluated FP32 pairs (hi + lo, compensated
// summation with TwoSum; the squares split exactly with a fused
// multiply-add), accurate to a few units in 2^-48 relative for runs this
// short, and turned into FP64 only when they are added to the global sums.
template <int NPER>  // coordinates per lane: ceil(D / 32)
__global__ void __launch_bounds__(kStatsThreads) k_stats_sum(Params p, int respect_done) {
    Ctrl *ctrl = p.ctrl;
    count_kernel(ctrl);
    if (respect_done && *(volatile int *)&ctrl->done) return;
    const bool full = *(volatile int *)&ctrl->stats_full;
    const int64_t ne = stats_entries(p, full);
    const int D = p.D;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * kStatsThreads + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * kStatsThreads) >> 5;
    constexpr int kB = 8;  // points per batch
    // entries placed: the hist kernel's count (entries without a cluster are
    // not placed), read from the segment ends
    const int64_t placed = ne == 0 ? 0 : (int64_t)__ldcg(p.hcur + (p.K - 1));
    const int run = (full || ne * 8 > p.N) ? kSumRun : kSumRunMoved;
    for (int64_t r0 = warp * run; r0 < placed; r0 += nwarps * run) {
        const int64_t r1 = min(r0 + run, placed);
        float sh[NPER], sl[NPER];
#pragma unroll
        for (int j = 0; j < NPER; ++j) sh[j] = sl[j] = 0.f;
        float qh = 0.f, ql = 0.f;
        long long dn = 0;  // count change of cluster `cur` (incremental mode)
        int cur = p.slab[r0];
        float rv[NPER];  // reference point of cluster `cur`, this lane's coordinates
        auto load_ref = [&]() {
#pragma unroll
            for (int j = 0; j < NPER; ++j) {
                const int i = lane + 32 * j;
                rv[j] = i < D ? p.R[(size_t)cur * p.Dp + i] : 0.f;
            }
        };
        load_ref();
        auto flush = [&]() {
            const double qs = warp_sum_d((double)qh + (double)ql);
#pragma unroll
            for (int j = 0; j < NPER; ++j) {
                const int i = lane + 32 * j;
                const double v = (double)sh[j] + (double)sl[j];
                if (i < D && v != 0.0) atomicAdd(&p.S[(size_t)cur * D + i], v);
                sh[j] = sl[j] = 0.f;
            }
            if (lane == 0 && qs != 0.0) atomicAdd(&p.Q[cur], qs);
            if (lane == 0 && dn != 0 && !full) atomicAdd(&p.cnt[cur], (unsigned long long)dn);  // two's complement
            qh = ql = 0.f;
            dn = 0;
        };
        for (int64_t rb = r0; rb < r1; rb += kB) {
            int nb[kB], kb[kB];
            bool neg[kB];
            float xv[kB][NPER];
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                const bool ok = rb + b < r1;
                const uint32_t id = ok ? (uint32_t)p.perm[rb + b] : 0u;
                nb[b] = (int)(id & ~kNegEntry);
                neg[b] = (id & kNegEntry) != 0u;
                kb[b] = ok ? p.slab[rb + b] : -1;
            }
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                const float *x = p.X + (int64_t)nb[b] * D;
#pragma unroll
                for (int j = 0; j < NPER; ++j) {
                    const int i = lane + 32 * j;
                    xv[b][j] = (kb[b] >= 0 && i < D) ? __ldg(x + i) : 0.f;
                }
            }
#pragma unroll
            for (int b = 0; b < kB; ++b) {
                if (kb[b] < 0) break;
                if (kb[b] != cur) {  // warp-uniform
                    flush();
                    cur = kb[b];
                    load_ref();
                }
                const float sg = neg[b] ? -1.f : 1.f;
                dn += neg[b] ? -1 : 1;
#pragma unroll
                for (int j = 0; j < NPER; ++j) {
                    const float xi = xv[b][j];
                    float s, e;
                    two_sum(sh[j], sg * xi, s, e);
                    sh[j] = s;
                    sl[j] = __fadd_rn(sl[j], e);
                    // x - r as an exact pair dh + dl, its square as sq + sqe (exact)
                    // plus 2 dh dl + dl^2 (below 2^-47 of the square)
                    float dh, dl;
                    two_sum(xi, -rv[j], dh, dl);
                    const float sq = __fmul_rn(dh, dh);
                    const float sqe = __fmaf_rn(dh, dh, -sq);
                    const float cross = __fmaf_rn(__fmul_rn(2.f, dh), dl, __fmul_rn(dl, dl));
                    two_sum(qh, sg * sq, s, e);
                    qh = s;
                    ql = __fadd_rn(ql, __fadd_rn(e, sg * __fadd_rn(sqe, cross)));
                }
            }
        }
        flush();
    }
}

bool stats_full_supported(const Params &p) { return p.perm != nullptr && p.D <= 32 * kSumMaxPer; }

cudaError_t launch_stats_full(const Params &p, cudaStream_t s, int all_points, int respect_done, int num_sms) {
    {
        const size_t h1 = p.K <= p.hist_smem_k ? (size_t)p.K * 4 : 0;
        const size_t h2 = 2 * h1;
        cudaError_t e = cudaFuncSetAttribute(k_stats_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h2);
        if (e != cudaSuccess) return e;
        const int64_t blocks = (p.N + kStatsTile - 1) / kStatsTile;
        // two blocks per SM: each block adds its counts to the K global ones
        // and takes a ticket, so fewer blocks mean fewer contended atomics
        const unsigned grid = (unsigned)std::max<int64_t>(1, std::min<int64_t>(blocks, (int64_t)num_sms * 2));
        count_launch();
        k_stats_hist<<<grid, kStatsThreads, h1, s>>>(p, all_points, respect_done);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        count_launch();
        k_stats_scatter<<<grid, kStatsThreads, h2, s>>>(p, respect_done);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        const int64_t runs = (p.N + kSumRun - 1) / kSumRun;
        const unsigned sgrid = (unsigned)std::max<int64_t>(
            1, std::min<int64_t>((runs + kStatsThreads / 32 - 1) / (kStatsThreads / 32), (int64_t)num_sms * 8));
        count_launch();
        const int nper = (p.D + 31) / 32;
        if (nper <= 1) k_stats_sum<1><<<sgrid, kStatsThreads, 0, s>>>(p, respect_done);
        else if (nper <= 2) k_stats_sum<2><<<sgrid, kStatsThreads, 0, s>>>(p, respect_done);
        else if (nper <= 4) k_stats_sum<4><<<sgrid, kStatsThreads, 0, s>>>(p, respect_done);
        else k_stats_sum<kSumMaxPer><<<sgrid, kStatsThreads, 0, s>>>(p, respect_done);
        return cudaGetLastError();
    }
}

}  // namespace kp
