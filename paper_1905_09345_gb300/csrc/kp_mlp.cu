// kp_mlp.cu -- the learned group proposal's network on the 5th-generation
// tensor cores: inference, and training (forward, backward, Adam).
//
// The paper's filters (Sec. I) start from bounds that iteration 0 makes; the
// proposal is the library's layered form that predicts each point's centroid
// group so that those bounds can be seeded without a dense pass.  The network
// is a multilayer perceptron  D -> H -> H -> G  with GELU activations (the
// exact erf form), trained with softmax cross-entropy (mean over the batch)
// and Adam, FP32 master weights and bfloat16 compute weights.
//
// Every matrix product is one kernel, k_mlp_gemm:
//     C[M x N] = A[M x K] . B[N x K]^T
// with both operands bfloat16 and K-major in global memory, staged into shared
// memory by TMA (128-byte swizzle, one 64-element K slice per stage, a ring of
// stages), multiplied by tcgen05.mma (kind::f16, M = 128 rows per CTA, up to
// two N chunks of <= 256 columns) into FP32 accumulators in TMEM, and read back
// by four epilogue warps (one TMEM lane quadrant each, one row per thread)
// that apply the layer's fused epilogue:
//     GELU     bias + GELU -> bfloat16 activations (row-major and/or
//              transposed) and the FP32 derivative GELU'(z) for the backward
//              pass;
//     SOFTMAX  bias + softmax cross-entropy: the loss, and the logit gradient
//              (p - onehot(y)) / B as bfloat16 (row-major and transposed), with
//              its per-warp column sums (the bias gradient);
//     ARGMAX   bias + the first largest logit (inference);
//     MUL      the backpropagated gradient times GELU'(z) (row-major and/or
//              transposed bfloat16, per-warp column sums);
//     F32      the FP32 tile itself (split-K partial products of a weight
//              gradient, summed by the update kernel).
// The weight-gradient products contract over the batch, so the forward and
// backward epilogues also write the transposed copies those products read
// K-major; every operand stays in the layout the tensor cores take directly.
//
// Shapes are padded once: D to Dk (a multiple of 64, the K slice), the hidden
// width H to Hp (a multiple of 64) with zero weights and biases (a padded unit
// computes GELU(0) = 0 and has zero outgoing weights, so it changes nothing
// and its gradients stay zero), G to Gk (a multiple of 64) for the products
// that contract over the classes.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "kp_tc.cuh"

namespace kp {
namespace {

constexpr int kMM = 128;       // rows per tile (TMEM lanes)
constexpr int kMK = 64;        // K per stage: one 128-byte row of bfloat16
constexpr int kMThreads = 192; // warp 0 TMA, warp 1 MMA (and TMEM allocation), warps 2..5 epilogue
constexpr uint32_t kMPolls = 1u << 22;

enum Epi : int { E_GELU = 0, E_SOFTMAX = 1, E_ARGMAX = 2, E_MUL = 3, E_F32 = 4 };

struct GemmCfg {
    int M, N;          // valid output rows / columns
    int k_steps;       // K slices of 64 per CTA (split-K: blockIdx.z selects the slice range)
    int nch, bn;       // N chunks per CTA and columns per chunk (multiple of 16, <= 256)
    int tmem_cols;     // power of two >= nch * bn
    int stages;
    int mode;          // Epi
    const float *bias; // N (GELU, SOFTMAX, ARGMAX)
    uint16_t *out;     // row-major bfloat16 M x ldo (nullable)
    int ldo;
    uint16_t *outT;    // transposed bfloat16 N x ldt (nullable)
    int ldt;
    float *aux;        // FP32 M x lda: GELU'(z) (written by GELU, read by MUL; nullable in GELU)
    int lda;
    float *part;       // F32: split z at part + z * part_split, row stride ldp
    int ldp;
    int64_t part_split;
    float *colsum;     // per-warp column sums: [M / 32] x ldc (nullable)
    int ldc;
    const int32_t *y;  // SOFTMAX: class of each row
    float scale;       // SOFTMAX: 1 / batch
    double *loss;      // SOFTMAX: [0] += cross-entropy, [1] += correct predictions, [2] += rows
    int32_t *pred;     // ARGMAX
    int *err;          // KM_ETIMEOUT when a bounded wait gave up
};

__device__ __forceinline__ bool mwait(uint64_t *b, uint32_t parity, int *err) {
    for (uint32_t i = 0; i < kMPolls; ++i)
        if (mbar_try_wait(b, parity)) return true;
    atomicExch(err, (int)KM_ETIMEOUT);
    return false;
}

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
// d/dz [z Phi(z)] = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_d(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.3989422804014327f * expf(-0.5f * z * z);
}
__device__ __forceinline__ uint16_t bf16_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// 16 bfloat16 values to 32 contiguous bytes (16-byte aligned)
__device__ __forceinline__ void store_bf16x16(uint16_t *dst, const float (&v)[16]) {
    uint32_t w[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) w[i] = (uint32_t)bf16_bits(v[2 * i]) | ((uint32_t)bf16_bits(v[2 * i + 1]) << 16);
    uint4 *d = reinterpret_cast<uint4 *>(dst);
    d[0] = make_uint4(w[0], w[1], w[2], w[3]);
    d[1] = make_uint4(w[4], w[5], w[6], w[7]);
}

// sum over the 32 lanes (rows) of a warp
__device__ __forceinline__ float lane_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(kMThreads, 1)
    k_mlp_gemm(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb, GemmCfg g) {
    extern __shared__ uint8_t raw[];
    uint8_t *sm = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(raw) + 1023) & ~(uintptr_t)1023);
    const int S = g.stages;
    constexpr uint32_t a_bytes = kMM * 128;
    const uint32_t b_bytes = (uint32_t)(g.nch * g.bn) * 128u;
    const uint32_t st_bytes = a_bytes + b_bytes;
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + (size_t)S * st_bytes);
    uint64_t *full = bars, *empty = bars + S, *accb = bars + 2 * S;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 2 * S + 1);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kMM;
    const int nb = blockIdx.y * g.nch * g.bn;  // first output column of this CTA
    const int ks0 = blockIdx.z * g.k_steps;

    if (threadIdx.x == 0) {
        for (int i = 0; i < S; ++i) {
            bar_init(&full[i], 1);
            bar_init(&empty[i], 1);
        }
        bar_init(accb, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(g.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;

    if (warp == 0) {
        // ------------------------------------------------------------ TMA
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&ta) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tb) : "memory");
            int i = 0;
            for (; i < g.k_steps; ++i) {
                const int s = i % S, f = i / S;
                if (f > 0 && !mwait(&empty[s], (f - 1) & 1, g.err)) break;
                uint8_t *st = sm + (size_t)s * st_bytes;
                mbar_arrive_expect_tx(&full[s], st_bytes);
                const int kc = (ks0 + i) * kMK;
                tma_2d(st, &ta, kc, m0, &full[s]);
                for (int c = 0; c < g.nch; ++c) tma_2d(st + a_bytes + c * g.bn * 128, &tb, kc, nb + c * g.bn, &full[s]);
            }
            // every issued copy has landed before the block can exit
            for (int j = i - S < 0 ? 0 : i - S; j < i; ++j) mwait(&full[j % S], (j / S) & 1, g.err);
        }
    } else if (warp == 1) {
        // ------------------------------------------------------------ MMA
        if (lane == 0) {
            // kind::f16: F32 accumulate, BF16 A and B, both K-major, N = bn, M = 128
            const uint32_t idesc =
                (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(g.bn >> 3) << 17) | ((uint32_t)(kMM >> 4) << 24);
            for (int i = 0; i < g.k_steps; ++i) {
                const int s = i % S;
                if (!mwait(&full[s], (i / S) & 1, g.err)) break;
                tc_fence_after();
                const uint8_t *st = sm + (size_t)s * st_bytes;
#pragma unroll
                for (int j = 0; j < 4; ++j) {  // four K = 16 steps inside the 128-byte row
                    const uint64_t da = desc_sw128(smem_u32(st + j * 32));
                    for (int c = 0; c < g.nch; ++c) {
                        const uint64_t db = desc_sw128(smem_u32(st + a_bytes + c * g.bn * 128 + j * 32));
                        const uint32_t acc = (i > 0 || j > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(
                                tmem + (uint32_t)(c * g.bn)),
                            "l"(da), "l"(db), "r"(idesc), "r"(acc)
                            : "memory");
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_u32(&empty[s]))
                             : "memory");
            }
            // the accumulators are complete (and no MMA of this thread is in
            // flight) once accb completes
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_u32(accb))
                         : "memory");
            mwait(accb, 0, g.err);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------- epilogue
        const int q = warp & 3;  // TMEM lane quadrant of this warp
        const int r = q * 32 + lane;
        const int row = m0 + r;
        const bool valid = row < g.M;
        const bool ok = __all_sync(0xffffffffu, mwait(accb, 0, g.err));
        tc_fence_after();
        const uint32_t tb_ = tmem + ((uint32_t)(q * 32) << 16);
        const int TC = g.nch * g.bn;
        const int rw = (m0 + q * 32) >> 5;  // row warp (for the per-warp column sums)
        if (ok) {
            if (g.mode == E_GELU || g.mode == E_MUL || g.mode == E_F32) {
                for (int c0 = 0; c0 < TC; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16_async(tb_ + c0, v);
                    tmem_wait16(v);
                    const int n0 = nb + c0;
                    if (n0 >= g.N) break;  // warp-uniform; N is a multiple of 16
                    float a[16];
                    if (g.mode == E_GELU) {
                        float d[16];
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float z = __uint_as_float(v[j]) + g.bias[n0 + j];
                            a[j] = gelu(z);
                            d[j] = gelu_d(z);
                        }
                        if (valid) {
                            if (g.out) store_bf16x16(g.out + (size_t)row * g.ldo + n0, a);
                            if (g.aux) {
                                float4 *ap = reinterpret_cast<float4 *>(g.aux + (size_t)row * g.lda + n0);
#pragma unroll
                                for (int j = 0; j < 4; ++j) ap[j] = make_float4(d[4 * j], d[4 * j + 1], d[4 * j + 2], d[4 * j + 3]);
                            }
                        }
                    } else if (g.mode == E_MUL) {
                        if (valid) {
                            const float4 *ap = reinterpret_cast<const float4 *>(g.aux + (size_t)row * g.lda + n0);
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                const float4 dd = ap[j];
                                a[4 * j] = __uint_as_float(v[4 * j]) * dd.x;
                                a[4 * j + 1] = __uint_as_float(v[4 * j + 1]) * dd.y;
                                a[4 * j + 2] = __uint_as_float(v[4 * j + 2]) * dd.z;
                                a[4 * j + 3] = __uint_as_float(v[4 * j + 3]) * dd.w;
                            }
                            if (g.out) store_bf16x16(g.out + (size_t)row * g.ldo + n0, a);
                        } else {
#pragma unroll
                            for (int j = 0; j < 16; ++j) a[j] = 0.f;
                        }
                        if (g.colsum) {
#pragma unroll
                            for (int j = 0; j < 16; ++j) {
                                const float cs = lane_sum(a[j]);
                                if (lane == 0) g.colsum[(size_t)rw * g.ldc + n0 + j] = cs;
                            }
                        }
                    } else {  // E_F32
                        if (valid) {
                            float4 *pp = reinterpret_cast<float4 *>(g.part + (size_t)blockIdx.z * g.part_split +
                                                                    (size_t)row * g.ldp + n0);
#pragma unroll
                            for (int j = 0; j < 4; ++j)
                                pp[j] = make_float4(__uint_as_float(v[4 * j]), __uint_as_float(v[4 * j + 1]),
                                                    __uint_as_float(v[4 * j + 2]), __uint_as_float(v[4 * j + 3]));
                        }
                        continue;
                    }
                    if (g.outT && valid) {
#pragma unroll
                        for (int j = 0; j < 16; ++j) g.outT[(size_t)(n0 + j) * g.ldt + row] = bf16_bits(a[j]);
                    }
                }
            } else if (g.mode == E_ARGMAX) {
                float best = -INFINITY;
                int bi = 0;
                for (int c0 = 0; c0 < TC; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16_async(tb_ + c0, v);
                    tmem_wait16(v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = c0 + j;  // one N tile: nb == 0
                        if (n < g.N) {
                            const float l = __uint_as_float(v[j]) + g.bias[n];
                            if (l > best) {
                                best = l;
                                bi = n;
                            }
                        }
                    }
                }
                if (valid) g.pred[row] = bi;
            } else {  // E_SOFTMAX (one N tile: nb == 0)
                float mx = -INFINITY;
                for (int c0 = 0; c0 < TC; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16_async(tb_ + c0, v);
                    tmem_wait16(v);
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c0 + j < g.N) mx = fmaxf(mx, __uint_as_float(v[j]) + g.bias[c0 + j]);
                }
                const int y = valid ? g.y[row] : -1;
                float s = 0.f, ly = 0.f, best = -INFINITY;
                int bi = 0;
                for (int c0 = 0; c0 < TC; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16_async(tb_ + c0, v);
                    tmem_wait16(v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = c0 + j;
                        if (n < g.N) {
                            const float l = __uint_as_float(v[j]) + g.bias[n];
                            s += expf(l - mx);
                            if (n == y) ly = l;
                            if (l > best) {
                                best = l;
                                bi = n;
                            }
                        }
                    }
                }
                const float inv_s = 1.0f / s;
                for (int c0 = 0; c0 < TC; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16_async(tb_ + c0, v);
                    tmem_wait16(v);
                    float d[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int n = c0 + j;
                        const float l = __uint_as_float(v[j]) + (n < g.N ? g.bias[n] : 0.f);
                        d[j] = (valid && n < g.N) ? (expf(l - mx) * inv_s - (n == y ? 1.f : 0.f)) * g.scale : 0.f;
                    }
                    if (valid) {
                        store_bf16x16(g.out + (size_t)row * g.ldo + c0, d);
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (c0 + j < g.N) g.outT[(size_t)(c0 + j) * g.ldt + row] = bf16_bits(d[j]);
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const float cs = lane_sum(d[j]);
                        if (lane == 0 && c0 + j < g.N) g.colsum[(size_t)rw * g.ldc + c0 + j] = cs;
                    }
                }
                const float ce = valid ? (logf(s) + mx - ly) : 0.f;
                const float hit = (valid && bi == y) ? 1.f : 0.f;
                const float ces = lane_sum(ce), hits = lane_sum(hit), rows = lane_sum(valid ? 1.f : 0.f);
                if (lane == 0) {
                    atomicAdd(&g.loss[0], (double)ces);
                    atomicAdd(&g.loss[1], (double)hits);
                    atomicAdd(&g.loss[2], (double)rows);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.tmem_cols)
                     : "memory");
    }
}

// ---------------------------------------------------------------------------
// data movement and the update
// ---------------------------------------------------------------------------
// SplitMix64 (Steele, Lea and Flood, OOPSLA 2014): a counter-based generator
__device__ __host__ __forceinline__ uint64_t splitmix64(uint64_t z) {
    z += 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

struct MlpState {
    int32_t t;      // Adam steps taken
    int32_t pad;
    double loss[3]; // cross-entropy sum, correct predictions, rows (since the last read)
};

// Batch of B rows: random rows of the training set (with replacement, a
// counter-based draw per (seed, step, row)), or rows 0..B-1 when seed is
// ~0ull.  Writes Xb (B x Dk bfloat16, zero padding), XbT (Dn x B, rows >= D
// zero) and the classes yb (labels mapped to contiguous groups when K > 0).
__global__ void k_mlp_gather(const float *X, int64_t N, int D, const int32_t *labels, int K, int G, int B, int Dk,
                             int Dn, uint64_t seed, const MlpState *st, uint16_t *Xb, uint16_t *XbT, int32_t *yb) {
    const int i = blockIdx.x;  // one block per row
    if (i >= B) return;
    int64_t src = i;
    if (seed != ~0ull) src = (int64_t)(splitmix64(seed ^ splitmix64(((uint64_t)st->t << 32) | (uint32_t)i)) % (uint64_t)N);
    for (int d = threadIdx.x; d < Dk; d += blockDim.x) {
        const float v = d < D ? X[src * D + d] : 0.f;
        const uint16_t b = bf16_bits(v);
        Xb[(size_t)i * Dk + d] = b;
        if (d < Dn) XbT[(size_t)d * B + i] = b;
    }
    if (threadIdx.x == 0) {
        int y = labels[src];
        if (K > 0) y = (int)(((int64_t)y * G) / K);
        yb[i] = (y >= 0 && y < G) ? y : 0;
    }
}

// X (rows r0.., m of them) -> bfloat16 m x Dk, zero padding
__global__ void k_mlp_cast_x(const float *X, int64_t m, int D, int Dk, uint16_t *Xc) {
    const int64_t total = m * Dk;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = e / Dk;
        const int d = (int)(e - r * Dk);
        Xc[e] = bf16_bits(d < D ? X[r * D + d] : 0.f);
    }
}

struct MlpDims {
    int D, H, G;        // logical sizes
    int Dk, Dn, Hp, Gk; // padded
    int64_t oW1, ob1, oW2, ob2, oW3, ob3, P;  // offsets of W1 b1 W2 b2 W3 b3 in the parameter vector
};

struct ApplyArgs {
    int mode;           // 0: gradient out, 1: Adam step, 2: copy the masters to the compute weights
    float *master, *m1, *m2;
    const float *pW1, *pW2, *pW3;  // split-K partials
    int s1, s2, s3;
    int64_t ps1, ps2, ps3;         // floats between splits
    const float *cs1, *cs2, *cs3;  // per-warp column sums
    int nrw;                       // row warps (B / 32)
    float *grad;                   // mode 0
    float lr, b1, b2, eps;
    MlpState *st;
    uint16_t *W1b, *W2b, *W2T, *W3b, *W3T;
    float *b1p, *b2p, *b3p;
};

// One thread per parameter: its gradient (sum of the split-K partials or of
// the per-warp column sums), then the requested action; the compute copies
// (bfloat16 weights, padded FP32 biases) are rewritten from the masters.
__global__ void k_mlp_apply(MlpDims d, ApplyArgs a) {
    const int t1 = a.mode == 1 ? a.st->t + 1 : 0;
    const float bc1 = a.mode == 1 ? 1.0f - powf(a.b1, (float)t1) : 1.f;
    const float bc2 = a.mode == 1 ? 1.0f - powf(a.b2, (float)t1) : 1.f;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += (int64_t)gridDim.x * blockDim.x) {
        int seg;
        int64_t o;
        if (i < d.ob1) { seg = 0; o = i - d.oW1; }
        else if (i < d.oW2) { seg = 1; o = i - d.ob1; }
        else if (i < d.ob2) { seg = 2; o = i - d.oW2; }
        else if (i < d.oW3) { seg = 3; o = i - d.ob2; }
        else if (i < d.ob3) { seg = 4; o = i - d.oW3; }
        else { seg = 5; o = i - d.ob3; }
        int r = 0, c = 0;  // (row, column) of a weight
        if (seg == 0) { r = (int)(o / d.D); c = (int)(o % d.D); }
        else if (seg == 2) { r = (int)(o / d.H); c = (int)(o % d.H); }
        else if (seg == 4) { r = (int)(o / d.H); c = (int)(o % d.H); }
        if (a.mode != 2) {
            float gsum = 0.f;
            switch (seg) {
                case 0: for (int z = 0; z < a.s1; ++z) gsum += a.pW1[z * a.ps1 + (int64_t)r * d.Dn + c]; break;
                case 1: for (int w = 0; w < a.nrw; ++w) gsum += a.cs1[(int64_t)w * d.Hp + o]; break;
                case 2: for (int z = 0; z < a.s2; ++z) gsum += a.pW2[z * a.ps2 + (int64_t)r * d.Hp + c]; break;
                case 3: for (int w = 0; w < a.nrw; ++w) gsum += a.cs2[(int64_t)w * d.Hp + o]; break;
                case 4: for (int z = 0; z < a.s3; ++z) gsum += a.pW3[z * a.ps3 + (int64_t)r * d.Hp + c]; break;
                default: for (int w = 0; w < a.nrw; ++w) gsum += a.cs3[(int64_t)w * d.G + o]; break;
            }
            if (a.mode == 0) {
                a.grad[i] = gsum;
                continue;
            }
            // Adam (Kingma and Ba): bias-corrected first and second moments
            const float m = a.b1 * a.m1[i] + (1.0f - a.b1) * gsum;
            const float v = a.b2 * a.m2[i] + (1.0f - a.b2) * gsum * gsum;
            a.m1[i] = m;
            a.m2[i] = v;
            a.master[i] -= a.lr * (m / bc1) / (sqrtf(v / bc2) + a.eps);
        }
        const float w = a.master[i];
        const uint16_t wb = bf16_bits(w);
        switch (seg) {
            case 0: a.W1b[(size_t)r * d.Dk + c] = wb; break;
            case 1: a.b1p[o] = w; break;
            case 2: a.W2b[(size_t)r * d.Hp + c] = wb; a.W2T[(size_t)c * d.Hp + r] = wb; break;
            case 3: a.b2p[o] = w; break;
            case 4: a.W3b[(size_t)r * d.Hp + c] = wb; a.W3T[(size_t)c * d.Gk + r] = wb; break;
            default: a.b3p[o] = w; break;
        }
    }
}

__global__ void k_mlp_step_end(MlpState *st) { st->t += 1; }

// Xavier-uniform weights U(-a, a), a = sqrt(6 / (fan_in + fan_out)), zero
// biases, from the counter-based generator (seed, parameter index)
__global__ void k_mlp_init(MlpDims d, float *master, uint64_t seed) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < d.P; i += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f;
        if (i < d.ob1) a = sqrtf(6.0f / (float)(d.D + d.H));
        else if (i >= d.oW2 && i < d.ob2) a = sqrtf(6.0f / (float)(2 * d.H));
        else if (i >= d.oW3 && i < d.ob3) a = sqrtf(6.0f / (float)(d.H + d.G));
        const float u = (float)(splitmix64(seed ^ splitmix64((uint64_t)i)) >> 40) * (1.0f / 16777216.0f);
        master[i] = a * (2.0f * u - 1.0f);
    }
}

int round_up(int x, int m) { return (x + m - 1) / m * m; }
int pow2_at_least(int x) {
    int p = 32;
    while (p < x) p <<= 1;
    return p;
}

}  // namespace
}  // namespace kp

using namespace kp;

// ---------------------------------------------------------------------------
// the network object
// ---------------------------------------------------------------------------
struct kmeans_mlp {
    int dev = 0, num_sms = 0;
    size_t smem_optin = 0;
    cudaStream_t stream = nullptr;
    MlpDims d{};
    int nch3 = 1, bn3 = 16;  // layer-3 N chunks
    int bnH = 64;            // columns per CTA of the hidden-layer products
    float *master = nullptr, *m1 = nullptr, *m2 = nullptr;
    uint16_t *W1b = nullptr, *W2b = nullptr, *W2T = nullptr, *W3b = nullptr, *W3T = nullptr;
    float *b1p = nullptr, *b2p = nullptr, *b3p = nullptr;
    MlpState *st = nullptr;
    int *err = nullptr;
    // training buffers (batch B)
    int B = 0;
    uint16_t *Xb = nullptr, *XbT = nullptr, *A1 = nullptr, *A1T = nullptr, *A2 = nullptr, *A2T = nullptr,
             *dZ3 = nullptr, *dZ3T = nullptr, *dZ2 = nullptr, *dZ2T = nullptr, *dZ1T = nullptr;
    float *G1 = nullptr, *G2 = nullptr, *pW1 = nullptr, *pW2 = nullptr, *pW3 = nullptr, *cs1 = nullptr,
          *cs2 = nullptr, *cs3 = nullptr;
    int32_t *yb = nullptr;
    int s1 = 1, s2 = 1, s3 = 1;
    std::vector<void *> batch_allocs;
    // inference buffers (chunk of Mc rows)
    int64_t Mc = 0;
    uint16_t *Xc = nullptr, *A1c = nullptr, *A2c = nullptr;
    std::vector<void *> allocs;
    char errmsg[512] = "";
};

namespace kp {
namespace {

thread_local char g_mlp_err[512] = "";

int mlp_fail(kmeans_mlp *m, int code, const char *fmt, ...) {
    char *buf = m ? m->errmsg : g_mlp_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, 512, fmt, ap);
    va_end(ap);
    if (!m) set_thread_error(buf);
    return code;
}

#define MLP_CUDA(m, call)                                                                                   \
    do {                                                                                                    \
        cudaError_t e_ = (call);                                                                            \
        if (e_ != cudaSuccess)                                                                              \
            return mlp_fail((m), e_ == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA, "%s: %s (%s:%d)", #call, \
                            cudaGetErrorString(e_), __FILE__, __LINE__);                                    \
    } while (0)

template <class T>
cudaError_t mlp_alloc(kmeans_mlp *m, T **p, size_t n, std::vector<void *> &list) {
    void *v = nullptr;
    cudaError_t e = pool_alloc(m->dev, &v, std::max<size_t>(n, 1) * sizeof(T), m->stream);
    if (e != cudaSuccess) return e;
    list.push_back(v);
    *p = static_cast<T *>(v);
    return cudaMemsetAsync(v, 0, std::max<size_t>(n, 1) * sizeof(T), m->stream);
}

// 2D bfloat16 tensor map: `rows` rows of `cols` elements (row stride `ld`
// elements), boxes of 64 x box_rows with 128-byte swizzle
int make_map(kmeans_mlp *m, CUtensorMap *map, const uint16_t *base, int64_t rows, int64_t cols, int64_t ld,
             int box_rows) {
    auto enc = encoder();
    if (!enc) return mlp_fail(m, KM_ECUDA, "cuTensorMapEncodeTiled is not available");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
    cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1u, 1u};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<uint16_t *>(base), dims, strides, box, es,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return mlp_fail(m, KM_ECUDA, "tensor map encoding failed (%d)", (int)r);
    return KM_OK;
}

// One product C = A . B^T.  A: rows x K (row stride lda_el), B: N rows x K.
// K must be a multiple of 64 (splits * 64 * k_steps).
struct GemmSpec {
    const uint16_t *A;
    int64_t a_rows, a_ld;
    const uint16_t *Bm;
    int64_t b_rows, b_ld;
    int64_t K;       // contraction length (multiple of 64 * splits)
    int M, N;        // valid output extent
    int nch, bn;     // columns per CTA: nch * bn
    int ntiles;      // CTAs along N
    int splits;
};

int launch_gemm(kmeans_mlp *m, const GemmSpec &sp, GemmCfg g, cudaStream_t s) {
    CUtensorMap ta, tb;
    int rc;
    if ((rc = make_map(m, &ta, sp.A, sp.a_rows, sp.K, sp.a_ld, kMM))) return rc;
    if ((rc = make_map(m, &tb, sp.Bm, sp.b_rows, sp.K, sp.b_ld, sp.bn))) return rc;
    g.M = sp.M;
    g.N = sp.N;
    g.nch = sp.nch;
    g.bn = sp.bn;
    g.k_steps = (int)(sp.K / kMK / sp.splits);
    g.tmem_cols = pow2_at_least(sp.nch * sp.bn);
    g.err = m->err;
    const size_t st_bytes = (size_t)kMM * 128 + (size_t)sp.nch * sp.bn * 128;
    int stages = 4;
    while (stages > 2 && 1024 + stages * st_bytes + 256 > m->smem_optin) --stages;
    g.stages = stages;
    size_t smem = 1024 + stages * st_bytes + 256;
    // CTAs resident on one SM must not ask for more than its 512 TMEM columns
    const size_t sm_smem = 233472;  // shared memory per SM
    while ((sm_smem / smem) * (size_t)g.tmem_cols > 512) smem += 4096;
    if (smem > m->smem_optin) return mlp_fail(m, KM_EINVAL, "product tile does not fit in shared memory");
    cudaError_t e = cudaFuncSetAttribute(k_mlp_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return mlp_fail(m, KM_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    dim3 grid((unsigned)((sp.M + kMM - 1) / kMM), (unsigned)sp.ntiles, (unsigned)sp.splits);
    count_launch();
    k_mlp_gemm<<<grid, kMThreads, smem, s>>>(ta, tb, g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(m, KM_ECUDA, "k_mlp_gemm launch: %s", cudaGetErrorString(e));
    return KM_OK;
}

GemmCfg cfg0(int mode) {
    GemmCfg g;
    memset(&g, 0, sizeof(g));
    g.mode = mode;
    return g;
}

// columns per CTA for a hidden-width output: all of them when M is large
// (one pass over A), else split in two for more CTAs
void hidden_tiles(const kmeans_mlp *m, int M, int &bn, int &ntiles) {
    const int Hp = m->d.Hp;
    if (Hp > 128 && (M + kMM - 1) / kMM < m->num_sms) {
        bn = Hp / 2;
        ntiles = 2;
    } else {
        bn = Hp;
        ntiles = 1;
    }
}

int alloc_batch(kmeans_mlp *m, int B) {
    if (m->B == B) return KM_OK;
    for (void *p : m->batch_allocs) cudaFreeAsync(p, m->stream);
    m->batch_allocs.clear();
    m->B = 0;
    const MlpDims &d = m->d;
    auto &L = m->batch_allocs;
    // split-K of the weight gradients: at least 4 slices of 64 per CTA, about
    // one wave of CTAs
    auto splits_for = [&](int mrows) {
        const int tiles = (mrows + kMM - 1) / kMM;
        int s = 1;
        while (s * 2 * tiles <= m->num_sms && (B / 64) % (s * 2) == 0 && B / 64 / (s * 2) >= 4) s *= 2;
        return s;
    };
    m->s1 = splits_for(d.Hp);
    m->s2 = splits_for(d.Hp);
    m->s3 = splits_for(d.G);
    MLP_CUDA(m, mlp_alloc(m, &m->Xb, (size_t)B * d.Dk, L));
    MLP_CUDA(m, mlp_alloc(m, &m->XbT, (size_t)d.Dn * B, L));
    MLP_CUDA(m, mlp_alloc(m, &m->A1, (size_t)B * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->A1T, (size_t)d.Hp * B, L));
    MLP_CUDA(m, mlp_alloc(m, &m->A2, (size_t)B * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->A2T, (size_t)d.Hp * B, L));
    MLP_CUDA(m, mlp_alloc(m, &m->dZ3, (size_t)B * d.Gk, L));
    MLP_CUDA(m, mlp_alloc(m, &m->dZ3T, (size_t)d.G * B, L));
    MLP_CUDA(m, mlp_alloc(m, &m->dZ2, (size_t)B * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->dZ2T, (size_t)d.Hp * B, L));
    MLP_CUDA(m, mlp_alloc(m, &m->dZ1T, (size_t)d.Hp * B, L));
    MLP_CUDA(m, mlp_alloc(m, &m->G1, (size_t)B * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->G2, (size_t)B * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->pW1, (size_t)m->s1 * d.Hp * d.Dn, L));
    MLP_CUDA(m, mlp_alloc(m, &m->pW2, (size_t)m->s2 * d.Hp * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->pW3, (size_t)m->s3 * d.G * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->cs1, (size_t)(B / 32) * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->cs2, (size_t)(B / 32) * d.Hp, L));
    MLP_CUDA(m, mlp_alloc(m, &m->cs3, (size_t)(B / 32) * d.G, L));
    MLP_CUDA(m, mlp_alloc(m, &m->yb, (size_t)B, L));
    m->B = B;
    return KM_OK;
}

// forward + backward of one batch already gathered into Xb / XbT / yb;
// leaves the split-K partials and the column sums for k_mlp_apply
int enqueue_fwd_bwd(kmeans_mlp *m, cudaStream_t s) {
    const MlpDims &d = m->d;
    const int B = m->B;
    int rc, bnh, nth;
    hidden_tiles(m, B, bnh, nth);
    // layer 1: A1 = GELU(Xb W1^T + b1), with A1^T and GELU'(z1)
    GemmCfg g = cfg0(E_GELU);
    g.bias = m->b1p; g.out = m->A1; g.ldo = d.Hp; g.outT = m->A1T; g.ldt = B; g.aux = m->G1; g.lda = d.Hp;
    if ((rc = launch_gemm(m, {m->Xb, B, d.Dk, m->W1b, d.Hp, d.Dk, d.Dk, B, d.Hp, 1, bnh, nth, 1}, g, s))) return rc;
    // layer 2
    g = cfg0(E_GELU);
    g.bias = m->b2p; g.out = m->A2; g.ldo = d.Hp; g.outT = m->A2T; g.ldt = B; g.aux = m->G2; g.lda = d.Hp;
    if ((rc = launch_gemm(m, {m->A1, B, d.Hp, m->W2b, d.Hp, d.Hp, d.Hp, B, d.Hp, 1, bnh, nth, 1}, g, s))) return rc;
    // layer 3 + softmax cross-entropy: dZ3 = (softmax - onehot) / B
    g = cfg0(E_SOFTMAX);
    g.bias = m->b3p; g.out = m->dZ3; g.ldo = d.Gk; g.outT = m->dZ3T; g.ldt = B; g.colsum = m->cs3; g.ldc = d.G;
    g.y = m->yb; g.scale = 1.0f / (float)B; g.loss = m->st->loss;
    if ((rc = launch_gemm(m, {m->A2, B, d.Hp, m->W3b, d.G, d.Hp, d.Hp, B, d.G, m->nch3, m->bn3, 1, 1}, g, s)))
        return rc;
    // dZ2 = (dZ3 W3) * GELU'(z2)
    g = cfg0(E_MUL);
    g.aux = m->G2; g.lda = d.Hp; g.out = m->dZ2; g.ldo = d.Hp; g.outT = m->dZ2T; g.ldt = B; g.colsum = m->cs2;
    g.ldc = d.Hp;
    if ((rc = launch_gemm(m, {m->dZ3, B, d.Gk, m->W3T, d.Hp, d.Gk, d.Gk, B, d.Hp, 1, bnh, nth, 1}, g, s))) return rc;
    // dZ1 = (dZ2 W2) * GELU'(z1)
    g = cfg0(E_MUL);
    g.aux = m->G1; g.lda = d.Hp; g.outT = m->dZ1T; g.ldt = B; g.colsum = m->cs1; g.ldc = d.Hp;
    if ((rc = launch_gemm(m, {m->dZ2, B, d.Hp, m->W2T, d.Hp, d.Hp, d.Hp, B, d.Hp, 1, bnh, nth, 1}, g, s))) return rc;
    // weight gradients, contracted over the batch: dW3 = dZ3^T A2, dW2 = dZ2^T A1, dW1 = dZ1^T X
    g = cfg0(E_F32);
    g.part = m->pW3; g.ldp = d.Hp; g.part_split = (int64_t)d.G * d.Hp;
    if ((rc = launch_gemm(m, {m->dZ3T, d.G, B, m->A2T, d.Hp, B, B, d.G, d.Hp, 1, d.Hp, 1, m->s3}, g, s))) return rc;
    g = cfg0(E_F32);
    g.part = m->pW2; g.ldp = d.Hp; g.part_split = (int64_t)d.Hp * d.Hp;
    if ((rc = launch_gemm(m, {m->dZ2T, d.Hp, B, m->A1T, d.Hp, B, B, d.Hp, d.Hp, 1, d.Hp, 1, m->s2}, g, s))) return rc;
    g = cfg0(E_F32);
    g.part = m->pW1; g.ldp = d.Dn; g.part_split = (int64_t)d.Hp * d.Dn;
    if ((rc = launch_gemm(m, {m->dZ1T, d.Hp, B, m->XbT, d.Dn, B, B, d.Hp, d.Dn, 1, d.Dn, 1, m->s1}, g, s))) return rc;
    return KM_OK;
}

ApplyArgs apply_args(kmeans_mlp *m, int mode) {
    ApplyArgs a;
    memset(&a, 0, sizeof(a));
    const MlpDims &d = m->d;
    a.mode = mode;
    a.master = m->master; a.m1 = m->m1; a.m2 = m->m2;
    a.pW1 = m->pW1; a.pW2 = m->pW2; a.pW3 = m->pW3;
    a.s1 = m->s1; a.s2 = m->s2; a.s3 = m->s3;
    a.ps1 = (int64_t)d.Hp * d.Dn; a.ps2 = (int64_t)d.Hp * d.Hp; a.ps3 = (int64_t)d.G * d.Hp;
    a.cs1 = m->cs1; a.cs2 = m->cs2; a.cs3 = m->cs3;
    a.nrw = m->B / 32;
    a.st = m->st;
    a.W1b = m->W1b; a.W2b = m->W2b; a.W2T = m->W2T; a.W3b = m->W3b; a.W3T = m->W3T;
    a.b1p = m->b1p; a.b2p = m->b2p; a.b3p = m->b3p;
    a.b1 = 0.9f; a.b2 = 0.999f; a.eps = 1e-8f;
    return a;
}

int launch_apply(kmeans_mlp *m, const ApplyArgs &a, cudaStream_t s) {
    const int64_t blocks = std::min<int64_t>((m->d.P + 255) / 256, (int64_t)m->num_sms * 8);
    count_launch();
    k_mlp_apply<<<(unsigned)blocks, 256, 0, s>>>(m->d, a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return mlp_fail(m, KM_ECUDA, "k_mlp_apply launch: %s", cudaGetErrorString(e));
    return KM_OK;
}

int check_err(kmeans_mlp *m) {
    int h = 0;
    MLP_CUDA(m, cudaMemcpyAsync(&h, m->err, 4, cudaMemcpyDeviceToHost, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    if (h) return mlp_fail(m, KM_ETIMEOUT, "a bounded wait in a tensor-core product gave up");
    return KM_OK;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DevGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// inference buffers for chunks of up to 2^17 rows (made once, before any
// capture of the inference launches)
int mlp_prepare(kmeans_mlp *m, int64_t N) {
    if (m->Mc) return KM_OK;
    const MlpDims &d = m->d;
    int64_t mc = std::min<int64_t>(std::max<int64_t>(N, 1), (int64_t)1 << 17);
    mc = (mc + kMM - 1) / kMM * kMM;
    MLP_CUDA(m, mlp_alloc(m, &m->Xc, (size_t)mc * d.Dk, m->allocs));
    MLP_CUDA(m, mlp_alloc(m, &m->A1c, (size_t)mc * d.Hp, m->allocs));
    MLP_CUDA(m, mlp_alloc(m, &m->A2c, (size_t)mc * d.Hp, m->allocs));
    m->Mc = mc;
    return KM_OK;
}

// pred[n] = the class with the largest logit (first maximum), on stream s
// (used by the context's seeded iteration 0 and by kmeans_mlp_predict_net)
int mlp_predict_enqueue(kmeans_mlp *m, const float *X, int64_t N, int32_t *pred, cudaStream_t s) {
    const MlpDims &d = m->d;
    int rc;
    if ((rc = mlp_prepare(m, N))) return rc;
    for (int64_t r0 = 0; r0 < N; r0 += m->Mc) {
        const int rows = (int)std::min<int64_t>(m->Mc, N - r0);
        count_launch();
        k_mlp_cast_x<<<(unsigned)std::min<int64_t>(((int64_t)rows * d.Dk + 255) / 256, (int64_t)m->num_sms * 8), 256,
                       0, s>>>(X + r0 * d.D, rows, d.D, d.Dk, m->Xc);
        MLP_CUDA(m, cudaGetLastError());
        GemmCfg g = cfg0(E_GELU);
        g.bias = m->b1p; g.out = m->A1c; g.ldo = d.Hp;
        if ((rc = launch_gemm(m, {m->Xc, m->Mc, d.Dk, m->W1b, d.Hp, d.Dk, d.Dk, rows, d.Hp, 1, d.Hp, 1, 1}, g, s)))
            return rc;
        g = cfg0(E_GELU);
        g.bias = m->b2p; g.out = m->A2c; g.ldo = d.Hp;
        if ((rc = launch_gemm(m, {m->A1c, m->Mc, d.Hp, m->W2b, d.Hp, d.Hp, d.Hp, rows, d.Hp, 1, d.Hp, 1, 1}, g, s)))
            return rc;
        g = cfg0(E_ARGMAX);
        g.bias = m->b3p; g.pred = pred + r0;
        if ((rc = launch_gemm(m, {m->A2c, m->Mc, d.Hp, m->W3b, d.G, d.Hp, d.Hp, rows, d.G, m->nch3, m->bn3, 1, 1},
                              g, s)))
            return rc;
    }
    return KM_OK;
}

int mlp_error_flag(kmeans_mlp *m) { return check_err(m); }
const char *mlp_message(const kmeans_mlp *m) { return m->errmsg; }

}  // namespace kp

extern "C" {

KM_API int kmeans_mlp_create(kmeans_mlp **out, int32_t D, int32_t hidden, int32_t classes, uint64_t seed,
                             void *stream) {
    if (!out) return mlp_fail(nullptr, KM_EINVAL, "out is NULL");
    *out = nullptr;
    if (D < 1 || D > 256) return mlp_fail(nullptr, KM_EINVAL, "D out of range [1, 256]");
    if (hidden < 1 || hidden > 256) return mlp_fail(nullptr, KM_EINVAL, "hidden out of range [1, 256]");
    if (classes < 1 || classes > 512) return mlp_fail(nullptr, KM_EINVAL, "classes out of range [1, 512]");
    kmeans_mlp *m = new (std::nothrow) kmeans_mlp();
    if (!m) return mlp_fail(nullptr, KM_ENOMEM, "host allocation failed");
    struct Guard {
        kmeans_mlp *&m;
        bool keep = false;
        ~Guard() {
            if (!keep && m) kmeans_mlp_destroy(m);
        }
    } guard{m};
    if (cudaGetDevice(&m->dev) != cudaSuccess) return mlp_fail(nullptr, KM_ECUDA, "cudaGetDevice failed");
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, m->dev) != cudaSuccess)
        return mlp_fail(nullptr, KM_ECUDA, "cudaDeviceGetAttribute failed");
    m->num_sms = v;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->dev) != cudaSuccess)
        return mlp_fail(nullptr, KM_ECUDA, "cudaDeviceGetAttribute failed");
    m->smem_optin = (size_t)v;
    m->stream = static_cast<cudaStream_t>(stream);
    MlpDims &d = m->d;
    d.D = D;
    d.H = hidden;
    d.G = classes;
    d.Dk = round_up(D, 64);
    d.Dn = round_up(D, 16);
    d.Hp = round_up(hidden, 64);
    d.Gk = round_up(classes, 64);
    d.oW1 = 0;
    d.ob1 = d.oW1 + (int64_t)hidden * D;
    d.oW2 = d.ob1 + hidden;
    d.ob2 = d.oW2 + (int64_t)hidden * hidden;
    d.oW3 = d.ob2 + hidden;
    d.ob3 = d.oW3 + (int64_t)classes * hidden;
    d.P = d.ob3 + classes;
    m->nch3 = (classes + 255) / 256;
    m->bn3 = round_up((classes + m->nch3 - 1) / m->nch3, 16);
    int rc;
    auto fail_cuda = [&](cudaError_t e) {
        return mlp_fail(nullptr, e == cudaErrorMemoryAllocation ? KM_ENOMEM : KM_ECUDA, "%s", cudaGetErrorString(e));
    };
    cudaError_t e;
#define MC(call) \
    if ((e = (call)) != cudaSuccess) return fail_cuda(e)
    MC(mlp_alloc(m, &m->master, (size_t)d.P, m->allocs));
    MC(mlp_alloc(m, &m->m1, (size_t)d.P, m->allocs));
    MC(mlp_alloc(m, &m->m2, (size_t)d.P, m->allocs));
    MC(mlp_alloc(m, &m->W1b, (size_t)d.Hp * d.Dk, m->allocs));
    MC(mlp_alloc(m, &m->W2b, (size_t)d.Hp * d.Hp, m->allocs));
    MC(mlp_alloc(m, &m->W2T, (size_t)d.Hp * d.Hp, m->allocs));
    MC(mlp_alloc(m, &m->W3b, (size_t)classes * d.Hp, m->allocs));
    MC(mlp_alloc(m, &m->W3T, (size_t)d.Hp * d.Gk, m->allocs));
    MC(mlp_alloc(m, &m->b1p, (size_t)d.Hp, m->allocs));
    MC(mlp_alloc(m, &m->b2p, (size_t)d.Hp, m->allocs));
    MC(mlp_alloc(m, &m->b3p, (size_t)classes, m->allocs));
    MC(mlp_alloc(m, &m->st, 1, m->allocs));
    MC(mlp_alloc(m, &m->err, 1, m->allocs));
    count_launch();
    k_mlp_init<<<(unsigned)std::min<int64_t>((d.P + 255) / 256, (int64_t)m->num_sms * 8), 256, 0, m->stream>>>(
        d, m->master, seed);
    MC(cudaGetLastError());
#undef MC
    ApplyArgs a = apply_args(m, 2);
    if ((rc = launch_apply(m, a, m->stream))) return mlp_fail(nullptr, rc, "%s", m->errmsg);
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return mlp_fail(nullptr, KM_ECUDA, "initialisation failed");
    guard.keep = true;
    *out = m;
    return KM_OK;
}

KM_API int kmeans_mlp_set_params(kmeans_mlp *m, const float *W1, const float *b1, const float *W2, const float *b2,
                                 const float *W3, const float *b3) {
    if (!m) return mlp_fail(nullptr, KM_EINVAL, "network is NULL");
    if (!W1 || !b1 || !W2 || !b2 || !W3 || !b3) return mlp_fail(m, KM_EINVAL, "a parameter pointer is NULL");
    DevGuard dg(m->dev);
    const MlpDims &d = m->d;
    const float *src[6] = {W1, b1, W2, b2, W3, b3};
    const int64_t off[7] = {d.oW1, d.ob1, d.oW2, d.ob2, d.oW3, d.ob3, d.P};
    for (int i = 0; i < 6; ++i)
        MLP_CUDA(m, cudaMemcpyAsync(m->master + off[i], src[i], (size_t)(off[i + 1] - off[i]) * 4, cudaMemcpyDefault,
                                    m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->m1, 0, (size_t)d.P * 4, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->m2, 0, (size_t)d.P * 4, m->stream));
    MLP_CUDA(m, cudaMemsetAsync(m->st, 0, sizeof(MlpState), m->stream));
    int rc;
    if ((rc = launch_apply(m, apply_args(m, 2), m->stream))) return rc;
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return KM_OK;
}

KM_API int kmeans_mlp_get_params(kmeans_mlp *m, float *W1, float *b1, float *W2, float *b2, float *W3, float *b3) {
    if (!m) return mlp_fail(nullptr, KM_EINVAL, "network is NULL");
    DevGuard dg(m->dev);
    const MlpDims &d = m->d;
    float *dst[6] = {W1, b1, W2, b2, W3, b3};
    const int64_t off[7] = {d.oW1, d.ob1, d.oW2, d.ob2, d.oW3, d.ob3, d.P};
    for (int i = 0; i < 6; ++i)
        if (dst[i])
            MLP_CUDA(m, cudaMemcpyAsync(dst[i], m->master + off[i], (size_t)(off[i + 1] - off[i]) * 4,
                                        cudaMemcpyDefault, m->stream));
    MLP_CUDA(m, cudaStreamSynchronize(m->stream));
    return KM_OK;
}

KM_API int kmeans_mlp_gradient(kmeans_mlp *m, const float *X, const int32_t *y, int32_t B, double *loss,
                               float *grad) {
    if (!m) return mlp_fail(nullptr, KM_EINVAL, "network is NULL");
    if (!X || !y || !grad) return mlp_fail(m, KM_EINVAL, "a pointer argument is NULL");
    if (B < 128 || B % 128 != 0 || B > (1 << 20)) return mlp_fail(m, KM_EINVAL, "B must be a multiple of 128 in [128, 2^20]");
    if (!dev_ptr(X) || !dev_ptr(y) || !dev_ptr(grad)) return mlp_fail(m, KM_EINVAL, "X, y and grad must be device memory");
    DevGuard dg(m->dev);
    int rc;
    if ((rc = alloc_batch(m, B))) return rc;
    cudaStream_t s = m->stream;
    MLP_CUDA(m, cudaMemsetAsync(m->err, 0, 4, s));
    MLP_CUDA(m, cudaMemsetAsync(m->st->loss, 0, sizeof(double) * 3, s));
    count_launch();
    k_mlp_gather<<<B, 64, 0, s>>>(X, B, m->d.D, y, 0, m->d.G, B, m->d.Dk, m->d.Dn, ~0ull, m->st, m->Xb, m->XbT, m->yb);
    MLP_CUDA(m, cudaGetLastError());
    if ((rc = enqueue_fwd_bwd(m, s))) return rc;
    ApplyArgs a = apply_args(m, 0);
    a.grad = grad;
    if ((rc = launch_apply(m, a, s))) return rc;
    if ((rc = check_err(m))) return rc;
    if (loss) {
        double h[3];
        MLP_CUDA(m, cudaMemcpy(h, m->st->loss, sizeof(h), cudaMemcpyDeviceToHost));
        *loss = h[2] > 0 ? h[0] / h[2] : 0.0;
    }
    return KM_OK;
}

KM_API int kmeans_mlp_train(kmeans_mlp *m, const float *X, int64_t N, const int32_t *labels, int32_t K,
                            int64_t steps, int32_t batch, float lr, uint64_t seed, double *mean_loss,
                            double *accuracy) {
    if (!m) return mlp_fail(nullptr, KM_EINVAL, "network is NULL");
    if (!X || !labels) return mlp_fail(m, KM_EINVAL, "a pointer argument is NULL");
    if (N < 1 || steps < 0 || K < 0 || !(lr > 0.f)) return mlp_fail(m, KM_EINVAL, "bad N, steps, K or lr");
    if (batch < 128 || batch % 128 != 0 || batch > (1 << 20))
        return mlp_fail(m, KM_EINVAL, "batch must be a multiple of 128 in [128, 2^20]");
    if (seed == ~0ull && N < batch) return mlp_fail(m, KM_EINVAL, "a fixed batch (seed ~0) needs N >= batch");
    if (!dev_ptr(X) || !dev_ptr(labels)) return mlp_fail(m, KM_EINVAL, "X and labels must be device memory");
    DevGuard dg(m->dev);
    int rc;
    if ((rc = alloc_batch(m, batch))) return rc;
    cudaStream_t s = m->stream;
    MLP_CUDA(m, cudaMemsetAsync(m->err, 0, 4, s));
    MLP_CUDA(m, cudaMemsetAsync(m->st->loss, 0, sizeof(double) * 3, s));
    // one step recorded once as a CUDA graph, replayed `steps` times (the
    // step counter on the device drives the row draw and Adam's bias correction)
    cudaStream_t cap = nullptr;
    MLP_CUDA(m, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    struct CapGuard {
        cudaStream_t s;
        ~CapGuard() { cudaStreamDestroy(s); }
    } cg{cap};
    MLP_CUDA(m, cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    count_launch();
    k_mlp_gather<<<batch, 64, 0, cap>>>(X, N, m->d.D, labels, K, m->d.G, batch, m->d.Dk, m->d.Dn, seed, m->st, m->Xb,
                                        m->XbT, m->yb);
    rc = cudaGetLastError() == cudaSuccess ? enqueue_fwd_bwd(m, cap) : mlp_fail(m, KM_ECUDA, "gather launch failed");
    if (!rc) {
        ApplyArgs a = apply_args(m, 1);
        a.lr = lr;
        rc = launch_apply(m, a, cap);
    }
    if (!rc) {
        count_launch();
        k_mlp_step_end<<<1, 1, 0, cap>>>(m->st);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    MLP_CUDA(m, e2);
    cudaGraphExec_t ex = nullptr;
    cudaError_t e3 = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    MLP_CUDA(m, e3);
    struct ExecGuard {
        cudaGraphExec_t x;
        ~ExecGuard() { cudaGraphExecDestroy(x); }
    } eg{ex};
    for (int64_t i = 0; i < steps; ++i) MLP_CUDA(m, cudaGraphLaunch(ex, s));
    if ((rc = check_err(m))) return rc;
    double h[3];
    MLP_CUDA(m, cudaMemcpy(h, m->st->loss, sizeof(h), cudaMemcpyDeviceToHost));
    if (mean_loss) *mean_loss = h[2] > 0 ? h[0] / h[2] : 0.0;
    if (accuracy) *accuracy = h[2] > 0 ? h[1] / h[2] : 0.0;
    return KM_OK;
}

KM_API int kmeans_mlp_predict_net(kmeans_mlp *m, const float *X, int64_t N, int32_t *pred) {
    if (!m) return mlp_fail(nullptr, KM_EINVAL, "network is NULL");
    if (!X || !pred || N < 1) return mlp_fail(m, KM_EINVAL, "bad X, pred or N");
    if (!dev_ptr(X) || !dev_ptr(pred)) return mlp_fail(m, KM_EINVAL, "X and pred must be device memory");
    DevGuard dg(m->dev);
    MLP_CUDA(m, cudaMemsetAsync(m->err, 0, 4, m->stream));
    int rc;
    if ((rc = mlp_predict_enqueue(m, X, N, pred, m->stream))) return rc;
    return check_err(m);
}

KM_API void kmeans_mlp_destroy(kmeans_mlp *m) {
    if (!m) return;
    DevGuard dg(m->dev);
    for (void *p : m->batch_allocs) cudaFreeAsync(p, m->stream);
    for (void *p : m->allocs) cudaFreeAsync(p, m->stream);
    cudaStreamSynchronize(m->stream);
    delete m;
}

KM_API const char *kmeans_mlp_last_error(const kmeans_mlp *m) { return m ? m->errmsg : kp::g_mlp_err; }

}  // extern "C"
