// kp_tc.cuh -- pieces shared by the tensor-core dense kernels: mbarrier and
// TMA helpers, tcgen05 descriptors and TMEM loads, the bfloat16 split, the
// 128-byte-swizzled tile layout, and the branch-free row scan of the
// epilogue (group minima, winner, runner-up).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "kp_common.cuh"

namespace kp {
namespace {

constexpr int kTM = 128;          // points per tile
constexpr uint32_t kPolls = 1u << 22;
constexpr int kAtomBytes = kTM * 128;  // one 64-element bfloat16 column block of a tile

__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)1 << 16;            // leading byte offset (unused for swizzled K-major)
    d |= (uint64_t)(1024 >> 4) << 32;  // stride byte offset: 8 rows x 128 B
    d |= (uint64_t)1 << 46;            // descriptor version
    d |= (uint64_t)2 << 61;            // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void bar_init(uint64_t *b, uint32_t n) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(uint64_t *b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(b)) : "memory");
}
// bounded wait; on time-out records KM_ETIMEOUT and returns false
__device__ __forceinline__ bool bar_wait(uint64_t *b, uint32_t parity, Ctrl *ctrl) {
    for (uint32_t i = 0; i < kPolls; ++i)
        if (mbar_try_wait(b, parity)) return true;
    atomicExch(&ctrl->err, (int)KM_ETIMEOUT);
    return false;
}
__device__ __forceinline__ void tma_2d(void *dst, const CUtensorMap *m, int c0, int c1, uint64_t *b) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"((uint64_t)m), "r"(c0), "r"(c1), "r"(smem_u32(b))
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Asynchronous TMEM read of 32 columns; the registers may be used only after
// tmem_wait32 on the same array (which names them, so that the compiler
// cannot move their uses above the wait).
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait32(uint32_t (&r)[32]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]), "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]), "+r"(r[15]), "+r"(r[16]), "+r"(r[17]), "+r"(r[18]), "+r"(r[19]), "+r"(r[20]), "+r"(r[21]), "+r"(r[22]), "+r"(r[23]), "+r"(r[24]), "+r"(r[25]), "+r"(r[26]), "+r"(r[27]), "+r"(r[28]), "+r"(r[29]), "+r"(r[30]), "+r"(r[31]) : : "memory");
}

// Asynchronous TMEM read of 16 columns (see tmem_ld32_async)
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// byte offset of the 16-byte chunk holding bfloat16 elements [8q, 8q+8) of
// `row` in a 128-byte-swizzled K-major tile (64 elements per 128-byte row)
__device__ __forceinline__ uint32_t swz_chunk(int row, int q, int atom_bytes) {
    return (uint32_t)((q >> 3) * atom_bytes + row * 128 + (((q & 7) ^ (row & 7)) << 4));
}

__device__ __forceinline__ void split8(const float *v, uint4 &h, uint4 &l) {
    uint32_t hw[4], lw[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        __nv_bfloat16 h0 = __float2bfloat16_rn(v[2 * i]), h1 = __float2bfloat16_rn(v[2 * i + 1]);
        __nv_bfloat16 l0 = __float2bfloat16_rn(v[2 * i] - __bfloat162float(h0));
        __nv_bfloat16 l1 = __float2bfloat16_rn(v[2 * i + 1] - __bfloat162float(h1));
        hw[i] = (uint32_t)__bfloat16_as_ushort(h0) | ((uint32_t)__bfloat16_as_ushort(h1) << 16);
        lw[i] = (uint32_t)__bfloat16_as_ushort(l0) | ((uint32_t)__bfloat16_as_ushort(l1) << 16);
    }
    h = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    l = make_uint4(lw[0], lw[1], lw[2], lw[3]);
}
// Running scan of one row over a run of accumulator columns: the per-group
// minima (stored into the row's shared-memory slots as each group closes),
// and the smallest value with its index and the runner-up, in two independent
// chains (even and odd columns).  Branch-free: pen[c] is +inf where column c
// opens a group (0 elsewhere), so that gm + pen restarts the running minimum,
// and the closing minimum is stored by a predicated shared store.  A row is
// scanned as two such runs (the two halves of its columns) interleaved column
// by column, for instruction-level parallelism; merge() joins them.
struct RowScan {
    float b1[2], b2[2];
    int i1[2];
    float gm;     // minimum of the open group
    uint32_t rp;  // shared-memory address of the open group's slot

    __device__ __forceinline__ void init(const float *slot) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            b1[c] = INFINITY;
            b2[c] = INFINITY;
            i1[c] = 0;  // kept when no column is below +inf (then column 0)
        }
        gm = INFINITY;
        rp = smem_u32(slot);
    }
    __device__ __forceinline__ void col(float acc, float cnv, float pen, int c, int jpar) {
        const float t = fmaf(-2.f, acc, cnv);
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.f32 p, %2, 0f00000000;\n\t@p st.shared.f32 [%0], %1;\n\t"
            "@p add.u32 %0, %0, 4;\n\t}"
            : "+r"(rp)
            : "f"(gm), "f"(pen)
            : "memory");
        gm = fminf(__fadd_rn(gm, pen), t);
        b2[jpar] = fminf(b2[jpar], fmaxf(b1[jpar], t));
        const bool lt = t < b1[jpar];
        b1[jpar] = lt ? t : b1[jpar];
        i1[jpar] = lt ? c : i1[jpar];
    }
    // store the open group's minimum
    __device__ __forceinline__ void close() const {
        asm volatile("st.shared.f32 [%0], %1;" ::"r"(rp), "f"(gm) : "memory");
    }
    // winner (lowest index among equal values) and runner-up of both chains
    __device__ __forceinline__ void result(float &w1, int &wi, float &w2) const {
        const bool odd = b1[1] < b1[0] || (b1[1] == b1[0] && i1[1] < i1[0]);
        w1 = odd ? b1[1] : b1[0];
        wi = odd ? i1[1] : i1[0];
        w2 = fminf(fminf(b2[0], b2[1]), fmaxf(b1[0], b1[1]));
    }
};

template <int W>
__device__ __forceinline__ void scan_one(RowScan &A, const uint32_t (&ra)[W], int ca, const float *cn,
                                         const float *pen) {
#pragma unroll
    for (int j = 0; j < W; j += 4) {
        const float4 na = *reinterpret_cast<const float4 *>(cn + ca + j);
        const float4 pa = *reinterpret_cast<const float4 *>(pen + ca + j);
        const float nav[4] = {na.x, na.y, na.z, na.w}, pav[4] = {pa.x, pa.y, pa.z, pa.w};
#pragma unroll
        for (int jj = 0; jj < 4; ++jj) A.col(__uint_as_float(ra[j + jj]), nav[jj], pav[jj], ca + j + jj, jj & 1);
    }
}

// group of column `col` from the boundary masks (contiguous groups)
__device__ __forceinline__ int group_of(const uint32_t *bm, int col) {
    const int c = col >> 5;
    int g = __popc(bm[c] & ((2u << (col & 31)) - 1u));
    for (int i = 0; i < c; ++i) g += __popc(bm[i]);
    return g;
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        cudaDriverEntryPointQueryResult q;
        void *f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    });
    return fn;
}

}  // namespace
}  // namespace kp
