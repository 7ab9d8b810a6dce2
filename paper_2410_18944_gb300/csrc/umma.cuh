// Fifth-generation tensor-core primitives for sm_103a (inline PTX):
// TMEM allocation, tcgen05.mma (kind::f16, BF16 operands, FP32 accumulator
// in TMEM), commit to an mbarrier, TMEM loads, and the shared-memory matrix
// descriptors.
//
// Shared-memory operand layout used throughout ("core-matrix tiles", no
// swizzle): a row-major logical tile with R rows and C columns of bf16 (both
// multiples of 8) is stored as 8x8 core matrices of 128 contiguous bytes,
// core matrix (r/8, c/8) at byte ((r/8) * (C/8) + c/8) * 128, element
// (r%8, c%8) at +16 (r%8) + 2 (c%8).  The same bytes serve as
//   - a K-major operand with rows = M (or N) and columns = K:
//       leading (K-direction) core stride 128 B, stride (M/N-direction) (C/8)*128 B;
//   - an MN-major operand with rows = K and columns = M (or N):
//       leading (K-direction) core stride (C/8)*128 B, stride (M/N-direction) 128 B.
// One MMA consumes K = 16 (two core matrices along K).
#pragma once
#include <stdint.h>

namespace wost {

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__host__ __device__ __forceinline__ uint32_t cm_offset(int r, int c, int C) {
    return (uint32_t)(((r >> 3) * (C >> 3) + (c >> 3)) * 128 + (r & 7) * 16 + (c & 7) * 2);
}

// shared-memory matrix descriptor (sm_100 family): start >> 4 [0,14),
// leading byte offset >> 4 [16,30), stride byte offset >> 4 [32,46),
// version 1 at [46,48), base offset 0, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor, kind::f16: D f32 [4,6)=1, A bf16 [7,10)=1,
// B bf16 [10,13)=1, A major [15], B major [16] (1 = MN-major),
// N >> 3 [17,23), M >> 4 [24,29)
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int M, int N, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        :
        : "r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void umma_commit(uint64_t *mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :
                 : "r"(smem_u32(mbar))
                 : "memory");
}

// tcgen05.alloc takes a power-of-two column count in [32, 512]
__host__ __device__ constexpr uint32_t tmem_cols(uint32_t n) {
    uint32_t c = 32;
    while (c < n) c <<= 1;
    return c;
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :
                 : "r"(smem_u32(dst_smem)), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" : : "r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// generic-proxy shared-memory writes -> visible to the tensor core (async proxy)
__device__ __forceinline__ void fence_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 32 lanes x 32 bit, 16 consecutive columns: thread i of the warp gets lane
// (32 * (warp % 4) + i) of columns [col, col + 16)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- mbarrier ------------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" : : "r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits are bounded by time, not by poll count: a failing try_wait may
// suspend the warp for a hardware-chosen while, so a poll count says little
// about how long a wait lasts.
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait: false once limit_ns have passed (the caller reports a
// timeout).  Waits for the completion of the CTA's own tensor-core work keep
// the default: that work always completes, and the CTA must not release its
// TMEM while an MMA may still write it.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity,
                                                  unsigned long long limit_ns = kWaitNs) {
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer_ns();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer_ns() - t0 > limit_ns) return false;
    }
}

// named barrier over `count` threads and an OR-reduction over it
__device__ __forceinline__ void named_sync(int id, int count) {
    asm volatile("bar.sync %0, %1;" : : "r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ bool named_or(int id, int count, bool pred) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, %3, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(id), "r"(count)
        : "memory");
    return r != 0;
}

// 8 consecutive bf16 of one row into a core-matrix tile (16-byte store)
// 8 floats as BF16 (round to nearest even), in order
__device__ __forceinline__ uint4 pack8_bf16(const float *v) {
    __nv_bfloat162 p0 = __floats2bfloat162_rn(v[0], v[1]), p1 = __floats2bfloat162_rn(v[2], v[3]);
    __nv_bfloat162 p2 = __floats2bfloat162_rn(v[4], v[5]), p3 = __floats2bfloat162_rn(v[6], v[7]);
    uint4 u;
    u.x = *reinterpret_cast<uint32_t *>(&p0);
    u.y = *reinterpret_cast<uint32_t *>(&p1);
    u.z = *reinterpret_cast<uint32_t *>(&p2);
    u.w = *reinterpret_cast<uint32_t *>(&p3);
    return u;
}

__device__ __forceinline__ void st_row8_bf16(uint8_t *tile, int r, int c8, int C, const float *v) {
    *reinterpret_cast<uint4 *>(tile + cm_offset(r, c8, C)) = pack8_bf16(v);
}

__device__ __forceinline__ void ld_row8_bf16(const uint8_t *tile, int r, int c8, int C, float *v) {
    uint4 u = *reinterpret_cast<const uint4 *>(tile + cm_offset(r, c8, C));
    const __nv_bfloat162 *p = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        float2 f = __bfloat1622float2(p[i]);
        v[2 * i] = f.x;
        v[2 * i + 1] = f.y;
    }
}

// D[128 x N] (+)= A B^T over K (multiple of 16) with both operands in
// core-matrix tiles.  a_mn / b_mn select the operand's storage:
//   0: rows = M (N), cols = K   (K-major)      1: rows = K, cols = M (N)   (MN-major)
// a_cols / b_cols = number of columns C of the stored tile.
__device__ __forceinline__ void umma_gemm(uint32_t d_tmem, const uint8_t *A, int a_mn, int a_cols, const uint8_t *B,
                                          int b_mn, int b_cols, int N, int K, bool accumulate) {
    const uint32_t idesc = idesc_bf16(128, N, a_mn, b_mn);
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    const uint32_t a_row = (uint32_t)(a_cols >> 3) * 128u, b_row = (uint32_t)(b_cols >> 3) * 128u;
    for (int k = 0; k < K; k += 16) {
        // two core matrices along K per MMA
        uint64_t ad = a_mn ? smem_desc(a0 + (uint32_t)(k >> 3) * a_row, a_row, 128u)
                           : smem_desc(a0 + (uint32_t)(k >> 3) * 128u, 128u, a_row);
        uint64_t bd = b_mn ? smem_desc(b0 + (uint32_t)(k >> 3) * b_row, b_row, 128u)
                           : smem_desc(b0 + (uint32_t)(k >> 3) * 128u, 128u, b_row);
        umma_bf16(d_tmem, ad, bd, idesc, (accumulate || k > 0) ? 1u : 0u);
    }
}

}  // namespace wost
