// Diagnostic GEMM through the same tcgen05 / TMEM / descriptor path the walk
// and training kernels use: D[128 x N] = A[128 x K] B[N x K]^T with each
// operand stored K-major or MN-major in core-matrix tiles.  Used by the GPU
// tests to validate operand layouts independently of the field.
#include "internal.h"
#include "umma.cuh"

namespace wost {

__global__ void diag_umma_kernel(int a_mn, int b_mn, int N, int K, const float *A, const float *B, float *Dout, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *As = sm;                     // 128 x K  (32 KB max)
    uint8_t *Bs = sm + 32768 + 4096;      // N x K    (64 KB max)
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + 32768 + 4096 + 65536 + 4096);
    uint32_t *tptr = reinterpret_cast<uint32_t *>(mbar + 1);
    const int tid = threadIdx.x;
    __nv_bfloat16 *a16 = reinterpret_cast<__nv_bfloat16 *>(As), *b16 = reinterpret_cast<__nv_bfloat16 *>(Bs);
    for (int i = tid; i < 128 * K; i += blockDim.x) {
        int m = i / K, k = i % K;
        uint32_t off = a_mn ? cm_offset(k, m, 128) : cm_offset(m, k, K);
        a16[off / 2] = __float2bfloat16_rn(A[i]);
    }
    for (int i = tid; i < N * K; i += blockDim.x) {
        int n = i / K, k = i % K;
        uint32_t off = b_mn ? cm_offset(k, n, N) : cm_offset(n, k, K);
        b16[off / 2] = __float2bfloat16_rn(B[i]);
    }
    if (tid == 0) { mbar_init(mbar, 1); fence_mbar_init(); }
    if (tid < 32) tmem_alloc(tptr, 256);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tm = *tptr;
    if (tid == 0) {
        umma_gemm(tm, As, a_mn, a_mn ? 128 : K, Bs, b_mn, b_mn ? N : K, N, K, false);
        umma_commit(mbar);
    }
    bool ok = mbar_wait_bounded(mbar, 0);
    tc_fence_after();
    if (!ok) atomicOr(err, 2);
    if (ok) {
        for (int c = 0; c < N; c += 16) {
            float v[16];
            tmem_ld16(tm + ((uint32_t)(tid & ~31) << 16) + (uint32_t)c, v);
            tmem_ld_wait();
            for (int i = 0; i < 16; ++i) Dout[tid * N + c + i] = v[i];
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) tmem_dealloc(tm, 256);
}

// One warp waits, with the bounded wait of the walk kernels, on an mbarrier
// that receives its single arrival only when `arrive` is set.  Without it
// nothing ever arrives: the wait runs out after limit_ns and the kernel
// records a timeout in the error word and returns.
__global__ void diag_wait_kernel(unsigned long long limit_ns, int arrive, int *err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) { mbar_init(&bar, 1); fence_mbar_init(); }
    __syncwarp();
    if (arrive && threadIdx.x == 0)
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" : : "r"(smem_u32(&bar)) : "memory");
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!ok && threadIdx.x == 0) atomicOr(err, 2);
}

}  // namespace wost

using namespace wost;

extern "C" wost_status wost_diag_wait(int64_t limit_ns, int32_t arrive) {
    if (limit_ns <= 0 || limit_ns > 10000000000LL) {
        set_error("wost_diag_wait: limit_ns must be in (0, 1e10]");
        return WOST_ERR_INVALID_ARG;
    }
    diag_wait_kernel<<<1, 32>>>((unsigned long long)limit_ns, arrive ? 1 : 0, device_err_flag());
    WOST_CUDA(cudaGetLastError());
    return device_check(0);
}

extern "C" wost_status wost_diag_umma(int32_t a_mn, int32_t b_mn, int32_t N, int32_t K, const float *A,
                                      const float *B, float *D) {
    if (!A || !B || !D || N < 16 || N > 256 || N % 16 || K < 16 || K > 128 || K % 16) {
        set_error("wost_diag_umma: invalid argument");
        return WOST_ERR_INVALID_ARG;
    }
    float *dA, *dB, *dD;
    WOST_CUDA(cudaMalloc(&dA, 128 * K * sizeof(float)));
    WOST_CUDA(cudaMalloc(&dB, N * K * sizeof(float)));
    WOST_CUDA(cudaMalloc(&dD, 128 * N * sizeof(float)));
    WOST_CUDA(cudaMemcpy(dA, A, 128 * K * sizeof(float), cudaMemcpyHostToDevice));
    WOST_CUDA(cudaMemcpy(dB, B, N * K * sizeof(float), cudaMemcpyHostToDevice));
    const int smem = 32768 + 4096 + 65536 + 4096 + 64;
    WOST_CUDA(cudaFuncSetAttribute(diag_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    diag_umma_kernel<<<1, 128, smem>>>(a_mn, b_mn, N, K, dA, dB, dD, device_err_flag());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(D, dD, 128 * N * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dD);
    if (e != cudaSuccess) return cuda_status(e, "wost_diag_umma");
    return device_check(0);
}
