// Shared device-side definitions of libwost: scene/field views passed to the
// kernels, the counter-based generator, and small math helpers.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define WOST_PI 3.14159265358979323846f

namespace wost {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 products
// mixed with the other words and the key; key advanced by two Weyl constants.
// Counter = (point, walk, step, purpose), key = (seed_lo, seed_hi + scene_id).
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ U4 philox(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
#ifdef __CUDA_ARCH__
        uint32_t hA = __umulhi(0xD2511F53u, c0), lA = 0xD2511F53u * c0;
        uint32_t hB = __umulhi(0xCD9E8D57u, c2), lB = 0xCD9E8D57u * c2;
#else
        uint64_t pA = (uint64_t)0xD2511F53u * c0, pB = (uint64_t)0xCD9E8D57u * c2;
        uint32_t hA = (uint32_t)(pA >> 32), lA = (uint32_t)pA;
        uint32_t hB = (uint32_t)(pB >> 32), lB = (uint32_t)pB;
#endif
        uint32_t n0 = hB ^ c1 ^ k0, n2 = hA ^ c3 ^ k1;
        c0 = n0; c1 = lB; c2 = n2; c3 = lA;
    }
    return {c0, c1, c2, c3};
}
// 24-bit uniform in [0,1), exactly representable in float
__host__ __device__ __forceinline__ float u01(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }

// purposes of the counter's last word: 3 + j are the 2D vMF retries j < 64;
// P_NEU draws the point on the primitive chosen for <N>, P_RR the Russian
// roulette of a long walk, and P_NKEY | id the selection key of Neumann
// primitive id
enum Purpose : uint32_t { P_MIS = 0, P_DIR = 1, P_SRC = 2, P_VMF2 = 3, P_NEU = 96, P_RR = 97, P_NKEY = 0x80000000u };

// ---------------------------------------------------------------------------
// analytic data functions (kind codes of wost_fn)
// ---------------------------------------------------------------------------
struct DevFn {
    int kind;
    int n;
    float p[40];
};

template <int D>
__device__ __forceinline__ float eval_fn(const DevFn &fn, const float *x) {
    switch (fn.kind) {
    case 0: return 0.f;
    case 1: return fn.p[0];
    case 2: return __expf(fn.p[0] * x[0]) * cosf(fn.p[0] * x[1]);
    case 3: return x[0] * x[0] - x[1] * x[1];
    case 4: { float s = 0; for (int i = 0; i < D; ++i) s += x[i] * x[i]; return s; }
    case 5: {
        float s = 0;
        for (int i = 0; i < D; ++i) { float d = x[i] - fn.p[i]; s += d * d; }
        return rsqrtf(s);
    }
    case 6: {
        float s = 0;
        for (int i = 0; i < D; ++i) { float d = x[i] - fn.p[i]; s += d * d; }
        return 0.5f * logf(s);
    }
    case 7: {
        int n = (int)fn.p[0];
        float sg = fn.p[1], acc = 0.f, inv = 1.f / (2.f * sg * sg);
        for (int k = 0; k < n && k < 8; ++k) {
            const float *c = fn.p + 3 + 4 * k;
            float s = 0;
            for (int i = 0; i < D; ++i) { float d = x[i] - c[i]; s += d * d; }
            acc += fn.p[2 + 4 * k] * __expf(-s * inv);
        }
        return acc;
    }
    case 8: return coshf(fn.p[0] * x[0]) * cosf(fn.p[0] * x[1]);
    case 9: {
        const float X = x[0], Y = x[1], Z = D == 3 ? x[2] : 0.f;
        return fn.p[0] + fn.p[1] * X + fn.p[2] * Y + fn.p[3] * Z + fn.p[4] * X * X + fn.p[5] * Y * Y +
               fn.p[6] * Z * Z + fn.p[7] * X * Y + fn.p[8] * X * Z + fn.p[9] * Y * Z;
    }
    case 10: return fn.p[0] * atan2f(x[1], x[0]) + fn.p[1];
    }
    return __int_as_float(0x7fc00000);
}

// ---------------------------------------------------------------------------
// Scene view.  BVH node layout (binary BVH, child boxes stored in the parent):
//   2D: 3 float4 = (c0.lo.x, c0.lo.y, c0.hi.x, c0.hi.y), (c1 ...), (ref0, ref1, -, -)
//   3D: 4 float4 = (c0.lo.xyz, c0.hi.x), (c0.hi.yz, c1.lo.xy), (c1.lo.z, c1.hi.xyz), (ref0, ref1, -, -)
// ref >= 0: inner node index; ref < 0: leaf, ~ref = start << 4 | (count - 1).
// Primitives are stored in leaf order:
//   Dirichlet / Neumann 2D segment: 1 float4 (a.x, a.y, b.x, b.y)
//   3D triangle: 3 float4 (a.xyz, b.x), (b.yz, c.xy), (c.z, -, -, -)
//   silhouette 2D vertex: 2 float4 (v.xy, n0.xy), (n1.xy, always, -)
//   silhouette 3D edge:   4 float4 (a.xyz, b.x), (b.yz, n0.xy), (n0.z, n1.xyz), (always, -, -, -)
// n0/n1 are inward unit normals of the two adjacent Neumann primitives.
// ---------------------------------------------------------------------------
struct DevBVH {
    const float4 *nodes;  // global memory, or shared memory when a kernel staged them
    const float4 *prims;  // (likewise)
    const int *ids;       // original primitive / element id per leaf slot
    const double *prims64; // FP64 copy of the primitive vertices (leaf order), 2D: 4, 3D: 9 doubles
    int nprims;
    int nnodes;
};

struct DevScene {
    int dim;
    float scale;          // bounding-box diagonal
    float tau;            // silhouette edge-on tolerance (1e-6 * scale)
    DevBVH dir, neu, sil;
    const float4 *sil_cones;  // per silhouette-BVH node: one normal cone per child (axis.xyz, cos half-angle)
    const float *nin_neu; // inward normal of each Neumann prim, by leaf slot of the Neumann BVH (dim floats)
    DevFn g, f, h;
    int has_source;
    int has_flux;         // nonzero Neumann flux h and Neumann primitives
};

// BVH node, normal-cone and primitive loads: generic, as the arrays may
// have been staged in shared memory by the kernel
__device__ __forceinline__ float4 ldn(const float4 *p) { return *p; }

__device__ __forceinline__ int leaf_start(int ref) { return (~ref) >> 4; }
__device__ __forceinline__ int leaf_count(int ref) { return ((~ref) & 15) + 1; }

// warp-aggregated atomic increment: returns this lane's slot
__device__ __forceinline__ unsigned long long warp_fetch_add(unsigned long long *ctr, bool want) {
    unsigned mask = __activemask();
    unsigned vote = __ballot_sync(mask, want);
    int lane = threadIdx.x & 31;
    int leader = __ffs(vote) - 1;
    unsigned long long base = 0;
    if (vote && lane == leader) base = atomicAdd(ctr, (unsigned long long)__popc(vote));
    base = __shfl_sync(mask, base, leader < 0 ? 0 : leader);
    return base + __popc(vote & ((1u << lane) - 1u));
}

// warp-aggregated append to a 32-bit counter: returns this lane's slot
__device__ __forceinline__ unsigned warp_append(unsigned *ctr) {
    unsigned mask = __activemask();
    int lane = threadIdx.x & 31;
    int leader = __ffs(mask) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(ctr, (unsigned)__popc(mask));
    base = __shfl_sync(mask, base, leader);
    return base + __popc(mask & ((1u << lane) - 1u));
}

}  // namespace wost
