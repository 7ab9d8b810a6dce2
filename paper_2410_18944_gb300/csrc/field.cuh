// Neural field of the guiding distribution (Sec. 4.2 Eq. nn_to_theta,
// Sec. 5.2): multi-resolution hash-grid encoding (L = 16 levels, F = 2 FP16
// features per lattice vertex, bi/tri-linear interpolation, levels
// concatenated into 32 features) and a ReLU MLP 32 -> 64 -> 64 -> (d+2)K+1
// whose three layers run on tcgen05 tensor cores: BF16 operands in shared
// memory, FP32 accumulators in TMEM, one 128-row tile per 128 threads.
//
// Level l has resolution N_l = floor(N_min b^l) (N_{L-1} = N_max); levels
// whose (N_l + 1)^d vertices fit the table are indexed densely, finer ones
// by the spatial hash of Mueller et al. (2022) with primes 1, 2654435761,
// 805459861.
#pragma once
#include "../../include/wost.h"
#include "common.cuh"
#include "umma.cuh"

#ifndef WOST_GRID_L2_ONLY
#define WOST_GRID_L2_ONLY 1
#endif

namespace wost {

constexpr int kFeat = 32;     // L * F
constexpr int kHid = 64;      // hidden width
constexpr int kMaxLevels = 16;
// Lobe capacity of the kernels' internal output layout (below): 8 for the
// standard kernels (K = 1..8), 16 for the wide-mixture kernels (K = 9..16,
// the lobe-count ablation of Sec. 6.3).
constexpr int kMaxK = 8;
constexpr int kMaxKWide = 16;
__host__ __device__ constexpr int field_km(int K) { return K <= kMaxK ? kMaxK : kMaxKWide; }
// padded output width of the internal layout of KM lobes: (d + 2) KM + 1
// outputs (33 / 41 for KM = 8, 65 / 81 for KM = 16) rounded up to a
// multiple of 16, the N granule of the layer-3 MMA
__host__ __device__ constexpr int out_pad(int KM) { return KM <= kMaxK ? 48 : 96; }
constexpr int kOutPad = out_pad(kMaxK);

// bf16 weight image in shared memory (core-matrix tiles, rows = outputs)
constexpr int kW1Bytes = kHid * kFeat * 2;       // 64 x 32
constexpr int kW2Bytes = kHid * kHid * 2;        // 64 x 64
__host__ __device__ constexpr int w3_bytes(int KM) { return out_pad(KM) * kHid * 2; }   // 48 (96) x 64
__host__ __device__ constexpr int wimg_bytes(int KM) { return kW1Bytes + kW2Bytes + w3_bytes(KM); }
constexpr int kW3Bytes = w3_bytes(kMaxK);
constexpr int kWImgBytes = wimg_bytes(kMaxK);

// The kernels read decoded outputs in one internal layout of KM lobes:
// mu'_i (KM x d), kappa'_i, lambda'_i (KM each), c', zero padding to
// out_pad(KM).  A field of K < KM lobes keeps its exchange layout (K lobes,
// nout = (d + 2) K + 1 rows); lobes K.. of the internal layout are disabled:
// zero weights and a lambda' bias of kOffLambda, so their mixture weight is
// exactly zero and every gradient into them vanishes (each carries a factor
// of the weight).  Internal row -> exchange row (-1: none) and back:
constexpr float kOffLambda = -1.0e4f;
__host__ __device__ inline int out_row_to_exchange(int r, int d, int K, int KM = kMaxK) {
    if (r < KM * d) { int i = r / d; return i < K ? i * d + r % d : -1; }
    r -= KM * d;
    if (r < KM) return r < K ? K * d + r : -1;                      // kappa'
    r -= KM;
    if (r < KM) return r < K ? K * d + K + r : -1;                  // lambda'
    return r == KM ? K * (d + 2) : -1;                              // c', padding
}
__host__ __device__ inline int exchange_to_out_row(int e, int d, int K, int KM = kMaxK) {
    if (e < K * d) return (e / d) * d + e % d;
    e -= K * d;
    if (e < K) return KM * d + e;
    e -= K;
    if (e < K) return KM * d + KM + e;
    return KM * (d + 2);
}
__host__ __device__ inline bool is_off_lambda(int r, int d, int K, int KM = kMaxK) {
    const int i = r - (KM * d + KM);
    return i >= K && i < KM;
}

struct DevField {
    int dim, K, L, log2T, nout;
    uint32_t dense_mask;          // bit l: level l indexed densely
    uint32_t level_off[kMaxLevels];   // first entry of level l (l 2^log2T for the hash grid)
    int res[kMaxLevels];
    float lo[3], inv_ext[3];      // u = (x - lo) * inv_ext in [0,1]^d
    const __half2 *grid16;        // all levels' entries (F = 2), level l from level_off[l]
    const uint4 *wimg;            // kWImgBytes, layout above
    const float *b3;              // kOutPad (zero padded)
};

// interpolation corners of level l around x: T-table index and weight
template <int D>
__device__ __forceinline__ void level_corners(const DevField &f, int l, const float *u, uint32_t *idx, float *w) {
    const int N = f.res[l];
    const bool dense = (f.dense_mask >> l) & 1u;
    const uint32_t mask = (1u << f.log2T) - 1u;
    int c[3];
    float fr[3];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float p = u[k] * (float)N;
        float fl = floorf(p);
        fl = fminf(fmaxf(fl, 0.f), (float)(N - 1));
        c[k] = (int)fl;
        fr[k] = p - fl;
    }
#pragma unroll
    for (int m = 0; m < (1 << D); ++m) {
        uint32_t v[3];
        float wt = 1.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            int b = (m >> k) & 1;
            v[k] = (uint32_t)(c[k] + b);
            wt *= b ? fr[k] : 1.f - fr[k];
        }
        uint32_t id;
        if (dense) {
            uint32_t side = (uint32_t)N + 1u;
            id = v[0] + side * (v[1] + (D == 3 ? side * v[2] : 0u));
        } else {
            id = v[0] ^ (v[1] * 2654435761u);
            if (D == 3) id ^= v[2] * 805459861u;
            id &= mask;
        }
        idx[m] = id;
        w[m] = wt;
    }
}

template <int D>
__device__ __forceinline__ void unit_coords(const DevField &f, const float *x, float *u) {
#pragma unroll
    for (int k = 0; k < D; ++k) u[k] = (x[k] - f.lo[k]) * f.inv_ext[k];
}

// encode one position into a row of the bf16 feature tile (kFeat columns)
// groups of four levels whose corner gathers are in flight together (two
// groups measured 3-4% slower in the warp-specialised walk kernel and no
// faster in training, at 14-18 more registers)
#ifndef WOST_ENCODE_UNROLL
#define WOST_ENCODE_UNROLL 1
#endif
constexpr int kEncodeUnroll = WOST_ENCODE_UNROLL;

template <int D>
__device__ __forceinline__ void encode_row(const DevField &f, const float *x, uint8_t *xtile, int row) {
    float u[D];
    unit_coords<D>(f, x, u);
#pragma unroll kEncodeUnroll
    for (int l4 = 0; l4 < kMaxLevels; l4 += 4) {
        float feat[8];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            int l = l4 + j;
            uint32_t idx[1 << D];
            float w[1 << D];
            level_corners<D>(f, l, u, idx, w);
            float a0 = 0.f, a1 = 0.f;
#pragma unroll
            for (int m = 0; m < (1 << D); ++m) {
#if WOST_GRID_L2_ONLY
                // the table is gathered at random: keep it out of L1 (which
                // holds the BVH) and serve it from L2
                __half2 hv = __ldcg(f.grid16 + (size_t)f.level_off[l] + idx[m]);
#else
                __half2 hv = __ldg(f.grid16 + (size_t)f.level_off[l] + idx[m]);
#endif
                float2 g = __half22float2(hv);
                a0 = fmaf(w[m], g.x, a0);
                a1 = fmaf(w[m], g.y, a1);
            }
            feat[2 * j] = a0;
            feat[2 * j + 1] = a1;
        }
        st_row8_bf16(xtile, row, 2 * l4, kFeat, feat);
    }
}

// One 128-row tile: X (128 x 32) -> H1 -> H2 -> Y (128 x out_pad(KM)) in
// TMEM columns [tcol, tcol + tile_tmem_cols(KM)).  Called by all 128 threads
// of the tile; thread `row` owns row `row`.  `issuer` issues the MMAs.  On
// return out[0..out_pad(KM)) holds this row's raw outputs (+ bias).  Returns
// false if a bounded wait timed out.
__host__ __device__ constexpr int tile_tmem_cols(int KM) { return out_pad(KM) <= 64 ? 64 : 128; }
struct TileCtx {
    uint8_t *xtile;     // 128 x 32 bf16
    uint8_t *htile;     // 128 x 64 bf16
    const uint8_t *w;   // weight image
    uint64_t *mbar;
    uint32_t tmem;      // base column address of this tile (lane 0)
    uint32_t phase;
    int bar_id;         // named barrier of the tile (128 threads)
};

template <int KM = kMaxK>
__device__ __forceinline__ bool tile_mma_wait(TileCtx &t, bool issuer, int which, int *err) {
    // which: 0 = layer 1, 1 = layer 2, 2 = layer 3
    fence_async_smem();
    tc_fence_before();
    named_sync(t.bar_id, 128);
    if (issuer) {
        tc_fence_after();
        if (which == 0) umma_gemm(t.tmem, t.xtile, 0, kFeat, t.w, 0, kFeat, kHid, kFeat, false);
        else if (which == 1) umma_gemm(t.tmem, t.htile, 0, kHid, t.w + kW1Bytes, 0, kHid, kHid, kHid, false);
        else umma_gemm(t.tmem, t.htile, 0, kHid, t.w + kW1Bytes + kW2Bytes, 0, kHid, out_pad(KM), kHid, false);
        umma_commit(t.mbar);
    }
    bool ok = mbar_wait_bounded(t.mbar, t.phase);
    t.phase ^= 1u;
    tc_fence_after();
    // the give-up decision is taken by the whole tile, so that no thread is
    // left alone at a later named barrier
    ok = !named_or(t.bar_id, 128, !ok);
    if (!ok && (threadIdx.x & 127) == 0) atomicOr(err, 2);
    return ok;
}

__device__ __forceinline__ uint32_t lane_addr(uint32_t tmem, int row, int col) {
    return tmem + ((uint32_t)(row & ~31) << 16) + (uint32_t)col;
}

// TMEM row -> ReLU -> bf16 row of the hidden tile
__device__ __forceinline__ void hidden_epilogue(TileCtx &t, int row, float *keep /* nullable, 64 */) {
#pragma unroll
    for (int c = 0; c < kHid; c += 16) {
        float v[16];
        tmem_ld16(lane_addr(t.tmem, row, c), v);
        tmem_ld_wait();
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
        if (keep)
#pragma unroll
            for (int i = 0; i < 16; ++i) keep[c + i] = v[i];
        st_row8_bf16(t.htile, row, c, kHid, v);
        st_row8_bf16(t.htile, row, c + 8, kHid, v + 8);
    }
}

template <int KM = kMaxK>
__device__ __forceinline__ bool mlp_tile_forward(TileCtx &t, const DevField &f, int row, bool issuer, float *out,
                                                 int *err) {
    constexpr int OUT = out_pad(KM);
    if (!tile_mma_wait<KM>(t, issuer, 0, err)) return false;
    hidden_epilogue(t, row, nullptr);
    if (!tile_mma_wait<KM>(t, issuer, 1, err)) return false;
    hidden_epilogue(t, row, nullptr);
    if (!tile_mma_wait<KM>(t, issuer, 2, err)) return false;
#pragma unroll
    for (int c = 0; c < OUT; c += 16) {
        tmem_ld16(lane_addr(t.tmem, row, c), out + c);
        tmem_ld_wait();
    }
#pragma unroll
    for (int i = 0; i < OUT; ++i) out[i] += __ldg(f.b3 + i);
    return true;
}

// shared setup of a 256-thread CTA running two MLP tiles: weight image,
// two X and two H tiles, two mbarriers, the TMEM base address (two tiles of
// tile_tmem_cols(KM) columns)
__host__ __device__ constexpr int cta_tiles_smem(int KM) {
    return wimg_bytes(KM) + 2 * (128 * kFeat * 2) + 2 * (128 * kHid * 2) + 64;
}
constexpr int kCtaTilesSmem = cta_tiles_smem(kMaxK);

struct CtaTiles {
    uint8_t *wimg, *xt, *ht;
    uint64_t *mbar;
    uint32_t *tptr;
};

template <int KM = kMaxK>
__device__ __forceinline__ CtaTiles cta_tiles_setup(uint8_t *sm, const DevField &f) {
    constexpr int kImg = wimg_bytes(KM);
    CtaTiles c;
    c.wimg = sm;
    c.xt = sm + kImg;
    c.ht = c.xt + 2 * (128 * kFeat * 2);
    c.mbar = reinterpret_cast<uint64_t *>(c.ht + 2 * (128 * kHid * 2));
    c.tptr = reinterpret_cast<uint32_t *>(c.mbar + 2);
    const int tid = threadIdx.x;
    for (int i = tid; i < kImg / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(c.wimg)[i] = __ldg(f.wimg + i);
    if (tid == 0) {
        mbar_init(&c.mbar[0], 1);
        mbar_init(&c.mbar[1], 1);
        fence_mbar_init();
    }
    if (tid < 32) tmem_alloc(c.tptr, 2 * tile_tmem_cols(KM));
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return c;
}

template <int KM = kMaxK>
__device__ __forceinline__ void cta_tiles_teardown(const CtaTiles &c) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(*c.tptr, 2 * tile_tmem_cols(KM));
}

}  // namespace wost

// host-side field state
struct wost_field {
    wost_field_desc desc{};
    int device = -1;                         // CUDA device the field's buffers live on
    int nout = 0;
    int km = wost::kMaxK;                    // lobe capacity of the kernels serving the field: field_km(K)
    int64_t T = 0;
    int res[16] = {0};
    uint32_t dense_mask = 0;
    int64_t level_off[wost::kMaxLevels + 1] = {0};   // entry offsets per level; [L] = entries of all levels
    // device buffers
    float *grid32 = nullptr, *grid_m = nullptr, *grid_v = nullptr, *grid_g = nullptr;
    __half2 *grid16 = nullptr;
    float *mlp32 = nullptr, *mlp_m = nullptr, *mlp_v = nullptr, *mlp_g = nullptr;  // W1|W2|W3|b3 (exchange layout)
    uint8_t *wimg = nullptr;
    float *b3pad = nullptr;
    // training records: final buffer (12 floats each) and per-slot scratch
    float *rec = nullptr;
    int64_t rec_cap = 0;
    unsigned long long *rec_ctr = nullptr;   // [0] count, [1] dropped
    float *scratch = nullptr;
    size_t scratch_bytes = 0;
    float *loss_acc = nullptr;               // [0] FP64 loss sum, [1] Adam step count (u64),
                                             // [2] records the last step used (u64)
    // the Adam step count lives on the device so that a captured graph of
    // training steps advances it on every replay
    unsigned long long *adam_step() const { return reinterpret_cast<unsigned long long *>(loss_acc) + 1; }
    unsigned long long *used_records() const { return reinterpret_cast<unsigned long long *>(loss_acc) + 2; }
    int t_c_mode = 0, t_reflect = 1;         // MIS options of the records in the buffer
    float t_c_fixed = 0.5f;
    int64_t t_samples = 0;                   // records per training step (0 = all)
    int64_t n_mlp() const {
        int H = desc.hidden, nin = desc.levels * desc.features;
        return (int64_t)H * nin + (int64_t)H * H + (int64_t)nout * H + nout;
    }
    int64_t n_grid() const { return level_off[desc.levels] * desc.features; }
    wost::DevField dev() const;
    ~wost_field();
};
