// Online training step of the guiding field (Sec. 4.2, 4.4, 5.2).
//
// Per record (x, nu, Neumann normal n, q = p~ at sampling, target p_t) the
// surrogate loss
//   l = -(p_t / q) [ log p_g(nu | Theta(x)) + e log(c p_g0 + (1 - c) p_u) ]
// (p_g0 = p_g held constant) has exactly the paper's one-sample gradients:
// Eq. one_sample_kld for Theta and Eq. one_sample_sp for c.  The mean over
// records is back-propagated through the MLP and scattered onto the hash grid.
//
// One fused persistent kernel, two 128-record tiles per CTA (256 threads;
// one tile of 128 threads for fields of 9..16 lobes, whose 96 outputs widen
// the gradient tile and the TMEM columns beyond two tiles per SM):
//   forward recomputation (3 tcgen05 MMAs) -> per-thread loss and d raw ->
//   dH2 = dY W3, dZ2 = dH2 * [H2 > 0] -> dH1 = dZ2 W2 -> dZ1 -> dX = dZ1 W1
//   -> hash-grid scatter-add (FP32 atomics); the weight gradients
//   dW3 = dY^T H2, dW2 = dZ2^T H1, dW1 = dZ1^T X accumulate in TMEM across all
//   tiles of the CTA (MN-major operands read the same per-record tiles) and
//   are flushed once with atomics.  Activations are recomputed, not stored.
// Then one elementwise Adam kernel (Kingma & Ba 2015) updates the FP32
// masters and rewrites the FP16 grid and BF16 weight-image copies.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "field.cuh"
#include "internal.h"
#include "vmf.cuh"

namespace wost {

// Per KM (lobe capacity of the field's output layout, 8 or 16):
constexpr int kTX = 128 * kFeat * 2;     // X tile
constexpr int kTH = 128 * kHid * 2;      // H1 / H2 tiles
// G tile, gcols(KM) columns: [dY | 0 | dZ2] (dZ2 from column z2col(KM)),
// then [dZ1 | ... | dZ2].  KM = 8: 48 + 16 + 64 = 128; KM = 16: 96 + 64 = 160
__host__ __device__ constexpr int z2col(int KM) { return KM <= kMaxK ? 64 : 96; }
__host__ __device__ constexpr int gcols(int KM) { return z2col(KM) + kHid; }
__host__ __device__ constexpr int tg_bytes(int KM) { return 128 * gcols(KM) * 2; }
// gradient tiles are stored as a BF16 pair hi + lo (lo = bf16(v - hi)), so the
// MMAs see the FP32 gradient to ~16 bits; activations and weights are BF16
// exactly as in the forward pass
__host__ __device__ constexpr int tile_bytes(int KM) { return kTX + 2 * kTH + 2 * tg_bytes(KM); }
// 128-record tiles per CTA: two for KM = 8 (226 KB of shared memory); one for
// KM = 16, whose tile and TMEM columns (128 + 3 x 64) do not fit twice
__host__ __device__ constexpr int train_tiles(int KM) { return KM <= kMaxK ? 2 : 1; }
__host__ __device__ constexpr int train_block(int KM) { return 128 * train_tiles(KM); }
// TMEM columns of the scratch accumulator s0 of a tile (the layer-3 outputs)
__host__ __device__ constexpr int s0cols(int KM) { return tile_tmem_cols(KM); }
constexpr int kTrainCtl = 128;   // mbarriers, TMEM address, per-level gradient copy offsets
__host__ __device__ constexpr int train_smem(int KM) {
    return wimg_bytes(KM) + train_tiles(KM) * tile_bytes(KM) + kTrainCtl;
}
static_assert(train_smem(kMaxK) <= 227 * 1024 && train_smem(kMaxKWide) <= 227 * 1024, "training tiles");
static_assert(train_tiles(kMaxK) * (s0cols(kMaxK) + 3 * 64) <= 512 &&
              train_tiles(kMaxKWide) * (s0cols(kMaxKWide) + 3 * 64) <= 512, "training TMEM columns");

// Gradient copies of the coarse levels.  Every record scatters onto each
// level, so the few hundred to few thousand vertices of a coarse level take
// thousands of atomic adds each per step and serialise in L2.  A level of
// the hash grid that is indexed densely uses only (N + 1)^d of its table's
// entries; its gradient is scattered into R copies laid out one after the
// other in its table (copy c at entry c (N + 1)^d, the CTA's index mod R)
// and priv_reduce_kernel sums them into copy 0 and clears the rest, so
// every later reader sees the plain gradient.  Measured on one GB300 before
// the copies (star, 2^18 records per step): skipping the scatter of the six
// coarsest levels saved 0.067 ms of a 0.387 ms step, the ten finer ones
// 0.034 ms.
constexpr int kGradCopies = 16;
// only levels of at most this many vertices take copies (2^18 records give
// them hundreds of adds per vertex; finer levels gain less than the
// reduction costs)
#ifndef WOST_GRAD_COPY_MAXV
#define WOST_GRAD_COPY_MAXV 16384
#endif
struct GradCopies {
    int n;                         // levels with more than one copy
    int lvl[kMaxLevels];           // those levels
    unsigned long long off[kMaxLevels];   // first entry of the level
    int V[kMaxLevels], R[kMaxLevels];     // used entries, copies
    int start[kMaxLevels + 1];     // prefix sums of V (reduce-kernel indexing)
    int copy_V[kMaxLevels], copy_R[kMaxLevels];   // per level l (R 1: no copies)
};

struct TrainArgs {
    DevField f;
    const float *rec;
    const unsigned long long *rec_ctr;
    long long rec_cap;
    int c_mode;
    float c_fixed;
    int reflect;
    float e_sel;
    float *g_grid;   // L x T x F
    float *g_W1, *g_W2, *g_W3, *g_b3;
    double *loss_acc;
    long long max_samples;                  // records per step (0 = all)
    long long off_fixed;                    // stratum of this step (< 0: from the Adam step count)
    const unsigned long long *step;         // Adam step count before this step
    unsigned long long *used;               // records this step used
    int loss_only;                          // forward recomputation and loss only, no gradients
    int *err;
    GradCopies gc;                          // coarse-level gradient copies
};

struct TTile {
    uint8_t *X, *H1, *H2, *G, *Gl;
    const uint8_t *w;
    uint64_t *mbar;
    uint32_t s0, acc3, acc2, acc1;   // TMEM column addresses
    uint32_t phase;
    int bar;
};

template <class F>
__device__ __forceinline__ bool tt_issue_wait(TTile &t, bool issuer, F issue, int *err) {
    fence_async_smem();
    tc_fence_before();
    named_sync(t.bar, 128);
    if (issuer) {
        tc_fence_after();
        issue();
        umma_commit(t.mbar);
    }
    bool ok = mbar_wait_bounded(t.mbar, t.phase);
    t.phase ^= 1u;
    tc_fence_after();
    ok = !named_or(t.bar, 128, !ok);   // tile-uniform give-up decision
    if (!ok && (threadIdx.x & 127) == 0) atomicOr(err, 2);
    return ok;
}

// 8 values of a row as a BF16 hi/lo pair into the G tiles
__device__ __forceinline__ void st_row8_split(uint8_t *hi, uint8_t *lo, int r, int c8, int C, const float *v) {
    float h[8], l[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        h[i] = __bfloat162float(__float2bfloat16_rn(v[i]));
        l[i] = v[i] - h[i];
    }
    st_row8_bf16(hi, r, c8, C, h);
    st_row8_bf16(lo, r, c8, C, l);
}

__device__ __forceinline__ void ld_cols(uint32_t taddr, int row, int ncols, float *v) {
    for (int c = 0; c < ncols; c += 16) {
        tmem_ld16(lane_addr(taddr, row, c), v + c);
        tmem_ld_wait();
    }
}

// loss and gradient w.r.t. the raw outputs (internal layout of KM lobes) for
// one record
template <int D, int KM>
__device__ __forceinline__ float record_grad(const TrainArgs &a, const float *rec, const float *raw, float inv_n,
                                             float *draw) {
    constexpr int K = KM;
    Mixture<D, KM> m;
    theta_map<D, KM>(raw, m);
    const float c = a.c_mode ? a.c_fixed : m.c;
    float nu[2][3], nrm[3];
    for (int i = 0; i < 3; ++i) { nu[0][i] = rec[3 + i]; nrm[i] = rec[6 + i]; }
    const bool onN = rec[9] != 0.f;
    const float q = rec[10], pt = rec[11];
    int nd = 1;
    if (onN && a.reflect) {
        float t = 2.f * (nu[0][0] * nrm[0] + nu[0][1] * nrm[1] + (D == 3 ? nu[0][2] * nrm[2] : 0.f));
        for (int i = 0; i < D; ++i) nu[1][i] = nu[0][i] - t * nrm[i];
        nd = 2;
    }
    float v[2][KM], pg = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        float s = 0.f;
        for (int d2 = 0; d2 < nd; ++d2) {
            v[d2][j] = __expf(m.lognorm[j] - m.kappa[j] * half_dist2<D>(m.mu + j * D, nu[d2]));
            s += v[d2][j];
        }
        pg += m.lam[j] * s;
    }
    const float area = D == 2 ? 2.f * WOST_PI : 4.f * WOST_PI;
    const float pu = (onN ? 2.f : 1.f) / area;
    const float ptil = c * pg + (1.f - c) * pu;
    for (int i = 0; i < out_pad(KM); ++i) draw[i] = 0.f;
    if (!(pt > 0.f) || !(q > 0.f)) return 0.f;
    const float wt = pt / q;
    const float pgs = fmaxf(pg, 1e-30f);
    float loss = -wt * (__logf(pgs) + (a.c_mode == 0 ? a.e_sel * __logf(ptil) : 0.f));
    const float dpg = -wt / pgs * inv_n;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float *mu = m.mu + j * D;
        float sj = 0.f, dk = 0.f, dm[3] = {0.f, 0.f, 0.f};
        const float A = vmf_mean_cos<D>(m.kappa[j]);
        for (int d2 = 0; d2 < nd; ++d2) {
            float cm = 0.f;
            for (int i = 0; i < D; ++i) cm += mu[i] * nu[d2][i];
            sj += v[d2][j];
            dk += v[d2][j] * (cm - A);
            for (int i = 0; i < D; ++i) dm[i] += v[d2][j] * (nu[d2][i] - cm * mu[i]);
        }
        draw[K * D + K + j] = dpg * m.lam[j] * (sj - pg);
        float kp = raw[K * D + j];
        if (kp > -8.f && kp < 8.f) draw[K * D + j] = dpg * m.lam[j] * m.kappa[j] * dk;
        float nn = 0.f;
        for (int i = 0; i < D; ++i) nn += raw[j * D + i] * raw[j * D + i];
        if (nn > 0.f) {
            float inv = rsqrtf(nn);
            for (int i = 0; i < D; ++i) draw[j * D + i] = dpg * m.lam[j] * m.kappa[j] * dm[i] * inv;
        }
    }
    if (a.c_mode == 0) draw[K * (D + 2)] = -a.e_sel * wt * (pg - pu) / ptil * inv_n * c * (1.f - c);
    return loss;
}

template <int D, int KM>
__global__ void __launch_bounds__(train_block(KM), 1) train_kernel(TrainArgs a) {
    constexpr int TPC = train_tiles(KM), OUT = out_pad(KM), GC = gcols(KM), Z2 = z2col(KM), S0C = s0cols(KM);
    constexpr int kImg = wimg_bytes(KM), kTileB = tile_bytes(KM);
    extern __shared__ __align__(1024) uint8_t sm[];
    const int tid = threadIdx.x, tl = tid >> 7, row = tid & 127;
    const bool issuer = row == 0;
    uint8_t *wimg = sm;
    uint8_t *tb = sm + kImg + tl * kTileB;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + kImg + TPC * kTileB);
    uint32_t *tptr = reinterpret_cast<uint32_t *>(mbar + 2);
    uint32_t *copy_off = tptr + 2;   // [kMaxLevels]: this CTA's gradient copy of each level (entries)
    if (tid < kMaxLevels)
        copy_off[tid] = tid < a.f.L ? (uint32_t)((blockIdx.x % a.gc.copy_R[tid]) * a.gc.copy_V[tid]) : 0u;
    for (int i = tid; i < kImg / 16; i += train_block(KM)) reinterpret_cast<uint4 *>(wimg)[i] = __ldg(a.f.wimg + i);
    if (tid == 0) { mbar_init(&mbar[0], 1); mbar_init(&mbar[1], 1); fence_mbar_init(); }
    if (tid < 32) tmem_alloc(tptr, 512);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // TMEM of a tile: s0 (S0C columns), then the accumulators of dW3, dW2, dW1
    const uint32_t tb0 = *tptr + (uint32_t)(tl * (S0C + 3 * 64));
    TTile t{tb, tb + kTX, tb + kTX + kTH, tb + kTX + 2 * kTH, tb + kTX + 2 * kTH + tg_bytes(KM), wimg, &mbar[tl],
            tb0, tb0 + S0C, tb0 + S0C + 64, tb0 + S0C + 128, 0u, 1 + tl};

    // the records this step uses: all of them, or the stratum o, o + k, ...
    // of about max_samples records (k = ceil(n / max_samples), o from the
    // Adam step count)
    const long long nall = (long long)min((unsigned long long)a.rec_cap, *a.rec_ctr);
    long long kstride = 1, off = 0, nrec = nall;
    if (a.max_samples > 0 && nall > a.max_samples) {
        kstride = (nall + a.max_samples - 1) / a.max_samples;
        off = a.off_fixed >= 0 ? a.off_fixed % kstride
                               : (long long)((*a.step * 2654435761ull) % (unsigned long long)kstride);
        nrec = (nall - off + kstride - 1) / kstride;
    }
    if (blockIdx.x == 0 && tid == 0) *a.used = (unsigned long long)nrec;
    const float inv_n = nrec > 0 ? 1.f / (float)nrec : 0.f;
    const long long ntiles = (nrec + 127) / 128;
    bool have_acc = false, ok = true;
    float db3 = 0.f;      // column `row` (< OUT) of the bias gradient
    double loss_local = 0.0;

    for (long long tile = (long long)blockIdx.x * TPC + tl; tile < ntiles && ok; tile += (long long)gridDim.x * TPC) {
        const long long ri = off + (tile * 128 + row) * kstride;
        const bool valid = tile * 128 + row < nrec;
        float rec[12];
        if (valid) {
            const float4 *p = reinterpret_cast<const float4 *>(a.rec + ri * 12);
            float4 r0 = __ldg(p), r1 = __ldg(p + 1), r2 = __ldg(p + 2);
            rec[0] = r0.x; rec[1] = r0.y; rec[2] = r0.z; rec[3] = r0.w;
            rec[4] = r1.x; rec[5] = r1.y; rec[6] = r1.z; rec[7] = r1.w;
            rec[8] = r2.x; rec[9] = r2.y; rec[10] = r2.z; rec[11] = r2.w;
            encode_row<D>(a.f, rec, t.X, row);
        } else {
            for (int i = 0; i < 12; ++i) rec[i] = 0.f;
            for (int c = 0; c < kFeat; c += 8) *reinterpret_cast<uint4 *>(t.X + cm_offset(row, c, kFeat)) = make_uint4(0, 0, 0, 0);
        }
        // ---- forward recomputation ----
        ok = tt_issue_wait(t, issuer, [&] { umma_gemm(t.s0, t.X, 0, kFeat, t.w, 0, kFeat, kHid, kFeat, false); }, a.err);
        if (!ok) break;
        float h[kHid];
        ld_cols(t.s0, row, kHid, h);
        for (int c = 0; c < kHid; c += 8) {
            float v8[8];
            for (int i = 0; i < 8; ++i) v8[i] = fmaxf(h[c + i], 0.f);
            st_row8_bf16(t.H1, row, c, kHid, v8);
        }
        ok = tt_issue_wait(t, issuer, [&] { umma_gemm(t.s0, t.H1, 0, kHid, t.w + kW1Bytes, 0, kHid, kHid, kHid, false); }, a.err);
        if (!ok) break;
        ld_cols(t.s0, row, kHid, h);
        for (int c = 0; c < kHid; c += 8) {
            float v8[8];
            for (int i = 0; i < 8; ++i) v8[i] = fmaxf(h[c + i], 0.f);
            st_row8_bf16(t.H2, row, c, kHid, v8);
        }
        ok = tt_issue_wait(t, issuer, [&] { umma_gemm(t.s0, t.H2, 0, kHid, t.w + kW1Bytes + kW2Bytes, 0, kHid, OUT, kHid, false); }, a.err);
        if (!ok) break;
        float raw[OUT];
        ld_cols(t.s0, row, OUT, raw);
        for (int i = 0; i < OUT; ++i) raw[i] += __ldg(a.f.b3 + i);
        // ---- loss gradient at the raw outputs ----
        float dy[OUT];
        if (valid) loss_local += record_grad<D, KM>(a, rec, raw, inv_n, dy);
        else for (int i = 0; i < OUT; ++i) dy[i] = 0.f;
        if (a.loss_only) continue;   // uniform over the tile: no backward pass
        for (int c = 0; c < OUT; c += 8) st_row8_split(t.G, t.Gl, row, c, GC, dy + c);
        {
            float z8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            for (int c = OUT; c < Z2; c += 8) {
                st_row8_bf16(t.G, row, c, GC, z8);
                st_row8_bf16(t.Gl, row, c, GC, z8);
            }
        }
        // dH2 = dY W3 (W3 image rows = outputs = K here -> MN-major B)
        ok = tt_issue_wait(t, issuer, [&] {
            const uint8_t *W3 = t.w + kW1Bytes + kW2Bytes;
            umma_gemm(t.s0, t.G, 0, GC, W3, 1, kHid, kHid, OUT, false);
            umma_gemm(t.s0, t.Gl, 0, GC, W3, 1, kHid, kHid, OUT, true);
        }, a.err);
        if (!ok) break;
        // bias gradient: column sums of the dY tiles (hi + lo, what the MMAs see)
        if (row < OUT) {
            float s = 0.f;
            for (int r = 0; r < 128; ++r)
                s += __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(t.G + cm_offset(r, row, GC))) +
                     __bfloat162float(*reinterpret_cast<const __nv_bfloat16 *>(t.Gl + cm_offset(r, row, GC)));
            db3 += s;
        }
        ld_cols(t.s0, row, kHid, h);
        {
            float h2[kHid];
            for (int c = 0; c < kHid; c += 8) ld_row8_bf16(t.H2, row, c, kHid, h2 + c);
            for (int c = 0; c < kHid; c += 8) {
                float v8[8];
                for (int i = 0; i < 8; ++i) v8[i] = h2[c + i] > 0.f ? h[c + i] : 0.f;
                st_row8_split(t.G, t.Gl, row, Z2 + c, GC, v8);
            }
        }
        // dW3 (+)= [dY|..]^T H2 over G's first 128 columns (rows 0..OUT-1 used);
        // dH1 = dZ2 W2
        ok = tt_issue_wait(t, issuer, [&] {
            umma_gemm(t.acc3, t.G, 1, GC, t.H2, 1, kHid, kHid, 128, have_acc);
            umma_gemm(t.acc3, t.Gl, 1, GC, t.H2, 1, kHid, kHid, 128, true);
            umma_gemm(t.s0, t.G + cm_offset(0, Z2, GC), 0, GC, t.w + kW1Bytes, 1, kHid, kHid, kHid, false);
            umma_gemm(t.s0, t.Gl + cm_offset(0, Z2, GC), 0, GC, t.w + kW1Bytes, 1, kHid, kHid, kHid, true);
        }, a.err);
        if (!ok) break;
        ld_cols(t.s0, row, kHid, h);
        {
            float h1[kHid];
            for (int c = 0; c < kHid; c += 8) ld_row8_bf16(t.H1, row, c, kHid, h1 + c);
            for (int c = 0; c < kHid; c += 8) {
                float v8[8];
                for (int i = 0; i < 8; ++i) v8[i] = h1[c + i] > 0.f ? h[c + i] : 0.f;
                st_row8_split(t.G, t.Gl, row, c, GC, v8);
            }
        }
        // dW2 (+)= G[:, Z2-64 .. Z2+64)^T H1 (rows 64..127 = dZ2^T H1), dW1 (+)=
        // G[:, 0..128)^T X (rows 0..63 = dZ1^T X), dX = dZ1 W1
        ok = tt_issue_wait(t, issuer, [&] {
            umma_gemm(t.acc2, t.G + cm_offset(0, Z2 - 64, GC), 1, GC, t.H1, 1, kHid, kHid, 128, have_acc);
            umma_gemm(t.acc2, t.Gl + cm_offset(0, Z2 - 64, GC), 1, GC, t.H1, 1, kHid, kHid, 128, true);
            umma_gemm(t.acc1, t.G, 1, GC, t.X, 1, kFeat, kFeat, 128, have_acc);
            umma_gemm(t.acc1, t.Gl, 1, GC, t.X, 1, kFeat, kFeat, 128, true);
            umma_gemm(t.s0, t.G, 0, GC, t.w, 1, kFeat, kFeat, kHid, false);
            umma_gemm(t.s0, t.Gl, 0, GC, t.w, 1, kFeat, kFeat, kHid, true);
        }, a.err);
        if (!ok) break;
        have_acc = true;
        {
            float dx[kFeat];
            ld_cols(t.s0, row, kFeat, dx);   // warp-uniform TMEM load
            if (valid) {
                float u[D];
                unit_coords<D>(a.f, rec, u);
                for (int l = 0; l < a.f.L; ++l) {
                    uint32_t idx[1 << D];
                    float w[1 << D];
                    level_corners<D>(a.f, l, u, idx, w);
                    const size_t lo = (size_t)a.f.level_off[l] + copy_off[l];
                    for (int m = 0; m < (1 << D); ++m) {
                        float *gp = a.g_grid + (lo + idx[m]) * 2;
                        atomicAdd(reinterpret_cast<float2 *>(gp), make_float2(w[m] * dx[2 * l], w[m] * dx[2 * l + 1]));
                    }
                }
            }
        }
    }
    // flush TMEM accumulators (each warp reads its own 32 lanes)
    if (have_acc && ok) {
        // TMEM loads are warp-collective: every lane loads, then stores conditionally
        float v[kHid];
        ld_cols(t.acc3, row, kHid, v);
        // internal output row -> exchange row (padding and disabled lobes: none)
        const int er = row < OUT ? out_row_to_exchange(row, a.f.dim, a.f.K, KM) : -1;
        if (er >= 0) for (int i = 0; i < kHid; ++i) atomicAdd(a.g_W3 + (size_t)er * kHid + i, v[i]);
        ld_cols(t.acc2, row, kHid, v);
        if (row >= 64) for (int i = 0; i < kHid; ++i) atomicAdd(a.g_W2 + (size_t)(row - 64) * kHid + i, v[i]);
        ld_cols(t.acc1, row, kFeat, v);
        if (row < 64) for (int i = 0; i < kFeat; ++i) atomicAdd(a.g_W1 + (size_t)row * kFeat + i, v[i]);
        if (er >= 0) atomicAdd(a.g_b3 + er, db3);
    }
    // loss: warp reduction then one atomic per warp
    for (int o = 16; o; o >>= 1) loss_local += __shfl_xor_sync(0xffffffffu, loss_local, o);
    if ((tid & 31) == 0) atomicAdd(a.loss_acc, loss_local);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid < 32) tmem_dealloc(*tptr, 512);
}

// Adam on a flat FP32 array
// Adam (Kingma & Ba) over the grid and the MLP parameters in one launch:
// blocks [0, nb_grid) update the grid, the rest the MLP; the step count t is
// read from the device (advanced by adam_tick_kernel just before)
struct AdamGroup {
    float *p;
    const float *g;
    float *m, *v;
    int64_t n;
    float lr;
};

__global__ void adam_tick_kernel(unsigned long long *t) { *t += 1; }

// Four elements per thread (16-byte accesses; the arrays are separate
// allocations, so 16-byte aligned); the grid group also writes the FP16
// inference copy of the entries it updated (grid16[e] = features 2e, 2e + 1).
constexpr int kAdamBlock = 256;
constexpr int kAdamPer = 4;

__device__ __forceinline__ float adam_one(float &p, float g, float &m, float &v, float b1, float b2, float c1,
                                          float c2, float lr, float eps) {
    m = b1 * m + (1.f - b1) * g;
    v = b2 * v + (1.f - b2) * g * g;
    p -= lr * (m / c1) / (sqrtf(v / c2) + eps);
    return p;
}

__global__ void __launch_bounds__(kAdamBlock) adam_kernel(AdamGroup ga, AdamGroup gb, int nb_a, float b1, float b2,
                                                          float eps, const unsigned long long *t_dev,
                                                          __half2 *grid16) {
    __shared__ float corr[2];
    if (threadIdx.x == 0) {
        const float t = (float)*t_dev;
        corr[0] = 1.f - powf(b1, t);
        corr[1] = 1.f - powf(b2, t);
    }
    __syncthreads();
    const float c1 = corr[0], c2 = corr[1];
    const bool first = (int)blockIdx.x < nb_a;
    const AdamGroup &G = first ? ga : gb;
    const int64_t i = ((int64_t)(first ? blockIdx.x : blockIdx.x - nb_a) * blockDim.x + threadIdx.x) * kAdamPer;
    if (i >= G.n) return;
    if (i + kAdamPer <= G.n) {
        float4 p = *reinterpret_cast<const float4 *>(G.p + i), g = *reinterpret_cast<const float4 *>(G.g + i);
        float4 m = *reinterpret_cast<const float4 *>(G.m + i), v = *reinterpret_cast<const float4 *>(G.v + i);
        adam_one(p.x, g.x, m.x, v.x, b1, b2, c1, c2, G.lr, eps);
        adam_one(p.y, g.y, m.y, v.y, b1, b2, c1, c2, G.lr, eps);
        adam_one(p.z, g.z, m.z, v.z, b1, b2, c1, c2, G.lr, eps);
        adam_one(p.w, g.w, m.w, v.w, b1, b2, c1, c2, G.lr, eps);
        *reinterpret_cast<float4 *>(G.p + i) = p;
        *reinterpret_cast<float4 *>(G.m + i) = m;
        *reinterpret_cast<float4 *>(G.v + i) = v;
        if (first) {
            grid16[i / 2] = __floats2half2_rn(p.x, p.y);
            grid16[i / 2 + 1] = __floats2half2_rn(p.z, p.w);
        }
        return;
    }
    // the ragged end (the grid holds an even number of floats)
    float q[kAdamPer];
    const int r = (int)(G.n - i);
    for (int j = 0; j < r; ++j) q[j] = adam_one(G.p[i + j], G.g[i + j], G.m[i + j], G.v[i + j], b1, b2, c1, c2, G.lr, eps);
    if (first)
        for (int j = 0; j + 1 < r; j += 2) grid16[(i + j) / 2] = __floats2half2_rn(q[j], q[j + 1]);
}

__global__ void grid_to_half_kernel(const float *g32, __half2 *g16, int64_t n) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) g16[i] = __floats2half2_rn(g32[2 * i], g32[2 * i + 1]);
}

// FP32 MLP master (exchange layout) -> BF16 core-matrix weight image + padded
// bias, in the internal output layout of KM lobes
template <int KM>
__global__ void weight_image_kernel(const float *mlp, int nout, int dim, int K, uint8_t *img, float *b3pad) {
    constexpr int OUT = out_pad(KM);
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    const float *W1 = mlp, *W2 = W1 + kHid * kFeat, *W3 = W2 + kHid * kHid, *b3 = W3 + nout * kHid;
    __nv_bfloat16 *o = reinterpret_cast<__nv_bfloat16 *>(img);
    if (i < kHid * kFeat) {
        int r = i / kFeat, c = i % kFeat;
        o[cm_offset(r, c, kFeat) / 2] = __float2bfloat16_rn(W1[i]);
    }
    if (i < kHid * kHid) {
        int r = i / kHid, c = i % kHid;
        o[(kW1Bytes + cm_offset(r, c, kHid)) / 2] = __float2bfloat16_rn(W2[i]);
    }
    if (i < OUT * kHid) {
        int r = i / kHid, c = i % kHid;
        const int er = out_row_to_exchange(r, dim, K, KM);
        float val = er >= 0 ? W3[er * kHid + c] : 0.f;
        o[(kW1Bytes + kW2Bytes + cm_offset(r, c, kHid)) / 2] = __float2bfloat16_rn(val);
    }
    if (i < OUT) {
        const int er = out_row_to_exchange(i, dim, K, KM);
        b3pad[i] = er >= 0 ? b3[er] : (is_off_lambda(i, dim, K, KM) ? kOffLambda : 0.f);
    }
}

// BF16 weight image and padded bias from the FP32 MLP masters
static wost_status refresh_weight_image(wost_field *f, cudaStream_t st) {
    constexpr int n8 = kHid * std::max(kHid, out_pad(kMaxK)), n16 = kHid * std::max(kHid, out_pad(kMaxKWide));
    if (f->km == kMaxK)
        weight_image_kernel<kMaxK><<<(n8 + 255) / 256, 256, 0, st>>>(f->mlp32, f->nout, f->desc.dim, f->desc.K,
                                                                     f->wimg, f->b3pad);
    else
        weight_image_kernel<kMaxKWide><<<(n16 + 255) / 256, 256, 0, st>>>(f->mlp32, f->nout, f->desc.dim,
                                                                          f->desc.K, f->wimg, f->b3pad);
    WOST_CUDA(cudaGetLastError());
    return WOST_OK;
}

wost_status refresh_inference_copy(wost_field *f, cudaStream_t st) {
    const int64_t ne = f->level_off[f->desc.levels];   // lattice entries of all levels (either encoding)
    grid_to_half_kernel<<<(int)((ne + 255) / 256), 256, 0, st>>>(f->grid32, f->grid16, ne);
    WOST_CUDA(cudaGetLastError());
    return refresh_weight_image(f, st);
}

// sums each privatised level's gradient copies into copy 0 and clears the
// others (one thread per used entry of those levels)
__global__ void priv_reduce_kernel(float2 *g, GradCopies gc) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= gc.start[gc.n]) return;
    int k = 0;
    while (e >= gc.start[k + 1]) ++k;
    const int V = gc.V[k], R = gc.R[k];
    float2 *base = g + gc.off[k] + (e - gc.start[k]);
    float2 acc = base[0];
    for (int c = 1; c < R; ++c) {
        const float2 v = base[(size_t)c * V];
        acc.x += v.x;
        acc.y += v.y;
        base[(size_t)c * V] = make_float2(0.f, 0.f);
    }
    base[0] = acc;
}

static GradCopies grad_copies(const wost_field *f) {
    GradCopies gc{};
    const int L = f->desc.levels, d = f->desc.dim;
    for (int l = 0; l < kMaxLevels; ++l) { gc.copy_V[l] = 1; gc.copy_R[l] = 1; }
    gc.start[0] = 0;
    for (int l = 0; l < L; ++l) {
        if (!((f->dense_mask >> l) & 1u)) continue;
        const int64_t V = (int64_t)std::pow((double)f->res[l] + 1.0, d) + 0.5;
        const int64_t slot = f->level_off[l + 1] - f->level_off[l];
        const int R = (int)std::min<int64_t>(kGradCopies, V > 0 ? slot / V : 1);
        if (R < 2 || V > WOST_GRAD_COPY_MAXV) continue;
        gc.copy_V[l] = (int)V;
        gc.copy_R[l] = R;
        gc.lvl[gc.n] = l;
        gc.off[gc.n] = (unsigned long long)f->level_off[l];
        gc.V[gc.n] = (int)V;
        gc.R[gc.n] = R;
        gc.start[gc.n + 1] = gc.start[gc.n] + (int)V;
        ++gc.n;
    }
    return gc;
}

// kernels one training step launches: gradient (and the copy reduction),
// Adam step count, Adam with the FP16 grid copy, BF16 weight image
int train_step_launches(const wost_field *f) { return 4 + (grad_copies(f).n > 0 ? 1 : 0); }

// one-time kernel attributes (also called before a stream capture, where
// the launches follow without further set-up)
wost_status train_prepare(int dim) {
    if (dim != 2 && dim != 3) return WOST_ERR_INVALID_ARG;
    return once_per_device(200 + dim, [&]() -> wost_status {
        const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
        constexpr int s8 = train_smem(kMaxK), s16 = train_smem(kMaxKWide);
        if (dim == 2) {
            WOST_CUDA(cudaFuncSetAttribute(train_kernel<2, kMaxK>, at, s8));
            WOST_CUDA(cudaFuncSetAttribute(train_kernel<2, kMaxKWide>, at, s16));
        } else {
            WOST_CUDA(cudaFuncSetAttribute(train_kernel<3, kMaxK>, at, s8));
            WOST_CUDA(cudaFuncSetAttribute(train_kernel<3, kMaxKWide>, at, s16));
        }
        return WOST_OK;
    });
}

// gradient of the mean loss over the record buffer into f->grid_g / f->mlp_g
// (loss_only: the loss alone, the gradient buffers untouched)
wost_status train_grad_launch(wost_field *f, int dim, cudaStream_t st, long long off, bool loss_only = false) {
    if (!loss_only) {
        WOST_CUDA(cudaMemsetAsync(f->grid_g, 0, f->n_grid() * sizeof(float), st));
        WOST_CUDA(cudaMemsetAsync(f->mlp_g, 0, f->n_mlp() * sizeof(float), st));
    }
    WOST_CUDA(cudaMemsetAsync(f->loss_acc, 0, sizeof(double), st));
    TrainArgs a{};
    a.f = f->dev();
    a.rec = f->rec;
    a.rec_ctr = f->rec_ctr;
    a.rec_cap = f->rec_cap;
    a.c_mode = f->t_c_mode;
    a.c_fixed = f->t_c_fixed;
    a.reflect = f->t_reflect;
    a.e_sel = f->desc.e_sel;
    a.g_grid = f->grid_g;
    a.g_W1 = f->mlp_g;
    a.g_W2 = a.g_W1 + kHid * kFeat;
    a.g_W3 = a.g_W2 + kHid * kHid;
    a.g_b3 = a.g_W3 + (size_t)f->nout * kHid;
    a.loss_acc = reinterpret_cast<double *>(f->loss_acc);
    a.max_samples = f->t_samples;
    a.off_fixed = off;
    a.step = f->adam_step();
    a.used = f->used_records();
    a.loss_only = loss_only ? 1 : 0;
    a.err = device_err_flag();
    a.gc = grad_copies(f);
    // one CTA per SM: each CTA holds all 512 TMEM columns of its SM
    wost_status rc = train_prepare(dim);
    if (rc != WOST_OK) return rc;
    constexpr int b8 = train_block(kMaxK), b16 = train_block(kMaxKWide);
    constexpr int s8 = train_smem(kMaxK), s16 = train_smem(kMaxKWide);
    if (f->km == kMaxK) {
        if (dim == 2) train_kernel<2, kMaxK><<<num_sms(), b8, s8, st>>>(a);
        else train_kernel<3, kMaxK><<<num_sms(), b8, s8, st>>>(a);
    } else {
        if (dim == 2) train_kernel<2, kMaxKWide><<<num_sms(), b16, s16, st>>>(a);
        else train_kernel<3, kMaxKWide><<<num_sms(), b16, s16, st>>>(a);
    }
    if (!loss_only && a.gc.n > 0)
        priv_reduce_kernel<<<(a.gc.start[a.gc.n] + 255) / 256, 256, 0, st>>>(reinterpret_cast<float2 *>(f->grid_g), a.gc);
    WOST_CUDA(cudaGetLastError());
    return WOST_OK;
}

__global__ void loss_out_kernel(const double *acc, float *out) {
    unsigned long long n = reinterpret_cast<const unsigned long long *>(acc)[2];
    *out = n > 0 ? (float)(acc[0] / (double)n) : 0.f;
}

// mean loss of the step's records, written to a device float on the stream
wost_status train_loss_launch(wost_field *f, int dim, cudaStream_t st, float *out_dev) {
    wost_status rc = train_grad_launch(f, dim, st, -1, true);
    if (rc != WOST_OK) return rc;
    if (out_dev) loss_out_kernel<<<1, 1, 0, st>>>(reinterpret_cast<const double *>(f->loss_acc), out_dev);
    WOST_CUDA(cudaGetLastError());
    return WOST_OK;
}

wost_status train_launch(wost_field *f, int dim, cudaStream_t st, bool apply_adam, float *, long long off) {
    wost_status rc = train_grad_launch(f, dim, st, off);
    if (rc != WOST_OK || !apply_adam) return rc;
    const wost_field_desc &d = f->desc;
    int64_t ng = f->n_grid(), nm = f->n_mlp();
    AdamGroup ga{f->grid32, f->grid_g, f->grid_m, f->grid_v, ng, d.lr_grid};
    AdamGroup gb{f->mlp32, f->mlp_g, f->mlp_m, f->mlp_v, nm, d.lr_mlp};
    constexpr int per_block = kAdamBlock * kAdamPer;
    const int nba = (int)((ng + per_block - 1) / per_block), nbb = (int)((nm + per_block - 1) / per_block);
    adam_tick_kernel<<<1, 1, 0, st>>>(f->adam_step());
    adam_kernel<<<nba + nbb, kAdamBlock, 0, st>>>(ga, gb, nba, d.beta1, d.beta2, d.adam_eps, f->adam_step(),
                                                  f->grid16);
    WOST_CUDA(cudaGetLastError());
    return refresh_weight_image(f, st);   // the FP16 grid copy came with the update
}

// Training after a batch of wost_solve (Sec. 5.2): one Adam step on every
// record of the batch, or, with train_samples = m > 0, minibatches: the
// batch's n records in k = ceil(n / m) strata of about m records (records
// j, j + k, j + 2k, ...), one Adam step each, so every record is used once.
wost_status train_after_batch(wost_field *f, int dim, cudaStream_t st, int *steps) {
    *steps = 0;
    if (f->t_samples <= 0) {
        *steps = 1;
        return train_launch(f, dim, st, true, nullptr, -1);
    }
    unsigned long long c = 0;
    WOST_CUDA(cudaMemcpyAsync(&c, f->rec_ctr, sizeof(c), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaStreamSynchronize(st));
    const long long n = std::min<long long>((long long)c, (long long)f->rec_cap);
    const long long k = n > f->t_samples ? (n + f->t_samples - 1) / f->t_samples : 1;
    for (long long j = 0; j < k; ++j) {
        wost_status rc = train_launch(f, dim, st, true, nullptr, k > 1 ? j : -1);
        if (rc != WOST_OK) return rc;
        ++*steps;
    }
    return WOST_OK;
}

}  // namespace wost
