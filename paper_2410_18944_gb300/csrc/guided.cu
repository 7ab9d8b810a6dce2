// Guided walk on stars (Sec. 4): per step, the walk's position is encoded by
// the hash grid and decoded by the MLP on tcgen05 tensor cores into a vMF
// mixture and a selection probability (Sec. 4.2, Tab. reg_map); the
// direction is drawn by one-sample MIS between the mixture and the uniform
// sphere (Sec. 4.4, Eq. mis_pdf), reflected below the tangent plane at
// Neumann points (Sec. 4.3), and weighted by 1 / (|S| alpha p~) (Sec. 4.1).
//
// Persistent kernel, 256 threads = two 128-walk tiles per CTA sharing the
// BF16 weight image in shared memory; each tile runs its own three-layer MMA
// chain (accumulators in 64 TMEM columns, MMAs issued by one thread,
// completion through an mbarrier) between named barriers, so the two tiles
// of a CTA progress independently.  Finished walks are replaced from the
// global work counter (warp-aggregated atomics) before every step.
// Training records (Sec. 5.2): each guided step of a recorded walk stores
// (x, nu, n, p~, weight, source term) in a per-thread scratch row; when the
// walk ends a suffix pass turns them into targets |<u(x_{k+1})>|
// (Sec. 4.1 Eq. guiding_dist) and appends them to the record buffer.
#include <cstring>

#include "field.cuh"
#include "internal.h"
#include "vmf.cuh"
#include "walkstep.cuh"

namespace wost {

constexpr int kGuidedBlock = 256;
constexpr int kXTileBytes = 128 * kFeat * 2;
constexpr int kHTileBytes = 128 * kHid * 2;
constexpr int kGuidedSmem = kWImgBytes + 2 * kXTileBytes + 2 * kHTileBytes + 64;
constexpr int kRecFloats = 12;

struct GuidedArgs {
    WalkArgs w;
    DevField f;
    int c_mode;
    float c_fixed;
    int reflect;
    int record;
    float *scratch;               // [slot][maxsteps][12]
    float *rec_out;               // [cap][12]
    unsigned long long *rec_ctr;  // [0] count, [1] dropped
    long long rec_cap;
};

// shared setup of a 256-thread CTA running two MLP tiles
struct CtaTiles {
    uint8_t *wimg, *xt, *ht;
    uint64_t *mbar;
    uint32_t *tptr;
};

__device__ __forceinline__ CtaTiles cta_tiles_setup(uint8_t *sm, const DevField &f) {
    CtaTiles c;
    c.wimg = sm;
    c.xt = sm + kWImgBytes;
    c.ht = c.xt + 2 * kXTileBytes;
    c.mbar = reinterpret_cast<uint64_t *>(c.ht + 2 * kHTileBytes);
    c.tptr = reinterpret_cast<uint32_t *>(c.mbar + 2);
    const int tid = threadIdx.x;
    for (int i = tid; i < kWImgBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4 *>(c.wimg)[i] = __ldg(f.wimg + i);
    if (tid == 0) {
        mbar_init(&c.mbar[0], 1);
        mbar_init(&c.mbar[1], 1);
        fence_mbar_init();
    }
    if (tid < 32) tmem_alloc(c.tptr, 128);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return c;
}

__device__ __forceinline__ void cta_tiles_teardown(const CtaTiles &c) {
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x < 32) tmem_dealloc(*c.tptr, 128);
}

__device__ __forceinline__ void zero_row(uint8_t *tile, int row, int C) {
    for (int c = 0; c < C; c += 8) *reinterpret_cast<uint4 *>(tile + cm_offset(row, c, C)) = make_uint4(0, 0, 0, 0);
}

template <int D>
__device__ __forceinline__ void end_recorded_walk(const GuidedArgs &g, int slot, int nrec, float term) {
    float *base = g.scratch + (size_t)slot * g.w.maxsteps * kRecFloats;
    unsigned long long at = atomicAdd(g.rec_ctr, (unsigned long long)nrec);
    bool keep = (long long)(at + nrec) <= g.rec_cap;
    if (!keep) atomicAdd(g.rec_ctr + 1, (unsigned long long)nrec);
    float v = term;
    for (int k = nrec - 1; k >= 0; --k) {
        float4 *r = reinterpret_cast<float4 *>(base + (size_t)k * kRecFloats);
        float4 a = r[0], b = r[1], c = r[2];   // x0 x1 x2 v0 | v1 v2 n0 n1 | n2 q w S
        float tgt = fabsf(v);
        v = c.z * v + c.w;
        if (keep) {
            float4 *o = reinterpret_cast<float4 *>(g.rec_out + (size_t)(at + k) * kRecFloats);
            float onN = (b.z != 0.f || b.w != 0.f || c.x != 0.f) ? 1.f : 0.f;
            o[0] = a;
            o[1] = b;
            o[2] = make_float4(c.x, onN, c.y, tgt);
        }
    }
}

// ===========================================================================
// Warp-specialised guided walk.  One CTA per SM:
//   warps 0-3  (server): issue the three tcgen05 MMAs of a decode tile and run
//              the TMEM epilogues (warp q owns TMEM lanes 32q..32q+31);
//   warps 4-19 (walkers): one walk per thread; per step each walker warp runs
//              its geometry, claims a 32-row quarter of a decode tile, writes
//              its features, and waits only for that tile.
// Tiles are formed from whichever walker warps are ready (quarters are claimed
// in order from a shared counter), through rings of mbarriers over kNT tile
// buffers: full (4 quarter arrivals), done (one per quarter), empty (4
// consumer arrivals).  When a tile stays partly claimed the server closes it
// (compare-and-swap on the claim counter) and zero-pads the missing quarters,
// so a few remaining walkers never wait for partners that will not come.
// Every wait is bounded; a give-up sets the error word and ends the loops.
// ===========================================================================
constexpr int kWsServerWarps = 4;
#ifndef WOST_WS_WALKERS
#define WOST_WS_WALKERS 12
#endif
#ifndef WOST_WS_TILES
#define WOST_WS_TILES 2
#endif
constexpr int kWsWalkerWarps = WOST_WS_WALKERS;
constexpr int kWsThreads = 32 * (kWsServerWarps + kWsWalkerWarps);
constexpr int kNT = WOST_WS_TILES;           // decode tile buffers (few: leaves L1 for the BVH)
constexpr uint32_t kWsTmemCols = tmem_cols(kNT * 64);   // allocation rounded up to a power of two
static_assert(kNT >= 1 && kNT * 64 <= 512, "decode tile buffers must fit in the 512 TMEM columns");
// mbarrier parity waits only tell phase k from k+1: the tiles a buffer can
// be asked for must never run two generations ahead of its consumption.  The
// outstanding claims (one per walker warp) span at most floor((W + 2) / 4)
// tiles beyond the oldest one, and a claim in tile T waits for tile T - kNT.
static_assert((kWsWalkerWarps + 2) / 4 <= 2 * kNT - 1,
              "too many walker warps for the decode tile ring (parity waits would alias)");
constexpr int kYStride = 50;                 // FP16 output row stride (25 words: conflict-free)
constexpr int kYBytes = 128 * kYStride * 2;  // aliases the hidden tile once layer 3 has run
static_assert(kYBytes <= kHTileBytes, "decoded outputs must fit in the hidden-activation tile");
constexpr int kBufBytes = kXTileBytes + kHTileBytes;
constexpr int kWsCtrlBytes = 512;
constexpr int kWsSmem = kWImgBytes + kNT * kBufBytes + kWsCtrlBytes;
constexpr uint32_t kFlushPolls = 256;        // server polls before closing a partial tile
constexpr uint32_t kWaitLimit = 1u << 22;    // bound of every wait loop

struct WsCtrl {
    uint64_t full[kNT], done[kNT][4], empty[kNT], mma;
    int qclaim, alive, go, padmask;
    uint32_t tmem;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" : : "r"(smem_u32(bar)) : "memory");
}

// all lanes of the calling warp poll; returns false on give-up
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity) {
    for (uint32_t i = 0; i < kWaitLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

template <int D>
__global__ void __launch_bounds__(kWsThreads, 1) guided_walk_kernel(GuidedArgs g) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const WalkArgs &a = g.w;
    uint8_t *wimg = sm;
    uint8_t *bufs = sm + kWImgBytes;
    WsCtrl *ctl = reinterpret_cast<WsCtrl *>(sm + kWImgBytes + kNT * kBufBytes);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto Xb = [&](int b) { return bufs + b * kBufBytes; };
    auto Hb = [&](int b) { return bufs + b * kBufBytes + kXTileBytes; };
    // decoded raw outputs (FP16) overwrite the hidden tile after the last MMA read it
    auto Yb = [&](int b) { return reinterpret_cast<__half *>(bufs + b * kBufBytes + kXTileBytes); };

    for (int i = tid; i < kWImgBytes / 16; i += kWsThreads) reinterpret_cast<uint4 *>(wimg)[i] = __ldg(g.f.wimg + i);
    if (tid == 0) {
        for (int b = 0; b < kNT; ++b) {
            mbar_init(&ctl->full[b], 4);
            mbar_init(&ctl->empty[b], 4);
            for (int q = 0; q < 4; ++q) mbar_init(&ctl->done[b][q], 1);
        }
        mbar_init(&ctl->mma, 1);
        ctl->qclaim = 0;
        ctl->alive = kWsWalkerWarps;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&ctl->tmem, kWsTmemCols);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem0 = ctl->tmem;

    Visits vis;
    unsigned long long nsteps = 0, ntrunc = 0, nwalks = 0;

    if (warp < kWsServerWarps) {
        // ------------------------------ server ------------------------------
        uint32_t mma_phase = 0;
        const int row = tid;   // TMEM lane of this thread (warp q owns 32q..32q+31)
        for (int T = 0;; ++T) {
            const int b = T % kNT;
            const uint32_t k = (uint32_t)(T / kNT);
            if (tid == 0) {
                int go = -1, pad = 0;
                uint32_t polls = 0;
                for (uint32_t it = 0; it < kWaitLimit; ++it) {
                    if (mbar_try_wait(&ctl->full[b], k & 1u)) { go = 1; break; }
                    if (++polls < kFlushPolls) continue;
                    polls = 0;
                    int q = *(volatile int *)&ctl->qclaim;
                    if (q <= 4 * T) {
                        if (*(volatile int *)&ctl->alive == 0) { go = 0; break; }
                    } else if (q < 4 * T + 4 && atomicCAS(&ctl->qclaim, q, 4 * T + 4) == q) {
                        // close the tile: zero-fill the unclaimed quarters and arrive for them
                        for (int qq = q - 4 * T; qq < 4; ++qq) {
                            pad |= 1 << qq;
                            for (int r = 32 * qq; r < 32 * qq + 32; ++r)
                                for (int c = 0; c < kFeat; c += 8)
                                    *reinterpret_cast<uint4 *>(Xb(b) + cm_offset(r, c, kFeat)) = make_uint4(0, 0, 0, 0);
                        }
                        fence_async_smem();
                        for (int qq = q - 4 * T; qq < 4; ++qq) mbar_arrive(&ctl->full[b]);
                    }
                }
                if (go < 0) atomicOr(a.err, 2);
                ctl->go = go;
                ctl->padmask = pad;
            }
            named_sync(1, 128);
            const int go = ctl->go, pad = ctl->padmask;
            named_sync(1, 128);
            if (go <= 0) break;
            const uint32_t tm = tmem0 + (uint32_t)(b * 64);
            bool ok = true;
            // three layers: X -> H -> H -> Y (TMEM columns [b*64, b*64 + 64))
            for (int layer = 0; layer < 3 && ok; ++layer) {
                if (tid == 0) {
                    tc_fence_after();
                    if (layer == 0) umma_gemm(tm, Xb(b), 0, kFeat, wimg, 0, kFeat, kHid, kFeat, false);
                    else if (layer == 1) umma_gemm(tm, Hb(b), 0, kHid, wimg + kW1Bytes, 0, kHid, kHid, kHid, false);
                    else umma_gemm(tm, Hb(b), 0, kHid, wimg + kW1Bytes + kW2Bytes, 0, kHid, kOutPad, kHid, false);
                    umma_commit(&ctl->mma);
                }
                ok = mbar_wait_bounded(&ctl->mma, mma_phase, kWaitLimit);
                mma_phase ^= 1u;
                tc_fence_after();
                ok = !named_or(1, 128, !ok);
                if (!ok) break;
                if (layer < 2) {
                    for (int c = 0; c < kHid; c += 16) {
                        float v[16];
                        tmem_ld16(lane_addr(tm, row, c), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
                        st_row8_bf16(Hb(b), row, c, kHid, v);
                        st_row8_bf16(Hb(b), row, c + 8, kHid, v + 8);
                    }
                    fence_async_smem();
                    tc_fence_before();
                    named_sync(1, 128);
                } else {
                    // the layer-3 MMA has completed: its H operand is dead, so
                    // the FP16 outputs can take its place
                    __half *y = Yb(b) + row * kYStride;
                    for (int c = 0; c < kOutPad; c += 16) {
                        float v[16];
                        tmem_ld16(lane_addr(tm, row, c), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int i = 0; i < 16; i += 2)
                            *reinterpret_cast<__half2 *>(y + c + i) =
                                __floats2half2_rn(v[i] + __ldg(g.f.b3 + c + i), v[i + 1] + __ldg(g.f.b3 + c + i + 1));
                    }
                    tc_fence_before();
                }
            }
            if (!ok) {
                if (tid == 0) atomicOr(a.err, 2);
                break;
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&ctl->done[b][warp]);
                if (pad & (1 << warp)) mbar_arrive(&ctl->empty[b]);   // no consumer for a padded quarter
            }
        }
    } else {
        // ------------------------------ walkers -----------------------------
        const int slot = blockIdx.x * (kWsWalkerWarps * 32) + (tid - 32 * kWsServerWarps);
        const float area = D == 2 ? 2.f * WOST_PI : 4.f * WOST_PI;
        Walk<D> w;
        bool active = false, exhausted = false, failed = false;
        for (;;) {
            if (!active && !exhausted) {
                unsigned long long item = warp_fetch_add(a.work_ctr, true);
                if (item >= a.total) {
                    exhausted = true;
                } else {
                    start_walk<D>(w, a, item);
                    if (a.status[w.pid] == 0) { active = true; nwalks++; }
                }
            }
            if (!__any_sync(0xffffffffu, active || !exhausted)) break;
            __syncwarp();
            float r = 0.f, S = 0.f;
            if (active) {
                nsteps++;
                float gv;
                bool trunc = false;
                if (step_geometry<D>(w, a, r, S, gv, trunc, &vis)) {
                    finish_walk(a, w.pid, w.acc);
                    if (g.record) end_recorded_walk<D>(g, slot, w.k, gv);
                    ntrunc += trunc;
                    active = false;
                }
            }
            const bool live = active;
            if (!__any_sync(0xffffffffu, live)) continue;
            // claim a quarter of a decode tile
            int qi = 0;
            if (lane == 0) qi = atomicAdd(&ctl->qclaim, 1);
            qi = __shfl_sync(0xffffffffu, qi, 0);
            const int T = qi >> 2, quarter = qi & 3, b = T % kNT;
            const uint32_t k = (uint32_t)(T / kNT);
            if (T >= kNT && !ws_wait(&ctl->empty[b], (k - 1u) & 1u)) { failed = true; break; }
            const int row = 32 * quarter + lane;
            if (live) encode_row<D>(g.f, w.x, Xb(b), row);
            else zero_row(Xb(b), row, kFeat);
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->full[b]);
            if (!ws_wait(&ctl->done[b][quarter], k & 1u)) { failed = true; break; }
            float nu[D];
            bool zero_density = false;
            float wgt = 1.f, ptil = 0.f;
            if (live) {
                RowMixture<D, 8> m;
                m.init(Yb(b) + row * kYStride);
                const float c = g.c_mode ? g.c_fixed : m.c();
                bool from_guide = sample_direction_row<D, 8>(m, c, w.pid, w.wid, (uint32_t)w.k, a.key0, a.key1, nu);
                const bool onN = w.prim >= 0;
                if (onN) {
                    float dn = dotv<D>(nu, w.n);
                    if (dn < 0.f && (g.reflect || !from_guide)) { reflect<D>(nu, w.n); dn = -dn; }
                    zero_density = dn <= 0.f;   // Eq. angular_req: the recursive term is 0
                }
                if (!zero_density) {
                    float nm[D];
                    const bool refl = onN && g.reflect;
                    if (refl) {
#pragma unroll
                        for (int i = 0; i < D; ++i) nm[i] = nu[i];
                        reflect<D>(nm, w.n);
                    }
                    const float pg = m.pdf(nu, refl ? nm : nullptr);
                    const float alpha = onN ? 0.5f : 1.f;
                    const float pu = (onN ? 2.f : 1.f) / area;
                    ptil = c * pg + (1.f - c) * pu;
                    // |S| alpha p_u == 1 exactly, so c = 0 gives weight 1 as in plain WoSt
                    wgt = 1.f / (c * area * alpha * pg + (1.f - c));
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->empty[b]);   // tile rows consumed
            if (live) {
                if (zero_density) {
                    finish_walk(a, w.pid, w.acc);
                    if (g.record) end_recorded_walk<D>(g, slot, w.k, S);
                    active = false;
                } else {
                    if (g.record) {
                        const bool onN = w.prim >= 0;
                        float4 *rr = reinterpret_cast<float4 *>(g.scratch + ((size_t)slot * a.maxsteps + w.k) * kRecFloats);
                        float n2 = onN && D == 3 ? w.n[D - 1] : 0.f;
                        rr[0] = make_float4(w.x[0], w.x[1], D == 3 ? w.x[2] : 0.f, nu[0]);
                        rr[1] = make_float4(nu[1], D == 3 ? nu[2] : 0.f, onN ? w.n[0] : 0.f, onN ? w.n[1] : 0.f);
                        rr[2] = make_float4(n2, ptil, wgt, S);
                    }
                    w.T *= wgt;
                    step_move<D>(w, a, nu, r, &vis);
                }
            }
        }
        if (failed) atomicOr(a.err, 2);
        __syncwarp();
        if (lane == 0) atomicSub(&ctl->alive, 1);
    }
    flush_counters(a, nsteps, ntrunc, nwalks, vis);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem0, kWsTmemCols);
}

// decode of arbitrary points: the same tile forward as inside the walk
template <int D>
__global__ void __launch_bounds__(kGuidedBlock, 1) decode_kernel(DevField f, const double *pts, int64_t n,
                                                                 float *out, int nout, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    CtaTiles ct = cta_tiles_setup(sm, f);
    const int tid = threadIdx.x, tile = tid >> 7, row = tid & 127;
    TileCtx t{ct.xt + tile * kXTileBytes, ct.ht + tile * kHTileBytes, ct.wimg, &ct.mbar[tile],
              *ct.tptr + (uint32_t)(tile * 64), 0u, 1 + tile};
    for (int64_t base = (int64_t)blockIdx.x * kGuidedBlock; base < n; base += (int64_t)gridDim.x * kGuidedBlock) {
        int64_t i = base + tid;
        float x[D];
        if (i < n) {
            for (int k = 0; k < D; ++k) x[k] = (float)pts[i * D + k];
            encode_row<D>(f, x, t.xtile, row);
        } else {
            zero_row(t.xtile, row, kFeat);
        }
        float raw[kOutPad];
        if (!mlp_tile_forward(t, f, row, row == 0, raw, err)) break;
        if (i < n)
            for (int k = 0; k < nout; ++k) out[i * nout + k] = raw[k];
    }
    cta_tiles_teardown(ct);
}

// mixture pdf / samples for given (normalised) parameters
template <int D>
__global__ void mixture_eval_kernel(int K, const float *mu, const float *kap, const float *lam, const float *nu,
                                    int64_t n, float *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Mixture<D> m;
    for (int j = 0; j < 8; ++j) {
        bool on = j < K;
        for (int k = 0; k < D; ++k) m.mu[j * D + k] = on ? mu[(i * K + j) * D + k] : 0.f;
        m.kappa[j] = on ? kap[i * K + j] : 1.f;
        m.lam[j] = on ? lam[i * K + j] : 0.f;
        m.lognorm[j] = vmf_lognorm<D>(m.kappa[j]);
    }
    float v[D];
    for (int k = 0; k < D; ++k) v[k] = nu[i * D + k];
    out[i] = mixture_pdf<D, 8>(m, v);
}

template <int D>
__global__ void mixture_sample_kernel(int K, const float *mu, const float *kap, const float *lam,
                                      const uint32_t *ctr, uint32_t k0, uint32_t k1, int64_t n, float *onu,
                                      float *opdf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Mixture<D> m;
    for (int j = 0; j < 8; ++j) {
        bool on = j < K;
        for (int k = 0; k < D; ++k) m.mu[j * D + k] = on ? mu[(i * K + j) * D + k] : 0.f;
        m.kappa[j] = on ? kap[i * K + j] : 1.f;
        m.lam[j] = on ? lam[i * K + j] : 0.f;
        m.lognorm[j] = vmf_lognorm<D>(m.kappa[j]);
    }
    float v[D];
    sample_direction<D, 8>(m, 1.f, ctr[3 * i], ctr[3 * i + 1], ctr[3 * i + 2], k0, k1, v);
    for (int k = 0; k < D; ++k) onu[i * D + k] = v[k];
    opdf[i] = mixture_pdf<D, 8>(m, v);
}

wost_status train_launch(wost_field *f, int dim, cudaStream_t st, bool apply_adam, float *loss_out_dev);

int guided_ctas_per_sm() { return 1; }

// the warp-specialised walk kernel runs one CTA (640 threads) per SM
wost_status guided_occupancy(int dim, int *per_sm) {
    static bool set[4] = {false, false, false, false};
    if (!set[dim]) {
        if (dim == 2) WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmem));
        else WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmem));
        set[dim] = true;
    }
    *per_sm = 1;
    return WOST_OK;
}

wost_status launch_guided(int dim, const GuidedArgs &g, int grid, cudaStream_t st) {
    if (dim == 2) guided_walk_kernel<2><<<grid, kWsThreads, kWsSmem, st>>>(g);
    else guided_walk_kernel<3><<<grid, kWsThreads, kWsSmem, st>>>(g);
    WOST_CUDA(cudaGetLastError());
    return WOST_OK;
}

wost_status ensure_records(wost_field *f, int64_t cap, size_t scratch_bytes);

wost_status guided_solve(wost_scene *s, wost_field *f, WalkArgs &a, int nwalks, const wost_exec &ex,
                         cudaStream_t st, wost_stats *stats, int walk_begin, CallTiming &tm) {
    if (f->desc.dim != s->dim) { set_error("wost_solve: field dimension differs from the scene"); return WOST_ERR_INVALID_ARG; }
    GuidedArgs g{};
    g.f = f->dev();
    g.c_mode = ex.c_mode;
    g.c_fixed = ex.c_fixed;
    g.reflect = ex.reflect;
    f->t_c_mode = ex.c_mode;
    f->t_c_fixed = ex.c_fixed;
    f->t_reflect = ex.reflect;
    int occ = 1;
    wost_status orc = guided_occupancy(s->dim, &occ);
    if (orc != WOST_OK) return orc;
    int cps = ex.ctas_per_sm > 0 ? std::min(ex.ctas_per_sm, occ) : occ;
    int grid = num_sms() * cps;
    const bool any_train = ex.train && walk_begin < ex.train_until_wpp;
    if (any_train) {
        int64_t cap = ex.max_train_records > 0 ? ex.max_train_records : std::max<int64_t>(a.npoints * 64, 1 << 20);
        size_t scratch = (size_t)grid * (kWsWalkerWarps * 32) * (size_t)std::max(a.maxsteps, 1) * kRecFloats * sizeof(float);
        wost_status rc = ensure_records(f, cap, scratch);
        if (rc != WOST_OK) return rc;
    }
    g.scratch = f->scratch;
    g.rec_out = f->rec;
    g.rec_ctr = f->rec_ctr;
    g.rec_cap = f->rec_cap;
    int ntrain = 0;
    for (int b = 0; b < nwalks; ++b) {
        g.w = a;
        g.w.walk_begin = walk_begin + b;
        g.w.total = (unsigned long long)a.npoints;
        g.record = ex.train && (walk_begin + b) < ex.train_until_wpp;
        WOST_CUDA(cudaMemsetAsync(a.work_ctr, 0, sizeof(unsigned long long), st));
        if (g.record) WOST_CUDA(cudaMemsetAsync(f->rec_ctr, 0, 2 * sizeof(unsigned long long), st));
        g.f = f->dev();
        tm.mark(tm.walk, st);
        wost_status rc = launch_guided(s->dim, g, grid, st);
        tm.mark(tm.walk, st);
        tm.launches++;
        tm.walk_launches++;
        if (rc != WOST_OK) return rc;
        if (g.record) {
            tm.mark(tm.train, st);
            rc = train_launch(f, s->dim, st, true, nullptr);
            tm.mark(tm.train, st);
            tm.launches += 5;   // gradient, 2 x Adam, FP16 grid copy, BF16 weight image
            if (rc != WOST_OK) return rc;
            ntrain++;
        }
    }
    if (stats) {
        stats->train_steps = ntrain;
        if (ntrain) {
            unsigned long long c[2];
            WOST_CUDA(cudaMemcpyAsync(c, f->rec_ctr, sizeof(c), cudaMemcpyDeviceToHost, st));
            WOST_CUDA(cudaStreamSynchronize(st));
            stats->records = (int64_t)c[0];
            stats->records_dropped = (int64_t)c[1];
        }
    }
    return WOST_OK;
}

}  // namespace wost

using namespace wost;

extern "C" wost_status wost_field_decode(wost_field *f, const double *points, int64_t n, float *out_raw,
                                         const wost_exec *exec) {
    if (!f || n < 0 || (n > 0 && (!points || !out_raw))) { set_error("wost_field_decode: invalid argument"); return WOST_ERR_INVALID_ARG; }
    if (n == 0) return WOST_OK;
    wost_exec ex;
    if (exec) ex = *exec; else wost_exec_defaults(&ex);
    cudaStream_t st = (cudaStream_t)ex.stream;
    const int D = f->desc.dim;
    double *dp = const_cast<double *>(points);
    float *dout = out_raw;
    bool own_p = false, own_o = false;
    if (!ex.points_on_device) {
        WOST_CUDA(cudaMalloc(&dp, n * D * sizeof(double)));
        own_p = true;
        WOST_CUDA(cudaMemcpyAsync(dp, points, n * D * sizeof(double), cudaMemcpyHostToDevice, st));
    }
    if (!ex.out_on_device) {
        WOST_CUDA(cudaMalloc(&dout, n * f->nout * sizeof(float)));
        own_o = true;
    }
    int grid = (int)std::min<int64_t>((n + kGuidedBlock - 1) / kGuidedBlock, (int64_t)num_sms() * 2);
    if (D == 2) {
        WOST_CUDA(cudaFuncSetAttribute(decode_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGuidedSmem));
        decode_kernel<2><<<grid, kGuidedBlock, kGuidedSmem, st>>>(f->dev(), dp, n, dout, f->nout, device_err_flag());
    } else {
        WOST_CUDA(cudaFuncSetAttribute(decode_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kGuidedSmem));
        decode_kernel<3><<<grid, kGuidedBlock, kGuidedSmem, st>>>(f->dev(), dp, n, dout, f->nout, device_err_flag());
    }
    WOST_CUDA(cudaGetLastError());
    if (own_o) WOST_CUDA(cudaMemcpyAsync(out_raw, dout, n * f->nout * sizeof(float), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaStreamSynchronize(st));
    if (own_p) cudaFree(dp);
    if (own_o) cudaFree(dout);
    return device_check(st);
}

namespace {
wost_status mixture_common(int dim, int K, int64_t n, const float *mu, const float *kappa, const float *lambda,
                           float **dmu, float **dk, float **dl) {
    if ((dim != 2 && dim != 3) || K < 1 || K > 8 || n < 0 || (n > 0 && (!mu || !kappa || !lambda))) {
        set_error("wost_mixture: invalid argument");
        return WOST_ERR_INVALID_ARG;
    }
    WOST_CUDA(cudaMalloc(dmu, std::max<int64_t>(n, 1) * K * dim * sizeof(float)));
    WOST_CUDA(cudaMalloc(dk, std::max<int64_t>(n, 1) * K * sizeof(float)));
    WOST_CUDA(cudaMalloc(dl, std::max<int64_t>(n, 1) * K * sizeof(float)));
    WOST_CUDA(cudaMemcpy(*dmu, mu, n * K * dim * sizeof(float), cudaMemcpyHostToDevice));
    WOST_CUDA(cudaMemcpy(*dk, kappa, n * K * sizeof(float), cudaMemcpyHostToDevice));
    WOST_CUDA(cudaMemcpy(*dl, lambda, n * K * sizeof(float), cudaMemcpyHostToDevice));
    return WOST_OK;
}
}  // namespace

extern "C" wost_status wost_mixture_eval(int32_t dim, int32_t K, const float *mu, const float *kappa,
                                         const float *lambda, const float *nu, int64_t n, float *out_pdf) {
    if (n > 0 && (!nu || !out_pdf)) { set_error("wost_mixture_eval: null argument"); return WOST_ERR_INVALID_ARG; }
    float *dmu = nullptr, *dk = nullptr, *dl = nullptr, *dn = nullptr, *dout = nullptr;
    wost_status rc = mixture_common(dim, K, n, mu, kappa, lambda, &dmu, &dk, &dl);
    if (rc != WOST_OK || n == 0) { cudaFree(dmu); cudaFree(dk); cudaFree(dl); return rc; }
    cudaError_t e = cudaMalloc(&dn, n * dim * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dout, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dn, nu, n * dim * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        int bs = 128, gr = (int)((n + bs - 1) / bs);
        if (dim == 2) mixture_eval_kernel<2><<<gr, bs>>>(K, dmu, dk, dl, dn, n, dout);
        else mixture_eval_kernel<3><<<gr, bs>>>(K, dmu, dk, dl, dn, n, dout);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_pdf, dout, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dmu); cudaFree(dk); cudaFree(dl); cudaFree(dn); cudaFree(dout);
    return e == cudaSuccess ? WOST_OK : cuda_status(e, "wost_mixture_eval");
}

extern "C" wost_status wost_mixture_sample(int32_t dim, int32_t K, const float *mu, const float *kappa,
                                           const float *lambda, const uint32_t *counters, uint64_t seed,
                                           uint32_t scene_id, int64_t n, float *out_nu, float *out_pdf) {
    if (n > 0 && (!counters || !out_nu || !out_pdf)) { set_error("wost_mixture_sample: null argument"); return WOST_ERR_INVALID_ARG; }
    float *dmu = nullptr, *dk = nullptr, *dl = nullptr, *dnu = nullptr, *dpdf = nullptr;
    uint32_t *dc = nullptr;
    wost_status rc = mixture_common(dim, K, n, mu, kappa, lambda, &dmu, &dk, &dl);
    if (rc != WOST_OK || n == 0) { cudaFree(dmu); cudaFree(dk); cudaFree(dl); return rc; }
    cudaError_t e = cudaMalloc(&dc, n * 3 * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&dnu, n * dim * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&dpdf, n * sizeof(float));
    if (e == cudaSuccess) e = cudaMemcpy(dc, counters, n * 3 * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        int bs = 128, gr = (int)((n + bs - 1) / bs);
        uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32) + scene_id;
        if (dim == 2) mixture_sample_kernel<2><<<gr, bs>>>(K, dmu, dk, dl, dc, k0, k1, n, dnu, dpdf);
        else mixture_sample_kernel<3><<<gr, bs>>>(K, dmu, dk, dl, dc, k0, k1, n, dnu, dpdf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_nu, dnu, n * dim * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_pdf, dpdf, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dmu); cudaFree(dk); cudaFree(dl); cudaFree(dc); cudaFree(dnu); cudaFree(dpdf);
    return e == cudaSuccess ? WOST_OK : cuda_status(e, "wost_mixture_sample");
}
