// The warp-specialised guided walk (Sec. 4), written once against a job
// source (jobsrc.cuh): one scene per launch (wost_solve) or many scenes with
// a field each (wost_solve_batch).
//
// Per step the walk's position is encoded by the hash grid and decoded by
// the MLP on tcgen05 tensor cores into a vMF mixture and a selection
// probability (Sec. 4.2, Tab. reg_map); the direction is drawn by one-sample
// MIS between the mixture and the uniform sphere (Sec. 4.4, Eq. mis_pdf),
// reflected below the tangent plane at Neumann points (Sec. 4.3), and
// weighted by 1 / (|S| alpha p~) (Sec. 4.1).  Training records (Sec. 5.2):
// each guided step of a recorded walk stores (x, nu, n, p~, weight, source
// term) in a per-thread scratch row; when the walk ends a suffix pass turns
// them into targets |<u(x_{k+1})>| (Sec. 4.1 Eq. guiding_dist) and appends
// them to the field's record buffer.
//
// One CTA per SM:
//   warps 0-3  (server): issue the three tcgen05 MMAs of a decode tile and run
//              the TMEM epilogues (warp q owns TMEM lanes 32q..32q+31);
//   warps 4-.. (walkers): one walk per thread; per step each walker warp runs
//              its geometry, claims a 32-row quarter of a decode tile, writes
//              its features, and waits only for that tile.
// Tiles are formed from whichever walker warps are ready (quarters are claimed
// in order from a shared counter) over kNT tile buffers: mbarriers `full`
// (4 quarter arrivals) and `done` (one per quarter), and per buffer a count
// of consumed quarters.  A claimant of tile T reuses buffer T % kNT only once
// all 4 (T / kNT) quarters of its earlier tiles are consumed: tiles can be
// consumed out of order (a walker holds its row while its geometry runs), so
// a parity wait on a barrier could mistake an old phase for the one it
// needs; the monotonic count cannot.  When a tile stays partly claimed the
// server closes it (compare-and-swap on the claim counter) and zero-pads the
// missing quarters, so a few remaining walkers never wait for partners that
// will not come.
// Every wait is bounded; a give-up sets the error word and ends the loops.
//
// Lobe capacity KM: the decoded rows hold the internal output layout of 8
// lobes (48 outputs, written over the dead hidden tile) or, for fields of
// 9..16 lobes, of 16 (96 outputs: 128 TMEM columns per tile buffer and a
// shared-memory region of their own); single-scene launches only.
//
// Multi-scene tiles: each row records the job of its walk.  The server runs
// the three-layer chain once per distinct job in the tile, with that job's
// weights (a small cache of weight images in shared memory, refilled from
// the job's field on a miss), and each epilogue thread keeps only the passes
// of its own row's job.  Rows are independent in a matrix product, so rows
// of other jobs only carry dead values through a pass.  Walks are handed out
// job-major, so nearly every tile holds one job and takes one pass.  The
// outputs of a pass go to a region the later passes do not write.
#pragma once
#include <climits>

#include "jobsrc.cuh"
#include "vmf.cuh"

namespace wost {

constexpr int kWsServerWarps = 4;
// Walker warps of the standard variant (640 threads, 102 registers each).
// Measured on one GB300, training batches of the bench: 2D star 58.1 /
// 55.0 / 55.2 / 57.5 / 59.5 ms with 12 / 16 / 20 / 24 / 28 walker warps,
// icosphere 403 / 340 / 335 / 341 / 334-357 ms (the latter run by the wide
// variant); fewer warps hide less latency, more impose a register cap that
// spills.
#ifndef WOST_WS_WALKERS
#define WOST_WS_WALKERS 16
#endif
#ifndef WOST_WS_TILES
#define WOST_WS_TILES 1
#endif
constexpr int kWsWalkerWarps = WOST_WS_WALKERS;
// Walker warps of the wide variant, for scenes whose traversal data misses
// L2: more walkers hide the latency of BVH loads from HBM (32 warps at 28,
// the 1024-thread limit; 64 registers per thread).
#ifndef WOST_WS_WALKERS_WIDE
#define WOST_WS_WALKERS_WIDE 28
#endif
constexpr int kWsWalkersWide = WOST_WS_WALKERS_WIDE;
static_assert(kWsServerWarps + kWsWalkersWide <= 32, "a CTA holds at most 32 warps");
// threads of a CTA with W walker warps beside the decode servers
__host__ __device__ constexpr int ws_threads(int W) { return 32 * (kWsServerWarps + W); }
constexpr int kWsThreads = ws_threads(kWsWalkerWarps);
// decode tile buffers.  Measured on one GB300: one buffer is 6% faster than
// two on the 2D star and 3-5% on the icosphere (equal on the genus-3 solid);
// three and four are slower still.  A walker warp that finds the buffer busy
// waits for the tile in flight, so tiles fill fuller and the shared memory
// the buffers do not take goes to the scene and to L1.
constexpr int kNT = WOST_WS_TILES;
// TMEM columns of a decode buffer: the 64 hidden columns, or the 96 outputs
// of a 16-lobe layout
__host__ __device__ constexpr int ws_buf_cols(int KM) { return tile_tmem_cols(KM); }
// allocation rounded up to a power of two
__host__ __device__ constexpr uint32_t ws_tmem_cols(int KM) { return tmem_cols(kNT * ws_buf_cols(KM)); }
static_assert(kNT >= 1 && kNT * ws_buf_cols(kMaxKWide) <= 512, "decode tile buffers must fit in the 512 TMEM columns");
// The `full` and `done` barriers of a buffer can never run two phases ahead
// of their waiters: a tile's quarters arrive only after the tile kNT earlier
// is consumed, which follows its `done`, which follows its `full`.
constexpr int kXTileBytes = 128 * kFeat * 2;
constexpr int kHTileBytes = 128 * kHid * 2;
// FP16 output row stride: an odd number of words, so the 32 rows of a warp
// fall in distinct banks (50 halves for 48 outputs, 98 for 96)
__host__ __device__ constexpr int ws_y_stride(int KM) { return out_pad(KM) + 2; }
__host__ __device__ constexpr int ws_y_bytes(int KM) { return 128 * ws_y_stride(KM) * 2; }
constexpr int kYStride = ws_y_stride(kMaxK);
constexpr int kYBytes = ws_y_bytes(kMaxK);   // aliases the hidden tile once layer 3 has run
static_assert(kYBytes <= kHTileBytes, "decoded outputs must fit in the hidden-activation tile");
constexpr int kBufBytes = kXTileBytes + kHTileBytes;
constexpr int kWsCtrlBytes = 512;
constexpr int kWSlots = 2;                   // weight images cached by a multi-scene CTA
constexpr int ws_weight_slots(bool multi) { return multi ? kWSlots : 1; }
// Multi-scene CTAs keep the decoded outputs in a region of their own: a
// later pass writes hidden activations of its rows in the core-matrix
// layout, which spans the bytes of other rows' row-major outputs.  So do
// 16-lobe layouts, whose 96 outputs exceed the hidden tile.
__host__ __device__ constexpr bool ws_y_separate(bool multi, int KM) { return multi || KM > kMaxK; }
__host__ __device__ constexpr int ws_smem_bytes(bool multi, int KM = kMaxK) {
    return wimg_bytes(KM) * ws_weight_slots(multi) + kNT * kBufBytes + kWsCtrlBytes + (multi ? kNT * 128 * 4 : 0) +
           (ws_y_separate(multi, KM) ? kNT * ws_y_bytes(KM) : 0);
}
// Server polls before closing a partial tile.  Fuller tiles measured faster
// (one GB300, training batches: icosphere 374 / 364 / 354 / 339-347 / 335 ms
// with 1 / 32 / 256 / 1024 / 4096 polls, genus-3 708 / 703 / 696 / 688-691 /
// 697, the 2D star 58 ms from 256 polls on and 65-67 below).
#ifndef WOST_FLUSH_POLLS
#define WOST_FLUSH_POLLS 1024
#endif
constexpr uint32_t kFlushPolls = WOST_FLUSH_POLLS;
// optional bound in time on the wait for a partial tile (0: polls only)
#ifndef WOST_FLUSH_NS
#define WOST_FLUSH_NS 0
#endif
constexpr unsigned long long kFlushNs = WOST_FLUSH_NS;
// Decode in flight during the step's geometry.  Measured on the 2D star
// workload it is slower (the terminal steps' decodes are wasted and tile
// buffers stay held through the geometry), so it is off by default.
#ifndef WOST_WS_OVERLAP
#define WOST_WS_OVERLAP 0
#endif
constexpr bool kOverlap = WOST_WS_OVERLAP != 0;

struct WsCtrl {
    uint64_t full[kNT], done[kNT][4], mma;
    unsigned consumed[kNT];   // quarters of the buffer's tiles consumed so far
    int qclaim, alive, go, padmask;
    uint32_t tmem;
    int pick, wnext;
    int wtag[kWSlots];
};
static_assert(sizeof(WsCtrl) <= kWsCtrlBytes, "control block too large");

// options of a guided launch shared by both job sources
struct WsOpts {
    int c_mode;                  // 0 learned c, 1 fixed c_fixed
    float c_fixed;
    int reflect;                 // sample reflection at Neumann points (Sec. 4.3)
    int record;                  // keep training records of this launch's walks
    float *scratch;              // [slot][scratch_steps][kRecFloats]
    int scratch_steps;
    uint32_t flush_polls;        // server polls before closing a partial tile
    unsigned long long wait_ns;  // limit of the waits on other warps (tile filled, decoded, consumed)
    int *err;
    unsigned long long *stat;
};

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" : : "r"(smem_u32(bar)) : "memory");
}

// all lanes of the calling warp poll (converged); returns false on give-up
__device__ __forceinline__ bool ws_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns) {
    return mbar_wait_bounded(bar, parity, limit_ns);
}

// until *count reaches target (monotonic); false on give-up
__device__ __forceinline__ bool wait_consumed(const unsigned *count, unsigned target, unsigned long long limit_ns) {
    if (*(volatile const unsigned *)count >= target) {
        __threadfence_block();
        return true;
    }
    const unsigned long long t0 = globaltimer_ns();
    while (*(volatile const unsigned *)count < target) {
        if (globaltimer_ns() - t0 > limit_ns) return false;
        __nanosleep(64);
    }
    __threadfence_block();
    return true;
}

__device__ __forceinline__ void zero_row(uint8_t *tile, int row, int C) {
    for (int c = 0; c < C; c += 8) *reinterpret_cast<uint4 *>(tile + cm_offset(row, c, C)) = make_uint4(0, 0, 0, 0);
}

// suffix pass of a finished recorded walk (Sec. 4.1): v_k = w_k v_{k+1} + S_k,
// target of record k = |v_{k+1}|; appends the nrec records to the buffer
// (or counts them as dropped when it is full)
__device__ __forceinline__ void end_recorded_walk(const RecDest &rd, const float *base, int nrec, float term) {
    unsigned long long at = atomicAdd(rd.ctr, (unsigned long long)nrec);
    bool keep = (long long)(at + nrec) <= rd.cap;
    if (!keep) atomicAdd(rd.ctr + 1, (unsigned long long)nrec);
    float v = term;
    for (int k = nrec - 1; k >= 0; --k) {
        const float4 *r = reinterpret_cast<const float4 *>(base + (size_t)k * kRecFloats);
        float4 a = r[0], b = r[1], c = r[2];   // x0 x1 x2 v0 | v1 v2 n0 n1 | n2 q w S
        float tgt = fabsf(v);
        v = c.z * v + c.w;
        if (keep) {
            float4 *o = reinterpret_cast<float4 *>(rd.out + (size_t)(at + k) * kRecFloats);
            float onN = (b.z != 0.f || b.w != 0.f || c.x != 0.f) ? 1.f : 0.f;
            o[0] = a;
            o[1] = b;
            o[2] = make_float4(c.x, onN, c.y, tgt);
        }
    }
}

// W walker warps (a template parameter: launches over scenes whose traversal
// data misses L2 take more walkers to hide its latency); KM: lobe capacity of
// the decoded output layout (8, or 16 for fields of 9..16 lobes; single-scene
// launches only)
template <int D, bool kMulti, int W = kWsWalkerWarps, int KM = kMaxK, class Src>
__device__ __forceinline__ void guided_ws_body(const Src &src, const WsOpts &o, uint8_t *sm) {
    static_assert(!kMulti || KM == kMaxK, "multi-scene launches decode 8-lobe layouts");
    constexpr int kThreads = ws_threads(W);
    constexpr int kSlots = ws_weight_slots(kMulti);
    constexpr int kImg = wimg_bytes(KM), OUT = out_pad(KM), YS = ws_y_stride(KM);
    constexpr uint32_t kTmemCols = ws_tmem_cols(KM);
    uint8_t *wslots = sm;
    uint8_t *bufs = sm + kSlots * kImg;
    WsCtrl *ctl = reinterpret_cast<WsCtrl *>(bufs + kNT * kBufBytes);
    int *rowjob = reinterpret_cast<int *>(bufs + kNT * kBufBytes + kWsCtrlBytes);   // [kNT][128], multi only
    // separate output region (multi-scene or 16-lobe layouts)
    uint8_t *ybufs = bufs + kNT * kBufBytes + kWsCtrlBytes + (kMulti ? kNT * 128 * 4 : 0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    auto Xb = [&](int b) { return bufs + b * kBufBytes; };
    auto Hb = [&](int b) { return bufs + b * kBufBytes + kXTileBytes; };
    // decoded raw outputs (FP16): one pass per tile overwrites the hidden
    // tile after the last MMA read it; several passes use their own region
    auto Yb = [&](int b) {
        return reinterpret_cast<__half *>(ws_y_separate(kMulti, KM) ? ybufs + b * ws_y_bytes(KM)
                                                                    : bufs + b * kBufBytes + kXTileBytes);
    };

    if (!kMulti)
        for (int i = tid; i < kImg / 16; i += kThreads)
            reinterpret_cast<uint4 *>(wslots)[i] = __ldg(src.wimg(0) + i);
    if (tid == 0) {
        for (int b = 0; b < kNT; ++b) {
            mbar_init(&ctl->full[b], 4);
            ctl->consumed[b] = 0;
            for (int q = 0; q < 4; ++q) mbar_init(&ctl->done[b][q], 1);
        }
        mbar_init(&ctl->mma, 1);
        ctl->qclaim = 0;
        ctl->alive = W;
        ctl->wnext = 0;
        for (int i = 0; i < kWSlots; ++i) ctl->wtag[i] = -1;
        fence_mbar_init();
    }
    if (warp == 0) tmem_alloc(&ctl->tmem, kTmemCols);
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
                const unsigned long long t0 = globaltimer_ns();
                for (;;) {
                    if (mbar_try_wait(&ctl->full[b], k & 1u)) { go = 1; break; }
                    if (globaltimer_ns() - t0 > o.wait_ns) break;
                    int q = *(volatile int *)&ctl->qclaim;
                    const int alive = *(volatile int *)&ctl->alive;
                    // every walker warp still running has claimed a quarter of
                    // this tile: no further claim can come before it is
                    // decoded, so close it now instead of after the poll budget
                    const bool all_in = q > 4 * T && q - 4 * T >= alive;
                    const bool late = kFlushNs > 0 && globaltimer_ns() - t0 > kFlushNs;
                    if (!all_in && !late && ++polls < o.flush_polls) continue;
                    polls = 0;
                    if (q <= 4 * T) {
                        if (alive == 0) { go = 0; break; }
                    } else if (q < 4 * T + 4 && atomicCAS(&ctl->qclaim, q, 4 * T + 4) == q) {
                        // close the tile: zero-fill the unclaimed quarters and arrive for them
                        for (int qq = q - 4 * T; qq < 4; ++qq) {
                            pad |= 1 << qq;
                            for (int r = 32 * qq; r < 32 * qq + 32; ++r) {
                                for (int c = 0; c < kFeat; c += 8)
                                    *reinterpret_cast<uint4 *>(Xb(b) + cm_offset(r, c, kFeat)) = make_uint4(0, 0, 0, 0);
                                if (kMulti) rowjob[b * 128 + r] = -1;
                            }
                        }
                        fence_async_smem();
                        for (int qq = q - 4 * T; qq < 4; ++qq) mbar_arrive(&ctl->full[b]);
                    }
                }
                if (go < 0) atomicOr(o.err, 2);
                ctl->go = go;
                ctl->padmask = pad;
            }
            named_sync(1, 128);
            const int go = ctl->go, pad = ctl->padmask;
            named_sync(1, 128);
            if (go <= 0) break;
            const uint32_t tm = tmem0 + (uint32_t)(b * ws_buf_cols(KM));
            const int rj = kMulti ? rowjob[b * 128 + row] : 0;   // -1: padding row
            bool pending = rj >= 0;
            bool ok = true;
            // one pass of the three layers per job among the tile's rows
            for (;;) {
                int pj = 0;
                const uint8_t *wimg = wslots;
                if (kMulti) {
                    // smallest job among the rows still to decode
                    if (tid == 0) ctl->pick = INT_MAX;
                    named_sync(1, 128);
                    if (pending) atomicMin(&ctl->pick, rj);
                    named_sync(1, 128);
                    pj = ctl->pick;
                    if (pj == INT_MAX) break;
                    int s = -1;
                    for (int i = 0; i < kSlots; ++i)
                        if (ctl->wtag[i] == pj) s = i;
                    if (s < 0) {
                        // no MMA is in flight between tiles and passes: any slot may be refilled
                        s = ctl->wnext;
                        named_sync(1, 128);
                        const uint4 *src_w = src.wimg(pj);
                        uint4 *dst = reinterpret_cast<uint4 *>(wslots + s * kImg);
                        for (int i = tid; i < kImg / 16; i += 128) dst[i] = __ldg(src_w + i);
                        fence_async_smem();
                        if (tid == 0) {
                            ctl->wtag[s] = pj;
                            ctl->wnext = (s + 1) % kSlots;
                        }
                        named_sync(1, 128);
                    }
                    wimg = wslots + s * kImg;
                }
                // this thread's row takes the pass; tcgen05.ld is warp-collective,
                // so a warp loads when any of its rows does
                const bool mine = !kMulti || rj == pj;
                const bool warp_mine = !kMulti || __any_sync(0xffffffffu, mine);
                // three layers: X -> H -> H -> Y (TMEM columns [tm, tm + ws_buf_cols(KM)))
                for (int layer = 0; layer < 3 && ok; ++layer) {
                    if (tid == 0) {
                        tc_fence_after();
                        if (layer == 0) umma_gemm(tm, Xb(b), 0, kFeat, wimg, 0, kFeat, kHid, kFeat, false);
                        else if (layer == 1) umma_gemm(tm, Hb(b), 0, kHid, wimg + kW1Bytes, 0, kHid, kHid, kHid, false);
                        else umma_gemm(tm, Hb(b), 0, kHid, wimg + kW1Bytes + kW2Bytes, 0, kHid, OUT, kHid, false);
                        umma_commit(&ctl->mma);
                    }
                    ok = mbar_wait_bounded(&ctl->mma, mma_phase);
                    mma_phase ^= 1u;
                    tc_fence_after();
                    ok = !named_or(1, 128, !ok);
                    if (!ok) break;
                    if (layer < 2) {
                        if (warp_mine) {
                            for (int c = 0; c < kHid; c += 16) {
                                float v[16];
                                tmem_ld16(lane_addr(tm, row, c), v);
                                tmem_ld_wait();
#pragma unroll
                                for (int i = 0; i < 16; ++i) v[i] = fmaxf(v[i], 0.f);
                                if (mine) {
                                    st_row8_bf16(Hb(b), row, c, kHid, v);
                                    st_row8_bf16(Hb(b), row, c + 8, kHid, v + 8);
                                }
                            }
                        }
                        fence_async_smem();
                        tc_fence_before();
                        named_sync(1, 128);
                    } else {
                        // the layer-3 MMA has completed: its H operand is dead, so
                        // (one pass, 8 lobes) the FP16 outputs can take its place
                        if (warp_mine) {
                            const float *b3 = src.b3(pj);
                            __half *y = Yb(b) + row * YS;
                            for (int c = 0; c < OUT; c += 16) {
                                float v[16];
                                tmem_ld16(lane_addr(tm, row, c), v);
                                tmem_ld_wait();
                                if (mine) {
#pragma unroll
                                    for (int i = 0; i < 16; i += 2)
                                        *reinterpret_cast<__half2 *>(y + c + i) = __floats2half2_rn(
                                            v[i] + __ldg(b3 + c + i), v[i + 1] + __ldg(b3 + c + i + 1));
                                }
                            }
                        }
                        tc_fence_before();
                    }
                }
                if (!kMulti || !ok) break;
                pending = pending && rj != pj;
                // TMEM of this pass read by every thread before the next MMA
                named_sync(1, 128);
            }
            if (!ok) {
                if (tid == 0) atomicOr(o.err, 2);
                break;
            }
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(&ctl->done[b][warp]);
                if (pad & (1 << warp)) atomicAdd(&ctl->consumed[b], 1u);   // no consumer for a padded quarter
            }
        }
    } else {
        // ------------------------------ walkers -----------------------------
        const int slot = blockIdx.x * (W * 32) + (tid - 32 * kWsServerWarps);
        float *scratch_row = o.scratch + (size_t)slot * o.scratch_steps * kRecFloats;
        const float area = D == 2 ? 2.f * WOST_PI : 4.f * WOST_PI;
        Walk<D> w;
        bool active = false, exhausted = false, failed = false;
        for (;;) {
            if (!active && !exhausted) {
                unsigned long long item = warp_fetch_add(src.work_ctr(), true);
                if (item >= src.total()) exhausted = true;
                else if (src.start(w, item)) { active = true; nwalks++; }
            }
            if (!__any_sync(0xffffffffu, active || !exhausted)) break;
            __syncwarp();
            float r = 0.f, S = 0.f;
            // The decode needs only the walk's position: with kOverlap the
            // row is submitted first and the step's geometry runs while the
            // tile fills and decodes (a walk that then ends leaves its row
            // unused).  Otherwise the geometry runs first and only walks that
            // go on are decoded.
            auto geometry = [&]() {
                if (active) {
                    nsteps++;
                    float gv;
                    bool trunc = false;
                    if (step_geometry<D>(w, src.env(w), r, S, gv, trunc, &vis)) {
                        src.finish(w);
                        if (o.record) end_recorded_walk(src.rec(w), scratch_row, w.k, gv);
                        ntrunc += trunc;
                        active = false;
                    }
                }
            };
            if (!kOverlap) geometry();
            const bool enc = active;
            if (!__any_sync(0xffffffffu, enc)) continue;
            // claim a quarter of a decode tile
            int qi = 0;
            if (lane == 0) qi = atomicAdd(&ctl->qclaim, 1);
            qi = __shfl_sync(0xffffffffu, qi, 0);
            const int T = qi >> 2, quarter = qi & 3, b = T % kNT;
            const uint32_t k = (uint32_t)(T / kNT);
            if (T >= kNT && !wait_consumed(&ctl->consumed[b], 4u * k, o.wait_ns)) { failed = true; break; }
            const int row = 32 * quarter + lane;
            if (enc) encode_row<D>(src.field(w), w.x, Xb(b), row);
            else zero_row(Xb(b), row, kFeat);
            if (kMulti) rowjob[b * 128 + row] = enc ? src.job(w) : -1;
            fence_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->full[b]);
            if (kOverlap) geometry();
            // reconverge before polling: lanes without a step must not spin
            // on the barrier while the others' geometry runs
            __syncwarp();
            const bool live = active;
            if (!ws_wait(&ctl->done[b][quarter], k & 1u, o.wait_ns)) { failed = true; break; }
            float nu[D];
            bool zero_density = false;
            float wgt = 1.f, ptil = 0.f;
            if (live) {
                RowMixture<D, KM> m;
                m.init(Yb(b) + row * YS);
                const float c = o.c_mode ? o.c_fixed : m.c();
                const StepEnv env = src.env(w);
                bool from_guide = sample_direction_row<D, KM>(m, c, w.pid, w.wid, (uint32_t)w.k, env.key0, env.key1, nu);
                const bool onN = w.prim >= 0;
                if (onN) {
                    float dn = dotv<D>(nu, w.n);
                    if (dn < 0.f && (o.reflect || !from_guide)) { reflect<D>(nu, w.n); dn = -dn; }
                    zero_density = dn <= 0.f;   // Eq. angular_req: the recursive term is 0
                }
                if (!zero_density) {
                    float nm[D];
                    const bool refl = onN && o.reflect;
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
            if (lane == 0) {   // tile rows consumed
                __threadfence_block();
                atomicAdd(&ctl->consumed[b], 1u);
            }
            if (live) {
                if (zero_density) {
                    src.finish(w);
                    if (o.record) end_recorded_walk(src.rec(w), scratch_row, w.k, S);
                    active = false;
                } else {
                    if (o.record) {
                        const bool onN = w.prim >= 0;
                        float4 *rr = reinterpret_cast<float4 *>(scratch_row + (size_t)w.k * kRecFloats);
                        float n2 = onN && D == 3 ? w.n[D - 1] : 0.f;
                        rr[0] = make_float4(w.x[0], w.x[1], D == 3 ? w.x[2] : 0.f, nu[0]);
                        rr[1] = make_float4(nu[1], D == 3 ? nu[2] : 0.f, onN ? w.n[0] : 0.f, onN ? w.n[1] : 0.f);
                        rr[2] = make_float4(n2, ptil, wgt * roulette_scale(src.env(w), w.k), S);
                    }
                    w.T *= wgt;
                    step_move<D>(w, src.env(w), nu, r, &vis);
                }
            }
        }
        if (failed) atomicOr(o.err, 2);
        __syncwarp();
        if (lane == 0) atomicSub(&ctl->alive, 1);
    }
    flush_stats(o.stat, nsteps, ntrunc, nwalks, vis);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem0, kTmemCols);
}

}  // namespace wost
