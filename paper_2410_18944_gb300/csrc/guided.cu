// Guided walk on stars (Sec. 4) for one scene: the launch loop with the
// online training schedule (Sec. 5.2), the field decode of arbitrary points,
// and the mixture evaluation / sampling entry points.  The walk kernel itself
// is the warp-specialised body of guided_ws.cuh over a single-scene source.
#include <cstring>

#include "guided_ws.cuh"
#include "internal.h"

namespace wost {

constexpr int kGuidedBlock = 256;
constexpr int kWsSmem = ws_smem_bytes(false);
// the 16-lobe kernel's tiles take this much more shared memory (weight image
// and output region), which its scene staging gives up
constexpr int kWsSmemWideExtra = ws_smem_bytes(false, kMaxKWide) - kWsSmem;

struct GuidedArgs {
    WalkArgs w;
    DevField f;
    WsOpts o;
    RecDest rd;
    int stage_mask;    // scene regions staged in shared memory (stage_plan)
};

// Walker warps of the single-scene kernel (exec walker_warps 0): kWsWalkerWarps
// (16) when the scene's traversal data (BVH nodes, cones, primitives) fits
// comfortably in L2 or shared memory, kWsWalkersWide beside the 4 servers
// when it does not.
// Measured on one GB300, one recording round: genus-3 solid (about 300 MB of
// traversal data) 1057 ms with 12 walker warps, 964 with 14, 798 with 20,
// 729 with 24, 695 with 28 (32 warps, the 1024-thread limit); icosphere of
// 82k triangles (about 20 MB) 168, 172, 174 ms with 12, 14, 20.  More
// walkers hide the latency of BVH loads that miss L2; with the scene in L2
// the register cap they impose (64 per thread at 1024 threads, with spills)
// costs more than it hides.
#ifndef WOST_WS_WIDE_MB
#define WOST_WS_WIDE_MB 64
#endif

// KM: lobe capacity of the field's output layout (8, or 16 for 9..16 lobes,
// which run the standard walker count only)
template <int D, int W, int KM = kMaxK>
__global__ void __launch_bounds__(ws_threads(W), 1) guided_walk_kernel(const __grid_constant__ GuidedArgs g) {
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ DevScene staged;
    const DevScene *sc = &g.w.sc;
    if (g.stage_mask) {
        stage_scene(g.w.sc, staged, reinterpret_cast<float4 *>(sm + ws_smem_bytes(false, KM)), g.stage_mask);
        sc = &staged;
    }
    guided_ws_body<D, false, W, KM>(SoloSrc<D>{g.w, &g.f, g.rd, sc}, g.o, sm);
}

// bytes of the scene's traversal data (the three BVHs' nodes and primitives
// and the silhouette cones)
static size_t traversal_bytes(const DevScene &s) {
    const size_t nb = 16 * (size_t)(s.dim == 2 ? node_f4<2>() : node_f4<3>());
    const size_t pd = s.dim == 2 ? 16 : 48, ps = s.dim == 2 ? 32 : 64;
    return nb * ((size_t)s.dir.nnodes + s.neu.nnodes + s.sil.nnodes) + pd * ((size_t)s.dir.nprims + s.neu.nprims) +
           ps * (size_t)s.sil.nprims + 16 * (size_t)bvh_width(s.dim) * s.sil.nnodes;
}

// the walker-warp count of a scene's guided launches of `walks` walks
// (`req`: the caller's choice, 0 = automatic): the wide kernel where the
// scene's traversal data misses L2, or, in 3D, where a launch gives each of
// its lanes about two walks or more (3D steps are long chains of dependent
// loads that more warps hide; a launch with fewer walks leaves the wide
// kernel's lanes idle and its register cap costs more).  Measured on one
// GB300: icosphere of 82k triangles, batches of 8 walks per point (376k
// walks) 400 ms with 12 walker warps, 357 with 28; one walk per point
// (47k walks) 168 / 174 ms with 12 / 20; the 2D star equal (58 / 59 ms).
static int ws_walkers_for(const DevScene &s, int req, unsigned long long walks) {
    if (req > 0) return req;
    if (traversal_bytes(s) > ((size_t)WOST_WS_WIDE_MB << 20)) return kWsWalkersWide;
    const unsigned long long wide_lanes = (unsigned long long)num_sms() * kWsWalkersWide * 32;
    return s.dim == 3 && walks >= 2 * wide_lanes ? kWsWalkersWide : kWsWalkerWarps;
}

bool ws_walker_warps_valid(int w) { return w == 0 || w == kWsWalkerWarps || w == kWsWalkersWide; }

// fields of 9..16 lobes run the standard walker count (the only 16-lobe
// instantiation of the walk kernel)
static int ws_walkers_for_field(const DevScene &s, const wost_field *f, int req, unsigned long long walks) {
    return f->km == kMaxK ? ws_walkers_for(s, req, walks) : kWsWalkerWarps;
}

// decode of arbitrary points: the same tile forward as inside the walk
// (KM: lobe capacity of the field's internal output layout)
template <int D, int KM>
__global__ void __launch_bounds__(kGuidedBlock, 1) decode_kernel(DevField f, const double *pts, int64_t n,
                                                                 float *out, int nout, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    CtaTiles ct = cta_tiles_setup<KM>(sm, f);
    const int tid = threadIdx.x, tile = tid >> 7, row = tid & 127;
    TileCtx t{ct.xt + tile * kXTileBytes, ct.ht + tile * kHTileBytes, ct.wimg, &ct.mbar[tile],
              *ct.tptr + (uint32_t)(tile * tile_tmem_cols(KM)), 0u, 1 + tile};
    for (int64_t base = (int64_t)blockIdx.x * kGuidedBlock; base < n; base += (int64_t)gridDim.x * kGuidedBlock) {
        int64_t i = base + tid;
        float x[D];
        if (i < n) {
            for (int k = 0; k < D; ++k) x[k] = (float)pts[i * D + k];
            encode_row<D>(f, x, t.xtile, row);
        } else {
            zero_row(t.xtile, row, kFeat);
        }
        float raw[out_pad(KM)];
        if (!mlp_tile_forward<KM>(t, f, row, row == 0, raw, err)) break;
        if (i < n)
            for (int k = 0; k < nout; ++k) out[i * nout + k] = raw[exchange_to_out_row(k, D, f.K, KM)];
    }
    cta_tiles_teardown<KM>(ct);
}

// mixture pdf / samples for given (normalised) parameters: K <= KC lobes,
// the remaining KC - K with weight 0
template <int D, int KC>
__global__ void mixture_eval_kernel(int K, const float *mu, const float *kap, const float *lam, const float *nu,
                                    int64_t n, float *out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Mixture<D, KC> m;
    for (int j = 0; j < KC; ++j) {
        bool on = j < K;
        for (int k = 0; k < D; ++k) m.mu[j * D + k] = on ? mu[(i * K + j) * D + k] : 0.f;
        m.kappa[j] = on ? kap[i * K + j] : 1.f;
        m.lam[j] = on ? lam[i * K + j] : 0.f;
        m.lognorm[j] = vmf_lognorm<D>(m.kappa[j]);
    }
    float v[D];
    for (int k = 0; k < D; ++k) v[k] = nu[i * D + k];
    out[i] = mixture_pdf<D, KC>(m, v);
}

template <int D, int KC>
__global__ void mixture_sample_kernel(int K, const float *mu, const float *kap, const float *lam,
                                      const uint32_t *ctr, uint32_t k0, uint32_t k1, int64_t n, float *onu,
                                      float *opdf) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    Mixture<D, KC> m;
    for (int j = 0; j < KC; ++j) {
        bool on = j < K;
        for (int k = 0; k < D; ++k) m.mu[j * D + k] = on ? mu[(i * K + j) * D + k] : 0.f;
        m.kappa[j] = on ? kap[i * K + j] : 1.f;
        m.lam[j] = on ? lam[i * K + j] : 0.f;
        m.lognorm[j] = vmf_lognorm<D>(m.kappa[j]);
    }
    float v[D];
    sample_direction<D, KC>(m, 1.f, ctr[3 * i], ctr[3 * i + 1], ctr[3 * i + 2], k0, k1, v);
    for (int k = 0; k < D; ++k) onu[i * D + k] = v[k];
    opdf[i] = mixture_pdf<D, KC>(m, v);
}

wost_status train_launch(wost_field *f, int dim, cudaStream_t st, bool apply_adam, float *loss_out_dev,
                         long long off = -1);
wost_status train_after_batch(wost_field *f, int dim, cudaStream_t st, int *steps);
int train_step_launches(const wost_field *f);

int guided_ctas_per_sm() { return 1; }

// The warp-specialised walk kernel runs one CTA (640 or 1024 threads) per SM; its
// dynamic shared memory holds the decode tiles and as much of the scene's
// traversal data as fits (stage_plan), at most WOST_STAGE_MAX_KB.
#ifndef WOST_STAGE_MAX_KB
#define WOST_STAGE_MAX_KB 1024
#endif

// bytes of dynamic shared memory beyond the tiles that a walk kernel may use
static int stage_budget_bytes() {
    static int budget = -1;
    if (budget < 0) {
        int dev = 0, optin = 0;
        cudaFuncAttributes f2{}, f3{};
        cudaFuncAttributes w2{}, w3{};
        cudaFuncAttributes k2{}, k3{};
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
            cudaFuncGetAttributes(&f2, guided_walk_kernel<2, kWsWalkerWarps>) != cudaSuccess ||
            cudaFuncGetAttributes(&f3, guided_walk_kernel<3, kWsWalkerWarps>) != cudaSuccess ||
            cudaFuncGetAttributes(&w2, guided_walk_kernel<2, kWsWalkersWide>) != cudaSuccess ||
            cudaFuncGetAttributes(&w3, guided_walk_kernel<3, kWsWalkersWide>) != cudaSuccess ||
            cudaFuncGetAttributes(&k2, guided_walk_kernel<2, kWsWalkerWarps, kMaxKWide>) != cudaSuccess ||
            cudaFuncGetAttributes(&k3, guided_walk_kernel<3, kWsWalkerWarps, kMaxKWide>) != cudaSuccess)
            return 0;
        const int stat = (int)std::max(std::max(std::max(f2.sharedSizeBytes, f3.sharedSizeBytes),
                                                std::max(w2.sharedSizeBytes, w3.sharedSizeBytes)),
                                       std::max(k2.sharedSizeBytes, k3.sharedSizeBytes));
        budget = std::max(0, std::min(optin - kWsSmem - stat - 1024, WOST_STAGE_MAX_KB * 1024));
    }
    return budget;
}

wost_status guided_occupancy(int dim, int *per_sm) {
    *per_sm = 1;
    return once_per_device(100 + dim, [&]() -> wost_status {
        const int bytes = kWsSmem + stage_budget_bytes();
        const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
        // (the 16-lobe kernel stages less of the scene: the same total)
        if (dim == 2) {
            WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<2, kWsWalkerWarps>, at, bytes));
            WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<2, kWsWalkersWide>, at, bytes));
            WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<2, kWsWalkerWarps, kMaxKWide>, at,
                                           std::max(bytes, ws_smem_bytes(false, kMaxKWide))));
        } else {
            WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<3, kWsWalkerWarps>, at, bytes));
            WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<3, kWsWalkersWide>, at, bytes));
            WOST_CUDA(cudaFuncSetAttribute(guided_walk_kernel<3, kWsWalkerWarps, kMaxKWide>, at,
                                           std::max(bytes, ws_smem_bytes(false, kMaxKWide))));
        }
        return WOST_OK;
    });
}

// regions of the scene to stage, and their size in float4 (km: lobe
// capacity of the launch's kernel)
static int stage_mask_for(const DevScene &sc, int *f4, int km = kMaxK) {
    const int budget = stage_budget_bytes() - (km == kMaxK ? 0 : kWsSmemWideExtra);
    return stage_plan(sc, std::max(budget, 0) / 16, f4);
}

wost_status launch_guided(int dim, const GuidedArgs &g, int grid, cudaStream_t st, int walkers, int km = kMaxK) {
    int f4 = 0;
    stage_mask_for(g.w.sc, &f4, km);
    constexpr int tn = ws_threads(kWsWalkerWarps), tw = ws_threads(kWsWalkersWide);
    if (km != kMaxK) {
        const int smem16 = ws_smem_bytes(false, kMaxKWide) + f4 * 16;
        if (dim == 2) guided_walk_kernel<2, kWsWalkerWarps, kMaxKWide><<<grid, tn, smem16, st>>>(g);
        else guided_walk_kernel<3, kWsWalkerWarps, kMaxKWide><<<grid, tn, smem16, st>>>(g);
        WOST_CUDA(cudaGetLastError());
        return WOST_OK;
    }
    const int smem = kWsSmem + f4 * 16;
    const bool wide = walkers == kWsWalkersWide;
    if (dim == 2 && wide) guided_walk_kernel<2, kWsWalkersWide><<<grid, tw, smem, st>>>(g);
    else if (dim == 2) guided_walk_kernel<2, kWsWalkerWarps><<<grid, tn, smem, st>>>(g);
    else if (wide) guided_walk_kernel<3, kWsWalkersWide><<<grid, tw, smem, st>>>(g);
    else guided_walk_kernel<3, kWsWalkerWarps><<<grid, tn, smem, st>>>(g);
    WOST_CUDA(cudaGetLastError());
    return WOST_OK;
}

// ---------------------------------------------------------------------------
// Longest walks first.  A launch of the warp-specialised kernel lasts until
// its last walk ends, and a walk of a hundred steps or more that starts late
// keeps the launch running while most walker lanes have nothing left to do.
// The walks of one point have correlated lengths (points near the Neumann
// boundary walk long), so after each launch the points are sorted by the
// walk-steps their walks took in it, longest first (a counting sort on the
// device, no host round trip), and the next launch hands out each walk
// index's points in that order.  A walk draws from the random streams of its
// (point, walk) pair whenever it runs: the order changes no walk, only
// which walker lane runs it and when.  The order is kept with the scene
// from call to call (a solve run batch by batch, one call per training
// batch, keeps it); a call on another number of points starts afresh, and a
// call on other points of the same number gets a valid if unhelpful order.
// ---------------------------------------------------------------------------
#ifndef WOST_LONGEST_FIRST
#define WOST_LONGEST_FIRST 1
#endif
constexpr int kOrderBins = 1024;   // walk-step counts at or above kOrderBins - 1 share the top bin

__device__ __forceinline__ int order_bin(unsigned len) {
    return kOrderBins - 1 - (int)min(len, (unsigned)(kOrderBins - 1));   // longest first
}

__global__ void order_hist_kernel(const unsigned *plen, int64_t n, unsigned *hist) {
    __shared__ unsigned h[kOrderBins];
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[order_bin(plen[p])], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], h[i]);
}

// exclusive prefix sum of the kOrderBins counts, in place (one block of
// kOrderBins threads)
__global__ void order_scan_kernel(unsigned *hist) {
    __shared__ unsigned buf[2][kOrderBins];
    const int t = threadIdx.x;
    int in = 0;
    buf[0][t] = t > 0 ? hist[t - 1] : 0u;
    __syncthreads();
    for (int off = 1; off < kOrderBins; off <<= 1) {
        buf[1 - in][t] = buf[in][t] + (t >= off ? buf[in][t - off] : 0u);
        in = 1 - in;
        __syncthreads();
    }
    hist[t] = buf[in][t];
}

__global__ void order_scatter_kernel(const unsigned *plen, int64_t n, unsigned *offset, uint32_t *order) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= n) return;
    order[atomicAdd(&offset[order_bin(plen[p])], 1u)] = (uint32_t)p;
}

// the next launch's order from this launch's walk lengths (stream-ordered)
static wost_status order_by_length(const unsigned *plen, int64_t n, unsigned *hist, uint32_t *order,
                                   cudaStream_t st, int64_t &launches) {
    WOST_CUDA(cudaMemsetAsync(hist, 0, kOrderBins * sizeof(unsigned), st));
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)num_sms() * 4);
    order_hist_kernel<<<blocks, 256, 0, st>>>(plen, n, hist);
    order_scan_kernel<<<1, kOrderBins, 0, st>>>(hist);
    order_scatter_kernel<<<(int)((n + 255) / 256), 256, 0, st>>>(plen, n, hist, order);
    WOST_CUDA(cudaGetLastError());
    launches += 3;
    return WOST_OK;
}

wost_status ensure_records(wost_field *f, int64_t cap, size_t scratch_bytes);
wost_status wavefront_run(wost_scene *sc, wost_field *f, const WalkArgs &a, const WsOpts &o, const RecDest &rd,
                          int max_slots, cudaStream_t st, int64_t *iters_out);

// walk slots of a wavefront launch that trains nothing (walks beyond the slots
// queue up behind them)
constexpr int kWfMaxSlots = 1 << 20;

wost_status guided_solve(wost_scene *s, wost_field *f, WalkArgs &a, int nwalks, const wost_exec &ex,
                         cudaStream_t st, wost_stats *stats, int walk_begin, CallTiming &tm) {
    if (f->desc.dim != s->dim) { set_error("wost_solve: field dimension differs from the scene"); return WOST_ERR_INVALID_ARG; }
    // fields of 9..16 lobes: the 16-lobe warp-specialised kernel serves every
    // launch (the wavefront path decodes 8-lobe layouts only)
    const bool wide_mix = f->km != kMaxK;
    if (wide_mix && ex.guided_kernel == 2) {
        set_error("wost_solve: the wavefront kernel serves fields of at most 8 lobes");
        return WOST_ERR_UNSUPPORTED;
    }
    if (wide_mix && ex.walker_warps != 0 && ex.walker_warps != kWsWalkerWarps) {
        set_error("wost_solve: fields of more than 8 lobes run the standard walker count");
        return WOST_ERR_UNSUPPORTED;
    }
    GuidedArgs g{};
    g.f = f->dev();
    {
        int f4 = 0;
        g.stage_mask = stage_mask_for(s->dev, &f4, f->km);
    }
    g.o.c_mode = ex.c_mode;
    g.o.c_fixed = ex.c_fixed;
    g.o.reflect = ex.reflect;
    g.o.flush_polls = kFlushPolls;
    g.o.wait_ns = ex.wait_ns > 0 ? (unsigned long long)ex.wait_ns : kWaitNs;
    g.o.err = a.err;
    g.o.stat = a.stat;
    f->t_c_mode = ex.c_mode;
    f->t_c_fixed = ex.c_fixed;
    f->t_reflect = ex.reflect;
    f->t_samples = ex.train_samples;
    // Launch selection.  A launch that records training data holds one walk
    // per point (the field trains after it), and its time is set by how fast
    // walkers finish a few walks each: the asynchronous warp-specialised
    // kernel serves that best.  Launches without records run every walk at
    // once, and the wavefront keeps its slots full of them.
    const int rounds = ex.train ? std::max(0, std::min(nwalks, ex.train_until_wpp - walk_begin)) : 0;
    const bool wavefront = !wide_mix && (ex.guided_kernel == 2 || (ex.guided_kernel == 0 && rounds == 0));
    const bool ws_then_wavefront = !wide_mix && ex.guided_kernel == 0 && rounds > 0 && rounds < nwalks;
    // walks per point in one training batch (the last one clipped at `rounds`)
    const int bwpp = std::max(1, std::min(ex.batch_wpp, std::max(rounds, 1)));
    int ntrain = 0;
    // one wavefront launch of `items` walks from walk index w0; a recording
    // launch appends to the batch's records (`fresh`: the batch's first)
    auto run_wavefront = [&](int w0, unsigned long long items, bool record, bool fresh) -> wost_status {
        WalkArgs w = a;
        w.walk_begin = w0;
        w.total = items;
        g.o.record = record;
        WOST_CUDA(cudaMemsetAsync(a.work_ctr, 0, sizeof(unsigned long long), st));
        if (record && fresh) WOST_CUDA(cudaMemsetAsync(f->rec_ctr, 0, 2 * sizeof(unsigned long long), st));
        int64_t iters = 0;
        const int slots = record ? (int)a.npoints : (ex.wavefront_slots > 0 ? ex.wavefront_slots : kWfMaxSlots);
        tm.mark(tm.walk, st);
        wost_status rc = wavefront_run(s, f, w, g.o, g.rd, slots, st, &iters);
        tm.mark(tm.walk, st);
        tm.launches += 2 * iters;
        tm.walk_launches += 2 * iters;
        return rc;
    };
    auto train_after = [&]() -> wost_status {
        tm.mark(tm.train, st);
        int k = 0;
        wost_status rc = train_after_batch(f, s->dim, st, &k);
        tm.mark(tm.train, st);
        tm.launches += train_step_launches(f) * k;
        ntrain += k;
        return rc;
    };
    g.rd = RecDest{f->rec, f->rec_ctr, f->rec_cap};
    g.o.scratch_steps = a.maxsteps;
    // record buffer of one batch: 64 records per walk by default
    const int64_t rec_cap = ex.max_train_records > 0 ? ex.max_train_records
                                                     : std::max<int64_t>(a.npoints * 64 * bwpp, 1 << 20);
    if (wavefront) {
        // a training batch of B walks per point is B recording launches of
        // one walk per point (a recording launch holds one slot per walk),
        // then the field trains on the batch's records; then every remaining
        // walk in one launch (the random numbers of a walk do not depend on
        // how walks are grouped into launches)
        if (rounds > 0) {
            size_t scratch = (size_t)a.npoints * (size_t)std::max(a.maxsteps, 1) * kRecFloats * sizeof(float);
            wost_status rc = ensure_records(f, rec_cap, scratch);
            if (rc != WOST_OK) return rc;
            g.rd = RecDest{f->rec, f->rec_ctr, f->rec_cap};
        }
        g.o.scratch = f->scratch;
        for (int b = 0; b < rounds; b += bwpp) {
            const int nb = std::min(bwpp, rounds - b);
            wost_status rc = WOST_OK;
            for (int j = 0; j < nb && rc == WOST_OK; ++j)
                rc = run_wavefront(walk_begin + b + j, (unsigned long long)a.npoints, true, j == 0);
            if (rc == WOST_OK) rc = train_after();
            if (rc != WOST_OK) return rc;
        }
        if (rounds < nwalks) {
            wost_status rc = run_wavefront(walk_begin + rounds, (unsigned long long)a.npoints * (nwalks - rounds), false, false);
            if (rc != WOST_OK) return rc;
        }
    } else {
        int occ = 1;
        wost_status orc = guided_occupancy(s->dim, &occ);
        if (orc != WOST_OK) return orc;
        int cps = ex.ctas_per_sm > 0 ? std::min(ex.ctas_per_sm, occ) : occ;
        int grid = num_sms() * cps;
        // the largest launch of the solve: a training batch, or one walk per point
        const int walkers = ws_walkers_for_field(s->dev, f, ex.walker_warps,
                                                 (unsigned long long)a.npoints * (unsigned long long)(rounds > 0 ? bwpp : 1));
        if (rounds > 0) {
            size_t scratch = (size_t)grid * (walkers * 32) * (size_t)std::max(a.maxsteps, 1) * kRecFloats *
                             sizeof(float);
            wost_status rc = ensure_records(f, rec_cap, scratch);
            if (rc != WOST_OK) return rc;
            g.rd = RecDest{f->rec, f->rec_ctr, f->rec_cap};
        }
        g.o.scratch = f->scratch;
        const int ws_walks = ws_then_wavefront ? rounds : nwalks;
        // walk lengths per point and the launch order (longest walks first)
        unsigned *plen = nullptr, *hist = nullptr;
        uint32_t *order = nullptr;
        const bool longest_first = WOST_LONGEST_FIRST && a.npoints > 1 && a.npoints < (int64_t)UINT32_MAX;
        if (longest_first) {
            const size_t n = (size_t)a.npoints;
            const size_t had = s->ws_order.bytes;
            wost_status rc = s->ws_order.ensure((2 * n + kOrderBins) * sizeof(unsigned));
            if (rc != WOST_OK) return rc;
            if (s->ws_order.bytes != had) s->order_n = 0;   // a new buffer holds no order
            plen = s->ws_order.as<unsigned>();
            order = reinterpret_cast<uint32_t *>(plen + n);
            hist = plen + 2 * n;
        }
        // one launch per training batch (its scratch rows belong to walker
        // lanes, so a launch may hold several walks per point), one launch
        // per walk index after training
        for (int b = 0, nb = 1; b < ws_walks; b += nb) {
            nb = b < rounds ? std::min(bwpp, rounds - b) : 1;
            g.w = a;
            g.w.walk_begin = walk_begin + b;
            g.w.total = (unsigned long long)a.npoints * (unsigned long long)nb;
            g.w.order = longest_first && s->order_n == a.npoints ? order : nullptr;   // else point order
            g.w.plen = longest_first ? plen : nullptr;
            g.o.record = b < rounds;
            WOST_CUDA(cudaMemsetAsync(a.work_ctr, 0, sizeof(unsigned long long), st));
            if (g.o.record) WOST_CUDA(cudaMemsetAsync(f->rec_ctr, 0, 2 * sizeof(unsigned long long), st));
            if (g.w.plen) WOST_CUDA(cudaMemsetAsync(plen, 0, (size_t)a.npoints * sizeof(unsigned), st));
            tm.mark(tm.walk, st);
            wost_status rc = launch_guided(s->dim, g, grid, st, walkers, f->km);
            tm.mark(tm.walk, st);
            tm.launches++;
            tm.walk_launches++;
            if (rc != WOST_OK) return rc;
            // (the order kernels run after the launch and before the
            // training step, which does not read them)
            if (g.w.plen) {
                if ((rc = order_by_length(plen, a.npoints, hist, order, st, tm.launches)) != WOST_OK) return rc;
                s->order_n = a.npoints;
            }
            if (g.o.record && (rc = train_after()) != WOST_OK) return rc;
        }
        if (ws_then_wavefront) {
            wost_status rc = run_wavefront(walk_begin + rounds, (unsigned long long)a.npoints * (nwalks - rounds), false, false);
            if (rc != WOST_OK) return rc;
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
    if (wost_status dc = check_device(f->device, "wost_field_decode")) return dc;
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
    auto launch = [&](auto kern, int smem) -> wost_status {
        WOST_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
        kern<<<grid, kGuidedBlock, smem, st>>>(f->dev(), dp, n, dout, f->nout, device_err_flag());
        return WOST_OK;
    };
    constexpr int s8 = cta_tiles_smem(kMaxK), s16 = cta_tiles_smem(kMaxKWide);
    wost_status lrc = f->km == kMaxK ? (D == 2 ? launch(decode_kernel<2, kMaxK>, s8) : launch(decode_kernel<3, kMaxK>, s8))
                                     : (D == 2 ? launch(decode_kernel<2, kMaxKWide>, s16)
                                               : launch(decode_kernel<3, kMaxKWide>, s16));
    if (lrc != WOST_OK) return lrc;
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
    if ((dim != 2 && dim != 3) || K < 1 || K > kMaxKWide || n < 0 || (n > 0 && (!mu || !kappa || !lambda))) {
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
        const bool wide = K > kMaxK;
        if (dim == 2 && !wide) mixture_eval_kernel<2, kMaxK><<<gr, bs>>>(K, dmu, dk, dl, dn, n, dout);
        else if (dim == 2) mixture_eval_kernel<2, kMaxKWide><<<gr, bs>>>(K, dmu, dk, dl, dn, n, dout);
        else if (!wide) mixture_eval_kernel<3, kMaxK><<<gr, bs>>>(K, dmu, dk, dl, dn, n, dout);
        else mixture_eval_kernel<3, kMaxKWide><<<gr, bs>>>(K, dmu, dk, dl, dn, n, dout);
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
        const bool wide = K > kMaxK;
        if (dim == 2 && !wide) mixture_sample_kernel<2, kMaxK><<<gr, bs>>>(K, dmu, dk, dl, dc, k0, k1, n, dnu, dpdf);
        else if (dim == 2) mixture_sample_kernel<2, kMaxKWide><<<gr, bs>>>(K, dmu, dk, dl, dc, k0, k1, n, dnu, dpdf);
        else if (!wide) mixture_sample_kernel<3, kMaxK><<<gr, bs>>>(K, dmu, dk, dl, dc, k0, k1, n, dnu, dpdf);
        else mixture_sample_kernel<3, kMaxKWide><<<gr, bs>>>(K, dmu, dk, dl, dc, k0, k1, n, dnu, dpdf);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out_nu, dnu, n * dim * sizeof(float), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_pdf, dpdf, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(dmu); cudaFree(dk); cudaFree(dl); cudaFree(dc); cudaFree(dnu); cudaFree(dpdf);
    return e == cudaSuccess ? WOST_OK : cuda_status(e, "wost_mixture_sample");
}
