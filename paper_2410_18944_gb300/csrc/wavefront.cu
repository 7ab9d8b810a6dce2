// Guided walk on stars as a wavefront (Sec. 5.1): the walks of a launch live
// in slots whose state (position, throughput, estimate, Neumann normal, ids,
// step) sits in global memory as structure-of-arrays, and every iteration runs
// two kernels over them:
//
//   step kernel   - one thread per slot: if the slot's walk has a decoded
//                   mixture pending, draw the direction by one-sample MIS
//                   (Sec. 4.4 Eq. mis_pdf), reflect it at Neumann points
//                   (Sec. 4.3), weight it by 1 / (|S| alpha p~) (Sec. 4.1),
//                   keep the training record (Sec. 5.2) and cast the star ray
//                   (the walk moves); then run the next step's geometry
//                   (closest Dirichlet point, epsilon-shell, silhouette, star
//                   radius, source term).  A walk that ends adds its value to
//                   the point's FP64 sums and the slot takes the next work
//                   item at once, so slots stay full while work remains.
//                   Walks that need a direction are appended (warp-aggregated)
//                   to the iteration's decode list.
//   decode kernel - the hash-grid encode and the three-layer MLP on tcgen05
//                   tensor cores for the decode list, 128 rows per tile,
//                   written as FP16 rows (the raw outputs of Tab. reg_map).
//
// The step kernel needs no tensor memory, no shared weights and no barrier,
// so it runs at the occupancy of the plain walk; the decode kernel runs dense
// tiles.  The two kernels alternate until no walk needs a direction and no
// work is left; the host checks that every few iterations.
#include <algorithm>
#include <cstring>

#include "guided_ws.cuh"
#include "internal.h"

namespace wost {

wost_status ensure_records(wost_field *f, int64_t cap, size_t scratch_bytes);

namespace {

constexpr int kWfBlock = 128;
constexpr int kThetaStride = kOutPad;   // FP16 decoded outputs per decode row
constexpr int kWfChunk = 8;             // iterations between host checks

// Iteration k's step kernel reads the decode list of iteration k-1 (entry j
// is an active walk whose pending step decoded into row j of theta) and
// appends the walks that need a direction to the list of parity k & 1; its
// decode kernel fills theta for that list and clears the other counter.
struct WfSlots {
    float4 *xT;        // position (D used), throughput T
    float4 *nA;        // Neumann normal (D used), estimate accumulated so far
    int4 *ids;         // point, walk, step, Neumann slot (-1 interior)
    int *job;          // job of the slot's walk
    float2 *rS;        // star radius and source term of the pending step
    int *dlist[2];     // slot of each decode row, by iteration parity
    unsigned *dcount;  // [2] decode rows, by iteration parity
    __half *theta;     // [rows][kThetaStride] decoded outputs of the last list
    int2 *ended;       // recording launches: (records, terminal value bits) of the slot's ended walk
    int nslots;
};

struct WfSoloArgs {
    WalkArgs w;
    DevField f;
    WsOpts o;
    RecDest rd;
    WfSlots S;
    int parity;
    int first;         // first iteration: every slot starts empty
};

template <int D>
__device__ __forceinline__ void load_walk(const WfSlots &S, int s, Walk<D> &w) {
    const float4 xT = S.xT[s], nA = S.nA[s];
    const int4 id = S.ids[s];
    w.x[0] = xT.x; w.x[1] = xT.y;
    w.n[0] = nA.x; w.n[1] = nA.y;
    if (D == 3) { w.x[D - 1] = xT.z; w.n[D - 1] = nA.z; }
    w.T = xT.w;
    w.acc = nA.w;
    w.pid = (uint32_t)id.x;
    w.wid = (uint32_t)id.y;
    w.k = id.z;
    w.prim = id.w;
}

template <int D>
__device__ __forceinline__ void store_walk(const WfSlots &S, int s, const Walk<D> &w) {
    S.xT[s] = make_float4(w.x[0], w.x[1], D == 3 ? w.x[D - 1] : 0.f, w.T);
    S.nA[s] = make_float4(w.n[0], w.n[1], D == 3 ? w.n[D - 1] : 0.f, w.acc);
    S.ids[s] = make_int4((int)w.pid, (int)w.wid, w.k, w.prim);
}

template <int D, class Src>
__device__ __forceinline__ void wf_step_body(const Src &src, const WsOpts &o, const WfSlots &S, int parity,
                                             bool first) {
    // one thread per entry of the previous iteration's decode list (or per
    // slot in the first iteration); blocks past the list's end leave at once
    const unsigned n_in = first ? (unsigned)S.nslots : S.dcount[parity ^ 1];
    const unsigned j = blockIdx.x * kWfBlock + threadIdx.x;
    if (blockIdx.x * kWfBlock >= n_in) return;
    const bool valid = j < n_in;
    // decoded rows are staged in shared memory (stride of 25 words: the
    // scalar reads of the mixture evaluation are free of bank conflicts)
    __shared__ __half rows[kWfBlock * kYStride];
    __half *myrow = rows + threadIdx.x * kYStride;
    const float area = D == 2 ? 2.f * WOST_PI : 4.f * WOST_PI;
    Visits vis;
    unsigned long long nsteps = 0, ntrunc = 0, nwalks = 0;
    const int s = valid ? (first ? (int)j : S.dlist[parity ^ 1][j]) : 0;
    Walk<D> w;
    bool active = valid && !first;
    float r = 0.f, Sx = 0.f;
    if (active) {
        load_walk<D>(S, s, w);
        w.job = S.job[s];
        // ---- the pending step: direction, weight, record, move ----
        const float2 rs = S.rS[s];
        r = rs.x;
        Sx = rs.y;
        const uint2 *src_row = reinterpret_cast<const uint2 *>(S.theta + (size_t)j * kThetaStride);
#pragma unroll
        for (int i = 0; i < kThetaStride / 4; ++i) {
            const uint2 v = __ldcs(src_row + i);
            reinterpret_cast<uint32_t *>(myrow)[2 * i] = v.x;
            reinterpret_cast<uint32_t *>(myrow)[2 * i + 1] = v.y;
        }
        RowMixture<D, 8> m;
        m.init(myrow);
        const float c = o.c_mode ? o.c_fixed : m.c();
        const StepEnv env = src.env(w);
        float nu[D];
        const bool from_guide =
            sample_direction_row<D, 8>(m, c, w.pid, w.wid, (uint32_t)w.k, env.key0, env.key1, nu);
        const bool onN = w.prim >= 0;
        bool zero_density = false;
        float wgt = 1.f, ptil = 0.f;
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
        float *scratch_row = o.scratch + (size_t)s * o.scratch_steps * kRecFloats;
        if (zero_density) {
            src.finish(w);
            if (o.record) S.ended[s] = make_int2(w.k, __float_as_int(Sx));
            active = false;
        } else {
            if (o.record) {
                float4 *rr = reinterpret_cast<float4 *>(scratch_row + (size_t)w.k * kRecFloats);
                const float n2 = onN && D == 3 ? w.n[D - 1] : 0.f;
                rr[0] = make_float4(w.x[0], w.x[1], D == 3 ? w.x[D - 1] : 0.f, nu[0]);
                rr[1] = make_float4(nu[1], D == 3 ? nu[D - 1] : 0.f, onN ? w.n[0] : 0.f, onN ? w.n[1] : 0.f);
                rr[2] = make_float4(n2, ptil, wgt * roulette_scale(env, w.k), Sx);
            }
            w.T *= wgt;
            step_move<D>(w, env, nu, r, &vis);
        }
    }
    // ---- the next step's geometry; an ended walk hands its slot to the next item ----
    for (;;) {
        if (!active) {
            if (!valid) break;
            const unsigned long long item = warp_fetch_add(src.work_ctr(), true);
            if (item >= src.total()) break;
            if (!src.start(w, item)) continue;
            active = true;
            nwalks++;
        }
        nsteps++;
        float gv;
        bool trunc = false;
        if (step_geometry<D>(w, src.env(w), r, Sx, gv, trunc, &vis)) {
            src.finish(w);
            // the suffix pass of a recorded walk waits for the end of the
            // launch (a recording launch gives every slot one walk, so its
            // scratch rows stay intact): a long pass inline would hold up
            // every iteration
            if (o.record) S.ended[s] = make_int2(w.k, __float_as_int(gv));
            ntrunc += trunc;
            active = false;
            continue;
        }
        break;
    }
    if (active) {
        store_walk<D>(S, s, w);
        S.job[s] = src.job(w);
        S.rS[s] = make_float2(r, Sx);
        S.dlist[parity][warp_append(S.dcount + parity)] = s;
    }
    flush_stats(o.stat, nsteps, ntrunc, nwalks, vis);
}

// suffix passes of the walks of a recording launch (one per slot)
__global__ void wf_suffix_kernel(RecDest rd, const float *scratch, int scratch_steps, const int2 *ended, int n) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    const int2 e = ended[s];
    if (e.x > 0)
        end_recorded_walk(rd, scratch + (size_t)s * scratch_steps * kRecFloats, e.x, __int_as_float(e.y));
}

template <int D>
__global__ void __launch_bounds__(kWfBlock) wf_step_kernel(const __grid_constant__ WfSoloArgs g) {
    wf_step_body<D>(SoloSrc<D>{g.w, &g.f, g.rd, &g.w.sc}, g.o, g.S, g.parity, g.first != 0);
}

// decode rows [0, dcount[parity]) of the list into FP16 rows; clears the
// other parity's counter for the next step kernel
template <int D>
__global__ void __launch_bounds__(256, 1) wf_decode_kernel(DevField f, WfSlots S, int parity, int *err) {
    extern __shared__ __align__(1024) uint8_t sm[];
    if (blockIdx.x == 0 && threadIdx.x == 0) S.dcount[parity ^ 1] = 0;
    const unsigned n = S.dcount[parity];
    if ((unsigned)blockIdx.x * 256u >= n) return;   // uniform per CTA, before any set-up
    CtaTiles ct = cta_tiles_setup(sm, f);
    const int tid = threadIdx.x, tile = tid >> 7, row = tid & 127;
    TileCtx t{ct.xt + tile * (128 * kFeat * 2), ct.ht + tile * (128 * kHid * 2), ct.wimg, &ct.mbar[tile],
              *ct.tptr + (uint32_t)(tile * 64), 0u, 1 + tile};
    for (unsigned base = blockIdx.x * 256u; base < n; base += gridDim.x * 256u) {
        const unsigned i = base + tid;
        const bool valid = i < n;
        if (valid) {
            const int s = S.dlist[parity][i];
            const float4 xT = S.xT[s];
            const float x[3] = {xT.x, xT.y, xT.z};
            encode_row<D>(f, x, t.xtile, row);
        } else {
            zero_row(t.xtile, row, kFeat);
        }
        float raw[kOutPad];
        if (!mlp_tile_forward(t, f, row, row == 0, raw, err)) break;
        if (valid) {
            uint2 *dst = reinterpret_cast<uint2 *>(S.theta + (size_t)i * kThetaStride);
#pragma unroll
            for (int c = 0; c < kOutPad; c += 4) {
                __half2 a = __floats2half2_rn(raw[c], raw[c + 1]), b = __floats2half2_rn(raw[c + 2], raw[c + 3]);
                __stcs(dst + c / 4, make_uint2(*reinterpret_cast<uint32_t *>(&a), *reinterpret_cast<uint32_t *>(&b)));
            }
        }
    }
    cta_tiles_teardown(ct);
}

template <class K>
int occupancy_grid(K kernel, int block, size_t smem) {
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, block, smem) != cudaSuccess || n < 1) n = 1;
    return n * num_sms();
}

}  // namespace

// Runs `items` walk items of a guided solve (a.total, a.work_ctr, a.walk_begin
// set by the caller) through the wavefront; returns the iterations taken.
wost_status wavefront_run(wost_scene *sc, wost_field *f, const WalkArgs &a, const WsOpts &o, const RecDest &rd,
                          int max_slots, cudaStream_t st, int64_t *iters_out) {
    if (f->km != kMaxK) {
        set_error("wost_solve: the wavefront kernel serves fields of at most 8 lobes");
        return WOST_ERR_UNSUPPORTED;
    }
    const int D = sc->dim;
    const unsigned long long items = a.total;
    const int nslots = (int)std::min<unsigned long long>(items, (unsigned long long)std::max(max_slots, 1));
    // carve the slot arrays out of one workspace
    const size_t n = (size_t)std::max(nslots, 1);
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o0 = off; off += (bytes + 255) & ~(size_t)255; return o0; };
    const size_t o_xT = take(n * sizeof(float4)), o_nA = take(n * sizeof(float4)), o_ids = take(n * sizeof(int4));
    const size_t o_jb = take(n * sizeof(int)), o_rS = take(n * sizeof(float2));
    const size_t o_dl0 = take(n * sizeof(int)), o_dl1 = take(n * sizeof(int));
    const size_t o_dc = take(2 * sizeof(unsigned)), o_th = take(n * kThetaStride * sizeof(__half));
    const size_t o_en = take(n * sizeof(int2));
    wost_status rc = sc->ws_wf.ensure(off);
    if (rc != WOST_OK) return rc;
    if (!sc->pinned) WOST_CUDA(cudaMallocHost(&sc->pinned, 4 * sizeof(unsigned long long)));
    uint8_t *b = sc->ws_wf.as<uint8_t>();
    WfSlots S;
    S.xT = reinterpret_cast<float4 *>(b + o_xT);
    S.nA = reinterpret_cast<float4 *>(b + o_nA);
    S.ids = reinterpret_cast<int4 *>(b + o_ids);
    S.job = reinterpret_cast<int *>(b + o_jb);
    S.rS = reinterpret_cast<float2 *>(b + o_rS);
    S.dlist[0] = reinterpret_cast<int *>(b + o_dl0);
    S.dlist[1] = reinterpret_cast<int *>(b + o_dl1);
    S.dcount = reinterpret_cast<unsigned *>(b + o_dc);
    S.theta = reinterpret_cast<__half *>(b + o_th);
    S.ended = reinterpret_cast<int2 *>(b + o_en);
    S.nslots = nslots;
    WOST_CUDA(cudaMemsetAsync(S.dcount, 0, 2 * sizeof(unsigned), st));
    if (o.record) {
        if ((unsigned long long)nslots != items) {
            set_error("guided wavefront: a recording launch needs one slot per walk");
            return WOST_ERR_INVALID_ARG;
        }
        WOST_CUDA(cudaMemsetAsync(S.ended, 0, n * sizeof(int2), st));
    }

    // decode grid: the attribute is set, and the occupancy taken, once per
    // device (the device model, and so the grid, is the same on all of them)
    static int grid_dec[4] = {0, 0, 0, 0};
    {
        wost_status rc = once_per_device(300 + D, [&]() -> wost_status {
            if (D == 2) {
                WOST_CUDA(cudaFuncSetAttribute(wf_decode_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCtaTilesSmem));
                grid_dec[D] = occupancy_grid(wf_decode_kernel<2>, 256, kCtaTilesSmem);
            } else {
                WOST_CUDA(cudaFuncSetAttribute(wf_decode_kernel<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, kCtaTilesSmem));
                grid_dec[D] = occupancy_grid(wf_decode_kernel<3>, 256, kCtaTilesSmem);
            }
            return WOST_OK;
        });
        if (rc != WOST_OK) return rc;
    }
    // one thread per list entry (at most one per slot): the block scheduler
    // balances the uneven step costs
    const int gs = (nslots + kWfBlock - 1) / kWfBlock;
    const int gd = std::min(grid_dec[D], (nslots + 255) / 256);
    WfSoloArgs g{};
    g.w = a;
    g.f = f->dev();
    g.o = o;
    g.rd = rd;
    g.S = S;
    // every walk ends within maxsteps + 1 geometry steps after it starts, and
    // a slot starts at most ceil(items / nslots) walks
    const int64_t limit = ((int64_t)(items / (unsigned long long)nslots) + 2) * ((int64_t)a.maxsteps + 2) + 2 * kWfChunk;
    int64_t it = 0;
    for (;;) {
        for (int j = 0; j < kWfChunk; ++j, ++it) {
            g.parity = (int)(it & 1);
            g.first = it == 0;
            if (D == 2) wf_step_kernel<2><<<gs, kWfBlock, 0, st>>>(g);
            else wf_step_kernel<3><<<gs, kWfBlock, 0, st>>>(g);
            if (D == 2) wf_decode_kernel<2><<<gd, 256, kCtaTilesSmem, st>>>(g.f, S, g.parity, a.err);
            else wf_decode_kernel<3><<<gd, 256, kCtaTilesSmem, st>>>(g.f, S, g.parity, a.err);
        }
        WOST_CUDA(cudaGetLastError());
        // rows the last step kernel queued, and work taken so far
        unsigned long long *h = sc->pinned;
        WOST_CUDA(cudaMemcpyAsync(h, S.dcount + ((it - 1) & 1), sizeof(unsigned), cudaMemcpyDeviceToHost, st));
        WOST_CUDA(cudaMemcpyAsync(h + 1, a.work_ctr, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st));
        WOST_CUDA(cudaStreamSynchronize(st));
        const unsigned pending = *reinterpret_cast<unsigned *>(h);
        if (pending == 0 && h[1] >= items) break;
        if (it > limit) {
            set_error("guided wavefront did not drain within its iteration bound");
            return WOST_ERR_TIMEOUT;
        }
    }
    if (o.record) {
        wf_suffix_kernel<<<(nslots + 255) / 256, 256, 0, st>>>(rd, o.scratch, o.scratch_steps, S.ended, nslots);
        WOST_CUDA(cudaGetLastError());
        ++it;
    }
    if (iters_out) *iters_out = it;
    return WOST_OK;
}

}  // namespace wost
