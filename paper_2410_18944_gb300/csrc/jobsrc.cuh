// Where a walk's work comes from.  The persistent walk loops (plain here,
// guided in guided_ws.cuh) are written once against a "job source":
//   SoloSrc  - one scene, one point set, one field: everything lives in the
//              kernel's argument block (wost_solve);
//   BatchSrc - many scenes of uneven size, each with its own points, walk
//              count, eps, step cap, seed and field, in a device job table
//              (wost_solve_batch).  Work items are laid out job-major, so the
//              walks in flight at any moment belong to few jobs.
// A source hands out work items, starts a walk from an item, gives the
// step its scene and scalars (StepEnv), and owns the per-point sums and the
// training-record buffer the walk writes to.  Either way every walk draws
// from the same Philox streams, counter (point, walk, step, purpose) and key
// (seed_lo, seed_hi + scene_id), so a job of a batch walks exactly as the
// same problem solved alone.
#pragma once
#include "field.cuh"
#include "lanewalk.cuh"
#include "walkstep.cuh"

// plain walks in 3D: 1 = per-lane query state machine (lanewalk.cuh), 0 =
// one warp-synchronous query at a time (plain_loop below).  Measured on
// one GB300 the state machine is 8-11% faster on the 3D workloads (82k and
// 994k triangles) and 26% slower in 2D (4096 segments), where its larger
// register footprint costs more occupancy than its convergence gains; both
// give identical results.
#ifndef WOST_PLAIN_LANES
#define WOST_PLAIN_LANES 1
#endif

namespace wost {

constexpr int kRecFloats = 12;   // training record: x[3] nu[3] n[3] on_neumann q target

// destination of finished training records (Sec. 5.2): buffer, counters
// ([0] appended, [1] dropped), capacity
struct RecDest {
    float *out;
    unsigned long long *ctr;
    long long cap;
};

// ---------------------------------------------------------------------------
// one scene
// ---------------------------------------------------------------------------
template <int D>
struct SoloSrc {
    const WalkArgs &a;
    const DevField *f;   // guided only
    RecDest rd;
    const DevScene *sc;  // the scene view the steps use (a.sc, or a copy on staged nodes)

    __device__ __forceinline__ unsigned long long *work_ctr() const { return a.work_ctr; }
    __device__ __forceinline__ unsigned long long total() const { return a.total; }
    __device__ __forceinline__ bool start(Walk<D> &w, unsigned long long item) const {
        if (a.order) {   // the same walk index, another point
            const unsigned long long p = item % (unsigned long long)a.npoints;
            item = item - p + a.order[p];
        }
        start_walk<D>(w, a, item);
        return a.status[w.pid] == 0;
    }
    __device__ __forceinline__ StepEnv env(const Walk<D> &) const {
        return StepEnv{*sc, a.eps, a.eps64, a.maxsteps, a.key0, a.key1, a.err, a.rr_depth, a.rr_q};
    }
    __device__ __forceinline__ void finish(const Walk<D> &w) const {
        finish_walk(a, w.pid, w.acc);
        if (a.plen) atomicAdd(a.plen + w.pid, (unsigned)w.k + 1u);
    }
    __device__ __forceinline__ const DevField &field(const Walk<D> &) const { return *f; }
    __device__ __forceinline__ RecDest rec(const Walk<D> &) const { return rd; }
    __device__ __forceinline__ int job(const Walk<D> &) const { return 0; }
    __device__ __forceinline__ const uint4 *wimg(int) const { return f->wimg; }
    __device__ __forceinline__ const float *b3(int) const { return f->b3; }
};

// Staging of a scene's traversal data in shared memory.  A walk step is a
// chain of dependent loads of BVH nodes and leaf primitives, so their
// latency is the step's latency; a kernel with shared memory to spare keeps
// as much of the data there as fits.  Regions, in the order they are taken:
// the three BVHs' nodes, the silhouette normal cones, then the Dirichlet,
// Neumann and silhouette primitives.
constexpr int kStageRegions = 7;

__host__ __device__ __forceinline__ void stage_regions(const DevScene &s, const float4 **src, int *cnt) {
    const int nb = s.dim == 2 ? node_f4<2>() : node_f4<3>();   // float4 per node
    const int pd = s.dim == 2 ? 1 : 3;       // per Dirichlet / Neumann primitive
    const int ps = s.dim == 2 ? 2 : 4;       // per silhouette element
    src[0] = s.dir.nodes; cnt[0] = s.dir.nnodes * nb;
    src[1] = s.neu.nodes; cnt[1] = s.neu.nnodes * nb;
    src[2] = s.sil.nodes; cnt[2] = s.sil.nnodes * nb;
    src[3] = s.sil_cones; cnt[3] = s.sil_cones ? bvh_width(s.dim) * s.sil.nnodes : 0;
    src[4] = s.dir.prims; cnt[4] = s.dir.nprims * pd;
    src[5] = s.neu.prims; cnt[5] = s.neu.nprims * pd;
    src[6] = s.sil.prims; cnt[6] = s.sil.nprims * ps;
}

// Which regions fit in budget_f4 float4 (bit r = region r), greedily in
// order: all node regions or none, then whole primitive arrays.
__host__ __forceinline__ int stage_plan(const DevScene &s, int budget_f4, int *total_f4) {
    const float4 *src[kStageRegions];
    int cnt[kStageRegions];
    stage_regions(s, src, cnt);
    int mask = 0, used = 0;
    const int nodes = cnt[0] + cnt[1] + cnt[2] + cnt[3];
    if (nodes <= budget_f4) {
        mask = 0xF;
        used = nodes;
        for (int r = 4; r < kStageRegions; ++r)
            if (cnt[r] > 0 && used + cnt[r] <= budget_f4) { mask |= 1 << r; used += cnt[r]; }
    }
    *total_f4 = used;
    return mask;
}

// Copies the regions in `mask` into shared memory `dst` (all threads of the
// block take part) and makes `out` (shared) a copy of the scene view whose
// pointers name the staged copies.
__device__ __forceinline__ void stage_scene(const DevScene &in, DevScene &out, float4 *dst, int mask) {
    const float4 *src[kStageRegions];
    int cnt[kStageRegions];
    stage_regions(in, src, cnt);
    float4 *start[kStageRegions];
    float4 *d = dst;
    for (int r = 0; r < kStageRegions; ++r) {
        start[r] = d;
        if (!(mask >> r & 1) || cnt[r] == 0) continue;
        for (int i = threadIdx.x; i < cnt[r]; i += blockDim.x) d[i] = __ldg(src[r] + i);
        d += cnt[r];
    }
    if (threadIdx.x == 0) {
        out = in;
        auto take = [&](int r) { return (mask >> r & 1) && cnt[r] > 0; };
        if (take(0)) out.dir.nodes = start[0];
        if (take(1)) out.neu.nodes = start[1];
        if (take(2)) out.sil.nodes = start[2];
        if (take(3)) out.sil_cones = start[3];
        if (take(4)) out.dir.prims = start[4];
        if (take(5)) out.neu.prims = start[5];
        if (take(6)) out.sil.prims = start[6];
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// many scenes
// ---------------------------------------------------------------------------
struct DevJob {
    DevScene sc;
    DevField f;                  // the job's field (guided batches)
    const double *points;        // npoints * D (device)
    int64_t npoints;
    int64_t point_off;           // first row of the job in the batch's per-point arrays
    int nwalks;
    int maxsteps;
    float eps;
    double eps64;
    uint32_t key0, key1;
    int rr_depth;                // Russian roulette from this step on (0 = off)
    float rr_q;                  // its survival probability
    RecDest rd;                  // the field's record buffer
    double *out_mean, *out_var;  // npoints each (device; out_var nullable)
};

// a contiguous run of work items of one launch: walks [walk_begin,
// walk_begin + n) of every point of one job, items ordered walk-major
// within the run (item = walk * npoints + point)
struct DevSeg {
    unsigned long long item_begin;
    int job;
    int walk_begin;
};

struct BatchArgs {
    const DevJob *jobs;
    const DevSeg *segs;
    int nseg;
    unsigned long long total;        // items in this launch
    unsigned long long *work_ctr;
    const uint8_t *status;           // per point of the batch: 0 walk, 1 shell, 2 outside
    double *sum, *sum2;              // per point of the batch (FP64)
    unsigned long long *stat;        // launch statistics (as WalkArgs::stat)
    int *err;
};

// index of the last segment whose item_begin <= item (segments sorted)
__device__ __forceinline__ int find_seg(const DevSeg *segs, int nseg, unsigned long long item) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (__ldg(&segs[mid].item_begin) <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int D>
struct BatchSrc {
    const BatchArgs &b;

    __device__ __forceinline__ unsigned long long *work_ctr() const { return b.work_ctr; }
    __device__ __forceinline__ unsigned long long total() const { return b.total; }
    __device__ __forceinline__ bool start(Walk<D> &w, unsigned long long item) const {
        const int s = find_seg(b.segs, b.nseg, item);
        const DevSeg sg = b.segs[s];
        const DevJob &J = b.jobs[sg.job];
        const unsigned long long local = item - sg.item_begin, np = (unsigned long long)J.npoints;
        w.job = sg.job;
        w.pid = (uint32_t)(local % np);
        w.wid = (uint32_t)(sg.walk_begin + local / np);
#pragma unroll
        for (int i = 0; i < D; ++i) { w.x[i] = (float)J.points[(size_t)w.pid * D + i]; w.n[i] = 0.f; }
        w.T = 1.f;
        w.acc = 0.f;
        w.k = 0;
        w.prim = -1;
        return b.status[J.point_off + w.pid] == 0;
    }
    __device__ __forceinline__ StepEnv env(const Walk<D> &w) const {
        const DevJob &J = b.jobs[w.job];
        return StepEnv{J.sc, J.eps, J.eps64, J.maxsteps, J.key0, J.key1, b.err, J.rr_depth, J.rr_q};
    }
    __device__ __forceinline__ void finish(const Walk<D> &w) const {
        const size_t i = (size_t)b.jobs[w.job].point_off + w.pid;
        atomicAdd(b.sum + i, (double)w.acc);
        atomicAdd(b.sum2 + i, (double)w.acc * (double)w.acc);
    }
    __device__ __forceinline__ const DevField &field(const Walk<D> &w) const { return b.jobs[w.job].f; }
    __device__ __forceinline__ RecDest rec(const Walk<D> &w) const { return b.jobs[w.job].rd; }
    __device__ __forceinline__ int job(const Walk<D> &w) const { return w.job; }
    __device__ __forceinline__ const uint4 *wimg(int j) const { return b.jobs[j].f.wimg; }
    __device__ __forceinline__ const float *b3(int j) const { return b.jobs[j].f.b3; }
};

// ---------------------------------------------------------------------------
// The plain persistent walk loop (uniform directions, Sec. 3.2).
// Every lane of a warp stays in the loop until the whole warp is out of
// work, and one loop iteration is one step of every active lane: lanes
// cannot drift into different phases of the step, so the warp re-converges
// after each query (a lane without a walk is predicated off).
// ---------------------------------------------------------------------------
template <int D, class Src>
__device__ __forceinline__ void plain_loop(const Src &src, unsigned long long *stat) {
    if (WOST_PLAIN_LANES && D == 3) {
        plain_loop_lanes<D>(src, stat);
        return;
    }
    Walk<D> w;
    Visits vis;
    bool active = false, exhausted = false;
    unsigned long long nsteps = 0, ntrunc = 0, nwalks = 0;
    for (;;) {
        if (!active && !exhausted) {
            unsigned long long item = warp_fetch_add(src.work_ctr(), true);
            if (item >= src.total()) exhausted = true;
            else if (src.start(w, item)) { active = true; nwalks++; }
        }
        if (!__any_sync(0xffffffffu, active || !exhausted)) break;
        __syncwarp();
        if (!active) continue;
        nsteps++;
        const StepEnv env = src.env(w);
        float r, S, gv;
        bool trunc = false;
        bool ended = step_geometry<D>(w, env, r, S, gv, trunc, &vis);
        float nu[D];
        if (!ended) {
            U4 u = philox(w.pid, w.wid, (uint32_t)w.k, P_DIR, env.key0, env.key1);
            uniform_dir<D>(u01(u.x), u01(u.y), nu);
            if (w.prim >= 0) {
                float dn = dotv<D>(nu, w.n);
                if (dn < 0.f) reflect<D>(nu, w.n);
                ended = dn == 0.f;   // zero density at the tangent plane (Eq. angular_req)
            }
        }
        if (ended) {
            src.finish(w);
            ntrunc += trunc;
            active = false;
        } else {
            step_move<D>(w, env, nu, r, &vis);
        }
    }
    flush_stats(stat, nsteps, ntrunc, nwalks, vis);
}

}  // namespace wost
