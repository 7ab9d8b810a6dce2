// Plain walk on stars (uniform directions, Sec. 3.2 / Sec. 4.1 Eq. for p_u),
// point classification, per-point reduction, the geometric query entry
// points, and wost_solve.
//
// The walk kernel is persistent: one walk per thread at a time; a thread
// whose walk ends takes the next work item from a global counter with one
// warp-aggregated atomic, so warps stay full until the work runs out
// (warp-compacted work queue).  One loop iteration is one walk-step for
// every lane.  Per-point sums and sums of squares are FP64 atomics.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>
#include <set>
#include <vector>

#include "field.cuh"
#include "internal.h"
#include "jobsrc.cuh"

namespace wost {

double walk_alg_bytes(int D, bool guided, const unsigned long long *hs, int64_t records) {
    // bytes per item of the leaf-order arrays (see common.cuh)
    const double node_b = 16.0 * (D == 2 ? node_f4<2>() : node_f4<3>()), prim_b = D == 2 ? 16 : 48,
                 sil_b = D == 2 ? 32 : 64;
    double b = hs[3] * node_b + hs[4] * prim_b + hs[5] * sil_b + hs[6] * prim_b;
    b += (double)hs[2] * (D * 8.0 + 2 * 8.0);          // start point, FP64 sum and sum of squares
    if (guided) {
        double decodes = (double)hs[0] - (double)hs[2];  // every non-terminal step decodes once
        b += decodes * 16.0 * (1 << D) * 4.0;            // L = 16 levels x 2^d corners x 2 FP16
        b += (double)records * (48.0 + 48.0 + 48.0);     // record write, suffix read, final write
    }
    return b;
}

wost_status once_per_device(int key, const std::function<wost_status()> &f) {
    static std::mutex m;
    static std::set<std::pair<int, int>> done;
    int dev = 0;
    WOST_CUDA(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(m);
    if (done.count({dev, key})) return WOST_OK;
    const wost_status rc = f();
    if (rc == WOST_OK) done.insert({dev, key});
    return rc;
}

int num_sms() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 1;
    }
    return n;
}

wost_status DevBuf::ensure(size_t n) {
    if (n <= bytes) return WOST_OK;
    release();
    size_t want = n + n / 4;
    cudaError_t e = cudaMalloc(&ptr, want);
    if (e != cudaSuccess) {
        ptr = nullptr;
        bytes = 0;
        set_error("device allocation of a work buffer failed");
        return e == cudaErrorMemoryAllocation ? WOST_ERR_OOM : WOST_ERR_CUDA;
    }
    bytes = want;
    return WOST_OK;
}

void DevBuf::release() {
    if (ptr) cudaFree(ptr);
    ptr = nullptr;
    bytes = 0;
}

constexpr int kPlainBlock = 128;

template <int D>
__global__ void __launch_bounds__(kPlainBlock) plain_walk_kernel(const __grid_constant__ WalkArgs a) {
    plain_loop<D>(SoloSrc<D>{a, nullptr, RecDest{}, &a.sc}, a.stat);
}

// status of every query point: 2 outside (odd/even crossing count of a ray
// against all primitives), 1 inside the epsilon-shell (value g(xbar)), 0 walk
template <int D>
__global__ void classify_kernel(WalkArgs a, double *shell_value) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.npoints) return;
    double val;
    const_cast<uint8_t *>(a.status)[i] = classify_point<D>(a.sc, a.eps64, a.points + i * D, a.err, val);
    shell_value[i] = val;
}

__global__ void finalize_kernel(const uint8_t *status, const double *shell_value, const double *sum,
                                const double *sum2, int64_t n, int nw, double *mean, double *var) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    finalize_point(status[i], shell_value[i], sum[i], sum2[i], nw, mean + i, var ? var + i : nullptr);
}

// ---- query kernels -----------------------------------------------------------
template <int D>
__global__ void q_closest_kernel(DevScene sc, const double *p, int64_t n, int32_t *oid, float *od, int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[D];
    for (int k = 0; k < D; ++k) x[k] = (float)p[i * D + k];
    float b;
    int s = closest_dirichlet<D>(sc.dir, x, b, err);
    oid[i] = s >= 0 ? sc.dir.ids[s] : -1;
    od[i] = sqrtf(b);
}

template <int D>
__global__ void q_sil_kernel(DevScene sc, const int64_t *keys, const double *p, int64_t n, int64_t *oid,
                             float *od, int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[D];
    for (int k = 0; k < D; ++k) x[k] = (float)p[i * D + k];
    float b = __int_as_float(0x7f800000);
    int s = closest_silhouette<D>(sc.sil, x, sc.tau, b, err, nullptr, sc.sil_cones);
    oid[i] = s >= 0 ? keys[s] : -1;
    od[i] = s >= 0 ? sqrtf(b) : b;
}

// kExit = false: first hit of any orientation, FP64 re-test of the winner
// against tmax.  kExit = true: the cast of a walk step (step_move): exit
// crossings only, from t > -tneg, and the winner re-tested in FP64 against
// the FP32 tmax when its FP32 parameter lies within the rounding band below it.
template <int D, bool kExit>
__global__ void q_ray_kernel(DevScene sc, const double *o, const double *v, const double *tmax,
                             const int32_t *skip_id, const int *slot_of_id, int64_t n, int32_t *oid, float *ot,
                             int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float x[D], d[D];
    for (int k = 0; k < D; ++k) { x[k] = (float)o[i * D + k]; d[k] = (float)v[i * D + k]; }
    int skip = skip_id && skip_id[i] >= 0 ? slot_of_id[skip_id[i]] : -1;
    float t;
    float tm = (float)tmax[i];
    int s;
    if (kExit) {
        const float tneg = kRoundBand * sc.scale;
        s = ray_neumann<D, true>(sc.neu, x, d, tm, skip, t, err, nullptr, tneg);
        if (s >= 0 && tm - t <= kRoundBand * (sc.scale + tm)) {
            double t64;
            if (!ray_prim64<D, true>(sc.neu, s, x, d, t64, tneg) || t64 > (double)tm) s = -1;
        }
    } else {
        s = ray_neumann<D>(sc.neu, x, d, tm, skip, t, err);
        if (s >= 0) {
            double t64;
            if (!ray_prim64<D>(sc.neu, s, x, d, t64) || t64 > tmax[i]) s = -1;
        }
    }
    oid[i] = s >= 0 ? sc.neu.ids[s] : -1;
    ot[i] = s >= 0 ? t : __int_as_float(0x7f800000);
}

__global__ void invert_ids_kernel(const int *ids, int n, int *slot_of) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) slot_of[ids[i]] = i;
}

}  // namespace wost

using namespace wost;

namespace {

template <class T>
struct Staged {
    T *dev = nullptr;
    bool owned = false;
    ~Staged() { if (owned && dev) cudaFree(dev); }
};

template <class T>
wost_status stage_in(const T *src, size_t n, bool on_device, Staged<T> &out) {
    if (on_device || !src) { out.dev = const_cast<T *>(src); return WOST_OK; }
    if (n == 0) return WOST_OK;
    WOST_CUDA(cudaMalloc(&out.dev, n * sizeof(T)));
    out.owned = true;
    WOST_CUDA(cudaMemcpy(out.dev, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return WOST_OK;
}

int blocks_for(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

int *g_err_dev = nullptr;
int *err_flag() {
    if (!g_err_dev) {
        cudaMalloc(&g_err_dev, sizeof(int));
        cudaMemset(g_err_dev, 0, sizeof(int));
    }
    return g_err_dev;
}

wost_status check_err_flag(cudaStream_t st) {
    int h = 0;
    WOST_CUDA(cudaMemcpyAsync(&h, err_flag(), sizeof(int), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaStreamSynchronize(st));
    if (h) {
        cudaMemsetAsync(err_flag(), 0, sizeof(int), st);
        if (h & 2) { set_error("a bounded device wait timed out"); return WOST_ERR_TIMEOUT; }
        set_error("BVH traversal stack overflow");
        return WOST_ERR_CUDA;
    }
    return WOST_OK;
}

}  // namespace

namespace wost {
wost_status guided_solve(wost_scene *s, wost_field *f, WalkArgs &a, int nwalks, const wost_exec &ex,
                         cudaStream_t st, wost_stats *stats, int walk_begin, CallTiming &tm);
int *device_err_flag() { return err_flag(); }
wost_status device_check(cudaStream_t st) { return check_err_flag(st); }
}

extern "C" wost_status wost_solve(wost_scene *s, wost_field *field, const double *points, int64_t npoints,
                                  int32_t nwalks, double eps, int32_t maxsteps, int32_t guided,
                                  double *out_mean, double *out_var, wost_stats *stats, const wost_exec *exec) {
    if (!s || (npoints > 0 && !out_mean) || npoints < 0 || nwalks <= 0 || !(eps > 0) || maxsteps < 0) {
        set_error("wost_solve: invalid argument");
        return WOST_ERR_INVALID_ARG;
    }
    if (npoints > 0 && !points) { set_error("wost_solve: null points"); return WOST_ERR_INVALID_ARG; }
    if (guided && !field) { set_error("wost_solve: guided solve needs a field"); return WOST_ERR_INVALID_ARG; }
    if (exec && (exec->rr_depth < 0 || (exec->rr_depth > 0 && !(exec->rr_survival > 0.f && exec->rr_survival <= 1.f)))) {
        set_error("wost_solve: rr_depth must be >= 0 and rr_survival in (0, 1]");
        return WOST_ERR_INVALID_ARG;
    }
    if (exec && exec->batch_wpp < 0) { set_error("wost_solve: batch_wpp must be >= 0"); return WOST_ERR_INVALID_ARG; }
    if (exec && !ws_walker_warps_valid(exec->walker_warps)) {
        set_error("wost_solve: walker_warps must be 0, 16 or 28");
        return WOST_ERR_INVALID_ARG;
    }
    {
        wost_status dc = check_device(s->device, "wost_solve (scene)");
        if (dc == WOST_OK && guided) dc = check_device(field->device, "wost_solve (field)");
        if (dc != WOST_OK) return dc;
    }
    wost_exec ex;
    if (exec) ex = *exec; else wost_exec_defaults(&ex);
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (npoints == 0) return WOST_OK;
    cudaStream_t st = (cudaStream_t)ex.stream;
    const int D = s->dim;
    wost_status rc;
    // points
    const double *pts = points;
    if (!ex.points_on_device) {
        if ((rc = s->ws_points.ensure(npoints * D * sizeof(double))) != WOST_OK) return rc;
        WOST_CUDA(cudaMemcpyAsync(s->ws_points.ptr, points, npoints * D * sizeof(double), cudaMemcpyHostToDevice, st));
        pts = s->ws_points.as<double>();
    }
    if ((rc = s->ws_status.ensure(npoints * (sizeof(uint8_t) + sizeof(double)) + 64)) != WOST_OK) return rc;
    if ((rc = s->ws_sum.ensure(npoints * sizeof(double))) != WOST_OK) return rc;
    if ((rc = s->ws_sum2.ensure(npoints * sizeof(double))) != WOST_OK) return rc;
    if ((rc = s->ws_ctr.ensure(16 * sizeof(unsigned long long))) != WOST_OK) return rc;
    double *shell_val = s->ws_status.as<double>();
    uint8_t *status = reinterpret_cast<uint8_t *>(shell_val + npoints);
    unsigned long long *ctr = s->ws_ctr.as<unsigned long long>();
    WOST_CUDA(cudaMemsetAsync(s->ws_sum.ptr, 0, npoints * sizeof(double), st));
    WOST_CUDA(cudaMemsetAsync(s->ws_sum2.ptr, 0, npoints * sizeof(double), st));
    WOST_CUDA(cudaMemsetAsync(ctr, 0, 16 * sizeof(unsigned long long), st));

    WalkArgs a{};
    a.sc = s->dev;
    a.points = pts;
    a.status = status;
    a.npoints = npoints;
    a.walk_begin = ex.walk_begin;
    a.work_ctr = ctr;
    a.sum = s->ws_sum.as<double>();
    a.sum2 = s->ws_sum2.as<double>();
    a.eps = (float)eps;
    a.eps64 = eps;
    a.maxsteps = maxsteps;
    a.key0 = (uint32_t)ex.seed;
    a.key1 = (uint32_t)(ex.seed >> 32) + s->scene_id;
    a.stat = ctr + 8;
    a.err = err_flag();
    a.rr_depth = ex.rr_depth;
    a.rr_q = ex.rr_survival;

    if (D == 2) classify_kernel<2><<<blocks_for(npoints, 128), 128, 0, st>>>(a, shell_val);
    else classify_kernel<3><<<blocks_for(npoints, 128), 128, 0, st>>>(a, shell_val);
    WOST_CUDA(cudaGetLastError());

    CallTiming tm;
    tm.launches = 1;   // classify
    if (!guided) {
        a.total = (unsigned long long)npoints * nwalks;
        static int occ[4] = {0, 0, 0, 0};
        if (!occ[D]) {
            int n = 0;
            if (D == 2) WOST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, plain_walk_kernel<2>, kPlainBlock, 0));
            else WOST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, plain_walk_kernel<3>, kPlainBlock, 0));
            occ[D] = std::max(1, n);
        }
        int cps = ex.ctas_per_sm > 0 ? std::min(ex.ctas_per_sm, occ[D]) : occ[D];
        int grid = num_sms() * cps;
        tm.mark(tm.walk, st);
        if (D == 2) plain_walk_kernel<2><<<grid, kPlainBlock, 0, st>>>(a);
        else plain_walk_kernel<3><<<grid, kPlainBlock, 0, st>>>(a);
        tm.mark(tm.walk, st);
        tm.launches++;
        tm.walk_launches++;
        WOST_CUDA(cudaGetLastError());
    } else {
        rc = guided_solve(s, field, a, nwalks, ex, st, stats, ex.walk_begin, tm);
        if (rc != WOST_OK) return rc;
    }
    // outputs
    double *om = out_mean, *ov = out_var;
    if (!ex.out_on_device) {
        if ((rc = s->ws_out.ensure(2 * npoints * sizeof(double))) != WOST_OK) return rc;
        om = s->ws_out.as<double>();
        ov = out_var ? om + npoints : nullptr;
    }
    finalize_kernel<<<blocks_for(npoints, 256), 256, 0, st>>>(status, shell_val, a.sum, a.sum2, npoints, nwalks, om, ov);
    WOST_CUDA(cudaGetLastError());
    if (!ex.out_on_device) {
        WOST_CUDA(cudaMemcpyAsync(out_mean, om, npoints * sizeof(double), cudaMemcpyDeviceToHost, st));
        if (out_var) WOST_CUDA(cudaMemcpyAsync(out_var, ov, npoints * sizeof(double), cudaMemcpyDeviceToHost, st));
    }
    unsigned long long hs[8];
    WOST_CUDA(cudaMemcpyAsync(hs, ctr + 8, sizeof(hs), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaStreamSynchronize(st));
    if ((rc = check_err_flag(st)) != WOST_OK) return rc;
    tm.launches++;   // finalize
    if (stats) {
        stats->walk_steps = (int64_t)hs[0];
        stats->truncated = (int64_t)hs[1];
        stats->walks = (int64_t)hs[2];
        stats->node_visits = (int64_t)hs[3];
        stats->prim_visits = (int64_t)(hs[4] + hs[5] + hs[6]);
        stats->dir_prim_visits = (int64_t)hs[4];
        stats->sil_prim_visits = (int64_t)hs[5];
        stats->neu_prim_visits = (int64_t)hs[6];
        stats->alg_bytes = walk_alg_bytes(D, guided, hs, stats->records);
        stats->ms_walk = CallTiming::sum(tm.walk);
        stats->ms_train = CallTiming::sum(tm.train);
        stats->kernel_launches = tm.launches;
        stats->walk_launches = tm.walk_launches;
    }
    return WOST_OK;
}

// ---- query entry points ----------------------------------------------------------
extern "C" wost_status wost_query_closest(wost_scene *s, const double *points, int64_t n, int32_t *out_prim,
                                          float *out_dist) {
    if (!s || (n > 0 && (!points || !out_prim || !out_dist)) || n < 0) { set_error("wost_query_closest: invalid argument"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(s->device, "wost_query_closest")) return dc;
    if (n == 0) return WOST_OK;
    Staged<double> p;
    wost_status rc;
    if ((rc = stage_in(points, (size_t)n * s->dim, false, p)) != WOST_OK) return rc;
    int32_t *di;
    float *dd;
    WOST_CUDA(cudaMalloc(&di, n * sizeof(int32_t)));
    WOST_CUDA(cudaMalloc(&dd, n * sizeof(float)));
    if (s->dim == 2) q_closest_kernel<2><<<blocks_for(n, 128), 128>>>(s->dev, p.dev, n, di, dd, err_flag());
    else q_closest_kernel<3><<<blocks_for(n, 128), 128>>>(s->dev, p.dev, n, di, dd, err_flag());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(out_prim, di, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_dist, dd, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(di);
    cudaFree(dd);
    if (e != cudaSuccess) return cuda_status(e, "wost_query_closest");
    return check_err_flag(0);
}

extern "C" wost_status wost_query_silhouette(wost_scene *s, const double *points, int64_t n, int64_t *out_elem,
                                             float *out_dist) {
    if (!s || (n > 0 && (!points || !out_elem || !out_dist)) || n < 0) { set_error("wost_query_silhouette: invalid argument"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(s->device, "wost_query_silhouette")) return dc;
    if (n == 0) return WOST_OK;
    Staged<double> p;
    wost_status rc;
    if ((rc = stage_in(points, (size_t)n * s->dim, false, p)) != WOST_OK) return rc;
    int64_t *di;
    float *dd;
    WOST_CUDA(cudaMalloc(&di, n * sizeof(int64_t)));
    WOST_CUDA(cudaMalloc(&dd, n * sizeof(float)));
    if (s->dim == 2) q_sil_kernel<2><<<blocks_for(n, 128), 128>>>(s->dev, s->sil_key, p.dev, n, di, dd, err_flag());
    else q_sil_kernel<3><<<blocks_for(n, 128), 128>>>(s->dev, s->sil_key, p.dev, n, di, dd, err_flag());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(out_elem, di, n * sizeof(int64_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_dist, dd, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(di);
    cudaFree(dd);
    if (e != cudaSuccess) return cuda_status(e, "wost_query_silhouette");
    return check_err_flag(0);
}

namespace {
wost_status query_ray(bool exit_only, const char *who, wost_scene *s, const double *org, const double *dir,
                      const double *tmax, const int32_t *skip, int64_t n, int32_t *out_prim, float *out_t) {
    if (!s || n < 0 || (n > 0 && (!org || !dir || !tmax || !out_prim || !out_t))) {
        set_error(std::string(who) + ": invalid argument");
        return WOST_ERR_INVALID_ARG;
    }
    if (wost_status dc = check_device(s->device, who)) return dc;
    if (n == 0) return WOST_OK;
    if (skip)
        for (int64_t i = 0; i < n; ++i)
            if (skip[i] >= s->nprims) { set_error(std::string(who) + ": skip id out of range"); return WOST_ERR_INVALID_ARG; }
    Staged<double> po, pv, pt;
    Staged<int32_t> ps;
    wost_status rc;
    if ((rc = stage_in(org, (size_t)n * s->dim, false, po)) != WOST_OK) return rc;
    if ((rc = stage_in(dir, (size_t)n * s->dim, false, pv)) != WOST_OK) return rc;
    if ((rc = stage_in(tmax, (size_t)n, false, pt)) != WOST_OK) return rc;
    if ((rc = stage_in(skip, (size_t)n, false, ps)) != WOST_OK) return rc;
    int *slot_of = nullptr;
    WOST_CUDA(cudaMalloc(&slot_of, (s->nprims + 1) * sizeof(int)));
    WOST_CUDA(cudaMemset(slot_of, 0xff, (s->nprims + 1) * sizeof(int)));
    if (s->nneu > 0) invert_ids_kernel<<<blocks_for(s->nneu, 128), 128>>>(s->dev.neu.ids, s->nneu, slot_of);
    int32_t *di;
    float *dt;
    WOST_CUDA(cudaMalloc(&di, n * sizeof(int32_t)));
    WOST_CUDA(cudaMalloc(&dt, n * sizeof(float)));
    const int nb = blocks_for(n, 128);
    if (s->dim == 2 && exit_only) q_ray_kernel<2, true><<<nb, 128>>>(s->dev, po.dev, pv.dev, pt.dev, ps.dev, slot_of, n, di, dt, err_flag());
    else if (s->dim == 2) q_ray_kernel<2, false><<<nb, 128>>>(s->dev, po.dev, pv.dev, pt.dev, ps.dev, slot_of, n, di, dt, err_flag());
    else if (exit_only) q_ray_kernel<3, true><<<nb, 128>>>(s->dev, po.dev, pv.dev, pt.dev, ps.dev, slot_of, n, di, dt, err_flag());
    else q_ray_kernel<3, false><<<nb, 128>>>(s->dev, po.dev, pv.dev, pt.dev, ps.dev, slot_of, n, di, dt, err_flag());
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpy(out_prim, di, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(out_t, dt, n * sizeof(float), cudaMemcpyDeviceToHost);
    cudaFree(di);
    cudaFree(dt);
    cudaFree(slot_of);
    if (e != cudaSuccess) return cuda_status(e, who);
    return check_err_flag(0);
}
}  // namespace

extern "C" wost_status wost_query_ray(wost_scene *s, const double *org, const double *dir, const double *tmax,
                                      const int32_t *skip, int64_t n, int32_t *out_prim, float *out_t) {
    return query_ray(false, "wost_query_ray", s, org, dir, tmax, skip, n, out_prim, out_t);
}

extern "C" wost_status wost_query_ray_exit(wost_scene *s, const double *org, const double *dir, const double *tmax,
                                           const int32_t *skip, int64_t n, int32_t *out_prim, float *out_t) {
    return query_ray(true, "wost_query_ray_exit", s, org, dir, tmax, skip, n, out_prim, out_t);
}
