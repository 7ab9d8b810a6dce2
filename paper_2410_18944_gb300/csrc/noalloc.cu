// Plain walk-on-stars solve that allocates no device memory.
//
// wost_solve obtains its per-solve work buffers with cudaMalloc the first
// time it needs them.  Some callers cannot allow that: for example a process
// in which another component has taken the whole device memory pool, or a
// tight loop that must not pay the device-wide synchronisation that
// cudaFree implies.  For them, wost_solve_plain_static runs the same plain
// walk with all of its scratch memory (per-point FP64 sums, point status,
// work counter, statistics, error word) in one fixed array that lives in
// this library's device image.  The array exists on every GPU that loads the
// library, for as long as the process runs, whether or not it is used.
//
// Set-up: the device address of the array is looked up with
// cudaGetSymbolAddress once per device, by the first call made while that
// device is current; make that first call before any stream capture.
// All calls share the one array and it keeps the last call's contents; each
// call clears what must start at zero.  Two calls whose work overlaps on the
// GPU (e.g. on different streams) race on the array.
#include <mutex>

#include "internal.h"
#include "walkstep.cuh"

namespace wost {
namespace {

constexpr int64_t kStaticMaxPoints = WOST_STATIC_MAX_POINTS;
constexpr size_t kCtrlBytes = 256;   // work counter, 8 statistics, error word
constexpr size_t kStaticBytes = kCtrlBytes + (size_t)kStaticMaxPoints * (3 * sizeof(double) + 1);

static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

struct StaticView {
    unsigned long long *work_ctr;   // [0]
    unsigned long long *stat;       // [1..8]
    int *err;                       // byte 80
    double *sum, *sum2, *shell;
    uint8_t *status;
};

StaticView view_of(unsigned char *base) {
    StaticView v;
    v.work_ctr = reinterpret_cast<unsigned long long *>(base);
    v.stat = v.work_ctr + 1;
    v.err = reinterpret_cast<int *>(base + 80);
    v.sum = reinterpret_cast<double *>(base + kCtrlBytes);
    v.sum2 = v.sum + kStaticMaxPoints;
    v.shell = v.sum2 + kStaticMaxPoints;
    v.status = reinterpret_cast<uint8_t *>(v.shell + kStaticMaxPoints);
    return v;
}

// per-device address of the array (looked up once per device)
constexpr int kMaxDevices = 64;
unsigned char *g_static_addr[kMaxDevices] = {nullptr};
std::mutex g_static_mutex;

wost_status static_base(unsigned char **out) {
    int dev = 0;
    WOST_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) {
        set_error("wost_solve_plain_static: device index out of range");
        return WOST_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> lock(g_static_mutex);
    if (!g_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return cuda_status(e, "wost_solve_plain_static: cudaGetSymbolAddress");
        g_static_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_static_addr[dev];
    return WOST_OK;
}

template <int D>
__global__ void static_classify_kernel(WalkArgs a, double *shell) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.npoints) return;
    float x[D];
    for (int k = 0; k < D; ++k) x[k] = (float)a.points[i * D + k];
    const float dir[3] = {0.5377844f, 0.7924136f, 0.2876523f};
    float v[D], nn = 0.f;
    for (int k = 0; k < D; ++k) { v[k] = dir[k]; nn += v[k] * v[k]; }
    for (int k = 0; k < D; ++k) v[k] *= rsqrtf(nn);
    int c = ray_count<D>(a.sc.dir, x, v, a.err) + ray_count<D>(a.sc.neu, x, v, a.err);
    uint8_t st = 0;
    double val = 0.0;
    if ((c & 1) == 0) {
        st = 2;
        val = __longlong_as_double(0x7ff8000000000000LL);
    } else {
        float bd2;
        int slot = closest_dirichlet<D>(a.sc.dir, x, bd2, a.err);
        double q[3];
        if (dirichlet_dist64<D>(a.sc.dir, slot, x, q) <= a.eps64) {
            st = 1;
            float xb[3] = {(float)q[0], (float)q[1], D == 3 ? (float)q[2] : 0.f};
            val = eval_fn<D>(a.sc.g, xb);
        }
    }
    const_cast<uint8_t *>(a.status)[i] = st;
    shell[i] = val;
}

// the plain persistent walk loop, on the static scratch
template <int D>
__global__ void __launch_bounds__(128) static_walk_kernel(WalkArgs a) {
    Walk<D> w;
    Visits vis;
    bool active = false, exhausted = false;
    unsigned long long nsteps = 0, ntrunc = 0, nwalks = 0;
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
        if (!active) continue;
        nsteps++;
        float r, S, gv;
        bool trunc = false;
        bool ended = step_geometry<D>(w, a, r, S, gv, trunc, &vis);
        float nu[D];
        if (!ended) {
            U4 u = philox(w.pid, w.wid, (uint32_t)w.k, P_DIR, a.key0, a.key1);
            uniform_dir<D>(u01(u.x), u01(u.y), nu);
            if (w.prim >= 0) {
                float dn = dotv<D>(nu, w.n);
                if (dn < 0.f) reflect<D>(nu, w.n);
                ended = dn == 0.f;
            }
        }
        if (ended) {
            finish_walk(a, w.pid, w.acc);
            ntrunc += trunc;
            active = false;
        } else {
            step_move<D>(w, a, nu, r, &vis);
        }
    }
    flush_counters(a, nsteps, ntrunc, nwalks, vis);
}

__global__ void static_finalize_kernel(const uint8_t *status, const double *shell, const double *sum,
                                       const double *sum2, int64_t n, int nw, double *mean, double *var) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (status[i] != 0) {
        mean[i] = shell[i];
        if (var) var[i] = status[i] == 1 ? 0.0 : shell[i];
        return;
    }
    double m = sum[i] / nw;
    mean[i] = m;
    if (var) {
        double v = nw > 1 ? (sum2[i] - nw * m * m) / ((double)nw * (nw - 1)) : 0.0;
        var[i] = v > 0 ? v : 0.0;
    }
}

}  // namespace
}  // namespace wost

using namespace wost;

extern "C" wost_status wost_solve_plain_static(wost_scene *s, const double *points_dev, int64_t npoints,
                                               int32_t nwalks, double eps, int32_t maxsteps, uint64_t seed,
                                               void *stream, double *out_mean_dev, double *out_var_dev,
                                               int64_t *out_walk_steps) {
    if (!s || npoints < 0 || nwalks <= 0 || !(eps > 0) || maxsteps < 0 ||
        (npoints > 0 && (!points_dev || !out_mean_dev))) {
        set_error("wost_solve_plain_static: invalid argument");
        return WOST_ERR_INVALID_ARG;
    }
    if (npoints > kStaticMaxPoints) {
        set_error("wost_solve_plain_static: npoints exceeds WOST_STATIC_MAX_POINTS (262144); "
                  "use wost_solve or split the points");
        return WOST_ERR_INVALID_ARG;
    }
    unsigned char *base = nullptr;
    wost_status rc = static_base(&base);
    if (rc != WOST_OK) return rc;
    if (out_walk_steps) *out_walk_steps = 0;
    if (npoints == 0) return WOST_OK;
    cudaStream_t st = (cudaStream_t)stream;
    StaticView v = view_of(base);
    // what must start at zero: counters, statistics, error word, the sums
    WOST_CUDA(cudaMemsetAsync(base, 0, kCtrlBytes, st));
    WOST_CUDA(cudaMemsetAsync(v.sum, 0, npoints * sizeof(double), st));
    WOST_CUDA(cudaMemsetAsync(v.sum2, 0, npoints * sizeof(double), st));
    const int D = s->dim;
    WalkArgs a{};
    a.sc = s->dev;
    a.points = points_dev;
    a.status = v.status;
    a.npoints = npoints;
    a.walk_begin = 0;
    a.total = (unsigned long long)npoints * nwalks;
    a.work_ctr = v.work_ctr;
    a.sum = v.sum;
    a.sum2 = v.sum2;
    a.eps = (float)eps;
    a.eps64 = eps;
    a.maxsteps = maxsteps;
    a.key0 = (uint32_t)seed;
    a.key1 = (uint32_t)(seed >> 32) + s->scene_id;
    a.stat = v.stat;
    a.err = v.err;
    const int blocks = (int)((npoints + 127) / 128);
    const int grid = num_sms() * 8;
    if (D == 2) {
        static_classify_kernel<2><<<blocks, 128, 0, st>>>(a, v.shell);
        static_walk_kernel<2><<<grid, 128, 0, st>>>(a);
    } else {
        static_classify_kernel<3><<<blocks, 128, 0, st>>>(a, v.shell);
        static_walk_kernel<3><<<grid, 128, 0, st>>>(a);
    }
    static_finalize_kernel<<<(int)((npoints + 255) / 256), 256, 0, st>>>(v.status, v.shell, v.sum, v.sum2, npoints,
                                                                        nwalks, out_mean_dev, out_var_dev);
    WOST_CUDA(cudaGetLastError());
    unsigned long long steps = 0;
    int err = 0;
    WOST_CUDA(cudaMemcpyAsync(&steps, v.stat, sizeof(steps), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaMemcpyAsync(&err, v.err, sizeof(err), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaStreamSynchronize(st));
    if (err) {
        set_error("wost_solve_plain_static: BVH traversal stack overflow");
        return WOST_ERR_CUDA;
    }
    if (out_walk_steps) *out_walk_steps = (int64_t)steps;
    return WOST_OK;
}
