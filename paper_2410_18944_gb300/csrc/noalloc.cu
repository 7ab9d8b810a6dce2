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
// device is current.
// All calls share the one array and it keeps the last call's contents; each
// call clears what must start at zero.  Two calls whose work overlaps on the
// GPU (e.g. on different streams) race on the array.
#include <mutex>

#include "internal.h"
#include "jobsrc.cuh"

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
__global__ void static_classify_kernel(WalkArgs a, double *shell_value) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= a.npoints) return;
    double val;
    const_cast<uint8_t *>(a.status)[i] = classify_point<D>(a.sc, a.eps64, a.points + i * D, a.err, val);
    shell_value[i] = val;
}

// the plain persistent walk loop, on the static scratch
template <int D>
__global__ void __launch_bounds__(128) static_walk_kernel(const __grid_constant__ WalkArgs a) {
    plain_loop<D>(SoloSrc<D>{a, nullptr, RecDest{}, &a.sc}, a.stat);
}

__global__ void static_finalize_kernel(const uint8_t *status, const double *shell_value, const double *sum,
                                const double *sum2, int64_t n, int nw, double *mean, double *var) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    finalize_point(status[i], shell_value[i], sum[i], sum2[i], nw, mean + i, var ? var + i : nullptr);
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
    // the scene's BVHs must be on the current device: the array looked up
    // below, and the kernels, are the current device's
    if (wost_status dc = check_device(s->device, "wost_solve_plain_static")) return dc;
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
