// Host-side internals of libwost shared between translation units.
#pragma once
#include <cuda_runtime.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/wost.h"
#include "common.cuh"

namespace wost {

void set_error(const std::string &msg);
wost_status cuda_status(cudaError_t e, const char *what);

#define WOST_CUDA(call)                                                  \
    do {                                                                 \
        cudaError_t e_ = (call);                                         \
        if (e_ != cudaSuccess) return ::wost::cuda_status(e_, #call);    \
    } while (0)

// device buffer that grows on demand and is freed with its owner
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    wost_status ensure(size_t n);
    void release();
    template <class T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

struct FieldDev;  // defined in field.cuh

// Kernel attributes belong to a device: set-up that must run once per device
// (and per key) runs under a lock the first time it is asked for while that
// device is current; a failed set-up runs again on the next call.
wost_status once_per_device(int key, const std::function<wost_status()> &f);

}  // namespace wost

struct wost_scene {
    int dim = 0;
    int device = -1;              // CUDA device the scene's data lives on (current at creation)
    int64_t nverts = 0, nprims = 0;
    uint32_t scene_id = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    wost::DevScene dev{};
    std::vector<void *> allocs;
    int64_t *sil_key = nullptr;   // device: canonical silhouette element id per leaf slot
    int ndir = 0, nneu = 0, nsil = 0;
    int depth_dir = 0, depth_neu = 0, depth_sil = 0;
    // per-solve workspace (grown on demand)
    wost::DevBuf ws_points, ws_status, ws_sum, ws_sum2, ws_ctr, ws_out;
    wost::DevBuf ws_wf;                        // guided wavefront slots
    wost::DevBuf ws_order;                     // walk lengths and launch order of the guided launches
    int64_t order_n = 0;                       // point count the order in ws_order was made for (0: none)
    unsigned long long *pinned = nullptr;      // host-pinned words for wavefront progress
    ~wost_scene();
};

namespace wost {
// CUDA-event timing of the kernels of one call (summed after the final sync)
struct CallTiming {
    std::vector<cudaEvent_t> walk, train;   // start/stop pairs
    int64_t launches = 0, walk_launches = 0;
    void mark(std::vector<cudaEvent_t> &v, cudaStream_t st) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        v.push_back(e);
    }
    static double sum(std::vector<cudaEvent_t> &v) {
        double ms = 0;
        for (size_t i = 0; i + 1 < v.size(); i += 2) {
            float m = 0;
            cudaEventElapsedTime(&m, v[i], v[i + 1]);
            ms += m;
        }
        return ms;
    }
    ~CallTiming() {
        for (auto e : walk) cudaEventDestroy(e);
        for (auto e : train) cudaEventDestroy(e);
    }
};
// launch helpers implemented in walk.cu
int num_sms();
// algorithmic bytes of walk launches from their statistics hs[0..6]
// (walk-steps, truncated, walks, node / Dirichlet / silhouette / Neumann visits)
double walk_alg_bytes(int D, bool guided, const unsigned long long *hs, int64_t records);
int *device_err_flag();                  // device word: bit 0 stack overflow, bit 1 wait timeout
wost_status device_check(cudaStream_t st);
// WOST_OK if `device` (a scene's or field's) is the current CUDA device; else
// WOST_ERR_INVALID_ARG (or the CUDA error of the lookup) with a message naming
// `who`.  Called before any launch: a kernel on the wrong device would read
// another GPU's pointers.
wost_status check_device(int device, const char *who);
// walker warps a guided launch may take (exec walker_warps: 0 = automatic)
bool ws_walker_warps_valid(int w);
}
