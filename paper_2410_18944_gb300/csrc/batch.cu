// Many scenes in one persistent launch (wost_solve_batch / wost_batch_*).
//
// A plan lays the work items of all jobs out job-major (a job's items are
// its walks of all its points, walk-major as in wost_solve) and splits them
// into launches: one launch for every walk when nothing trains; with online
// training (Sec. 5.2) one launch per training round (walk r of every point
// of every job that has it), each followed by the training steps of the
// jobs' fields, then one launch for all the remaining walks.  Walkers take
// items from one global counter per launch and find their job by binary
// search over the launch's segment table, so uneven jobs share the SMs with
// no per-job launch and no tail per job.
//
// The plan is captured once into a CUDA graph (memsets, point
// classification, walk launches, training steps, per-point finalisation)
// and replayed by wost_batch_run.  Before capture, an autotuner times the
// candidate launch shapes on one calibration walk per point of every job:
// resident CTAs per SM for the plain walk; for the guided walk the walker
// warps per CTA (16 or 28 beside the 4 decode servers: the queue of rows
// that feeds a decode tile) and the decode-tile flush threshold.
#include <algorithm>
#include <cstring>
#include <unordered_set>
#include <vector>

#include "guided_ws.cuh"
#include "internal.h"

namespace wost {

wost_status train_launch(wost_field *f, int dim, cudaStream_t st, bool apply_adam, float *loss_out_dev,
                         long long off = -1);
wost_status train_prepare(int dim);
wost_status ensure_records(wost_field *f, int64_t cap, size_t scratch_bytes);

namespace {

constexpr int kBatchPlainBlock = 128;
constexpr int kBatchGuidedSmem = ws_smem_bytes(true);
// counter block of a plan (unsigned long long words)
constexpr int kCtrStat = 8;       // [8, 15): launch statistics
constexpr int kCtrRec = 16;       // [16, 18): records appended / dropped over all rounds
constexpr int kCtrCalib = 23;     // work counter of calibration launches
constexpr int kCtrWork = 24;      // [24, 24 + launches): work counter per launch

struct BatchGuidedArgs {
    BatchArgs b;
    WsOpts o;
};

template <int D>
__global__ void __launch_bounds__(kBatchPlainBlock) batch_plain_kernel(const __grid_constant__ BatchArgs b) {
    plain_loop<D>(BatchSrc<D>{b}, b.stat);
}

template <int D, int W>
__global__ void __launch_bounds__(ws_threads(W), 1) batch_guided_kernel(const __grid_constant__ BatchGuidedArgs g) {
    extern __shared__ __align__(1024) uint8_t sm[];
    guided_ws_body<D, true, W>(BatchSrc<D>{g.b}, g.o, sm);
}

// job owning batch point i: the last job whose point_off <= i
__device__ __forceinline__ int find_job(const DevJob *jobs, int njobs, int64_t i) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (jobs[mid].point_off <= i) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

template <int D>
__global__ void batch_classify_kernel(const DevJob *jobs, int njobs, int64_t n, uint8_t *status, double *shell,
                                      int *err) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DevJob &J = jobs[find_job(jobs, njobs, i)];
    double val;
    status[i] = classify_point<D>(J.sc, J.eps64, J.points + (i - J.point_off) * D, err, val);
    shell[i] = val;
}

__global__ void batch_finalize_kernel(const DevJob *jobs, int njobs, int64_t n, const uint8_t *status,
                                      const double *shell, const double *sum, const double *sum2) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const DevJob &J = jobs[find_job(jobs, njobs, i)];
    const int64_t p = i - J.point_off;
    finalize_point(status[i], shell[i], sum[i], sum2[i], J.nwalks, J.out_mean + p, J.out_var ? J.out_var + p : nullptr);
}

// adds (when add) every job's record counters into acc and clears them
__global__ void batch_rec_roll_kernel(const DevJob *jobs, int njobs, unsigned long long *acc, int add) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= njobs) return;
    unsigned long long *c = jobs[j].rd.ctr;
    if (!c) return;
    if (add) {
        atomicAdd(acc, c[0]);
        atomicAdd(acc + 1, c[1]);
    }
    c[0] = 0;
    c[1] = 0;
}

int blocks_of(int64_t n, int bs) { return (int)((n + bs - 1) / bs); }

}  // namespace
}  // namespace wost

using namespace wost;

struct wost_batch {
    int dim = 0;
    int device = -1;                 // the device of its jobs' scenes and fields
    bool guided = false, record = false;
    wost_exec ex{};
    std::vector<wost_job> jobs;
    std::vector<DevJob> hjobs;
    int64_t total_points = 0;
    DevBuf djobs, dsegs, status, shell, sums, ctr, scratch;
    struct Launch {
        int seg0 = 0, nseg = 0;
        unsigned long long total = 0;
        bool record = false;
        std::vector<int> train_jobs;
    };
    std::vector<Launch> launches;
    Launch calib;
    wost_batch_info info{};
    int cps = 1;
    uint32_t polls = kFlushPolls;
    int walkers = kWsWalkerWarps;
    int scratch_steps = 1;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t gexec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;

    unsigned long long *ctr_at(int i) const { return ctr.as<unsigned long long>() + i; }
    double *sum() const { return sums.as<double>(); }
    double *sum2() const { return sums.as<double>() + total_points; }

    BatchArgs args(const Launch &L, unsigned long long *work) const {
        BatchArgs b{};
        b.jobs = djobs.as<DevJob>();
        b.segs = dsegs.as<DevSeg>() + L.seg0;
        b.nseg = L.nseg;
        b.total = L.total;
        b.work_ctr = work;
        b.status = status.as<uint8_t>();
        b.sum = sum();
        b.sum2 = sum2();
        b.stat = ctr_at(kCtrStat);
        b.err = device_err_flag();
        return b;
    }

    wost_status launch_walk(const Launch &L, unsigned long long *work, cudaStream_t st, int cps_, uint32_t polls_,
                            int walkers_) {
        const BatchArgs b = args(L, work);
        if (!guided) {
            const int grid = num_sms() * cps_;
            if (dim == 2) batch_plain_kernel<2><<<grid, kBatchPlainBlock, 0, st>>>(b);
            else batch_plain_kernel<3><<<grid, kBatchPlainBlock, 0, st>>>(b);
        } else {
            BatchGuidedArgs g{};
            g.b = b;
            g.o.c_mode = ex.c_mode;
            g.o.c_fixed = ex.c_fixed;
            g.o.reflect = ex.reflect;
            g.o.record = L.record;
            g.o.scratch = L.record ? scratch.as<float>() : nullptr;
            g.o.scratch_steps = scratch_steps;
            g.o.flush_polls = polls_;
            g.o.wait_ns = ex.wait_ns > 0 ? (unsigned long long)ex.wait_ns : kWaitNs;
            g.o.err = b.err;
            g.o.stat = b.stat;
            constexpr int tn = ws_threads(kWsWalkerWarps), tw = ws_threads(kWsWalkersWide);
            const bool wide = walkers_ == kWsWalkersWide;
            if (dim == 2 && wide) batch_guided_kernel<2, kWsWalkersWide><<<num_sms(), tw, kBatchGuidedSmem, st>>>(g);
            else if (dim == 2) batch_guided_kernel<2, kWsWalkerWarps><<<num_sms(), tn, kBatchGuidedSmem, st>>>(g);
            else if (wide) batch_guided_kernel<3, kWsWalkersWide><<<num_sms(), tw, kBatchGuidedSmem, st>>>(g);
            else batch_guided_kernel<3, kWsWalkerWarps><<<num_sms(), tn, kBatchGuidedSmem, st>>>(g);
        }
        WOST_CUDA(cudaGetLastError());
        return WOST_OK;
    }

    // everything a run does, enqueued on st (the capture stream)
    wost_status enqueue(cudaStream_t st) {
        const int nj = (int)hjobs.size();
        const DevJob *dj = djobs.as<DevJob>();
        WOST_CUDA(cudaMemsetAsync(sums.ptr, 0, 2 * total_points * sizeof(double), st));
        WOST_CUDA(cudaMemsetAsync(ctr.ptr, 0, (kCtrWork + launches.size()) * sizeof(unsigned long long), st));
        if (dim == 2) batch_classify_kernel<2><<<blocks_of(total_points, 128), 128, 0, st>>>(dj, nj, total_points, status.as<uint8_t>(), shell.as<double>(), device_err_flag());
        else batch_classify_kernel<3><<<blocks_of(total_points, 128), 128, 0, st>>>(dj, nj, total_points, status.as<uint8_t>(), shell.as<double>(), device_err_flag());
        WOST_CUDA(cudaGetLastError());
        bool rolled = false;
        for (size_t l = 0; l < launches.size(); ++l) {
            const Launch &L = launches[l];
            if (L.record) {
                batch_rec_roll_kernel<<<blocks_of(nj, 64), 64, 0, st>>>(dj, nj, ctr_at(kCtrRec), rolled ? 1 : 0);
                rolled = true;
            }
            wost_status rc = launch_walk(L, ctr_at(kCtrWork + (int)l), st, cps, polls, walkers);
            if (rc != WOST_OK) return rc;
            for (int j : L.train_jobs) {
                rc = train_launch(jobs[j].field, dim, st, true, nullptr);
                if (rc != WOST_OK) return rc;
            }
        }
        if (rolled) batch_rec_roll_kernel<<<blocks_of(nj, 64), 64, 0, st>>>(dj, nj, ctr_at(kCtrRec), 1);
        batch_finalize_kernel<<<blocks_of(total_points, 256), 256, 0, st>>>(dj, nj, total_points, status.as<uint8_t>(),
                                                                            shell.as<double>(), sum(), sum2());
        WOST_CUDA(cudaGetLastError());
        return WOST_OK;
    }

    // times the calibration launch under the candidate shapes; keeps the fastest
    wost_status autotune() {
        struct Cand { int cps; uint32_t polls; int walkers; };
        std::vector<Cand> cand;
        const int fixed_w = ex.walker_warps > 0 ? ex.walker_warps : kWsWalkerWarps;
        if (!guided) {
            int occ = 1;
            if (dim == 2) WOST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_plain_kernel<2>, kBatchPlainBlock, 0));
            else WOST_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, batch_plain_kernel<3>, kBatchPlainBlock, 0));
            occ = std::max(1, occ);
            for (int c = 1; c <= occ; ++c) cand.push_back({c, kFlushPolls, kWsWalkerWarps});
        } else {
            for (int w : {kWsWalkerWarps, kWsWalkersWide}) {
                if (ex.walker_warps > 0 && w != ex.walker_warps) continue;
                for (uint32_t p : {256u, 1024u, 4096u}) cand.push_back({1, p, w});
            }
        }
        if (ex.ctas_per_sm > 0 || calib.total == 0) {
            cps = ex.ctas_per_sm > 0 ? (guided ? 1 : std::min(ex.ctas_per_sm, cand.back().cps)) : cand.back().cps;
            polls = kFlushPolls;
            walkers = fixed_w;
            info.candidates = 0;
            return WOST_OK;
        }
        // calibration walks write the batch sums; every run clears them first
        WOST_CUDA(cudaMemsetAsync(ctr.ptr, 0, kCtrWork * sizeof(unsigned long long), cap));
        if (dim == 2) batch_classify_kernel<2><<<blocks_of(total_points, 128), 128, 0, cap>>>(djobs.as<DevJob>(), (int)hjobs.size(), total_points, status.as<uint8_t>(), shell.as<double>(), device_err_flag());
        else batch_classify_kernel<3><<<blocks_of(total_points, 128), 128, 0, cap>>>(djobs.as<DevJob>(), (int)hjobs.size(), total_points, status.as<uint8_t>(), shell.as<double>(), device_err_flag());
        WOST_CUDA(cudaGetLastError());
        double best = 1e300, worst = 0;
        for (auto &c : cand) {
            float ms = 0;
            for (int rep = 0; rep < 2; ++rep) {   // first run warms the caches
                WOST_CUDA(cudaMemsetAsync(ctr_at(kCtrCalib), 0, sizeof(unsigned long long), cap));
                WOST_CUDA(cudaEventRecord(ev0, cap));
                wost_status rc = launch_walk(calib, ctr_at(kCtrCalib), cap, c.cps, c.polls, c.walkers);
                if (rc != WOST_OK) return rc;
                WOST_CUDA(cudaEventRecord(ev1, cap));
            }
            WOST_CUDA(cudaEventSynchronize(ev1));
            WOST_CUDA(cudaEventElapsedTime(&ms, ev0, ev1));
            if (ms < best) { best = ms; cps = c.cps; polls = c.polls; walkers = c.walkers; }
            worst = std::max(worst, (double)ms);
        }
        wost_status rc = device_check(cap);
        if (rc != WOST_OK) return rc;
        info.candidates = (int)cand.size();
        info.best_ms = best;
        info.worst_ms = worst;
        return WOST_OK;
    }

    ~wost_batch() {
        if (cap) cudaStreamSynchronize(cap);
        if (gexec) cudaGraphExecDestroy(gexec);
        if (graph) cudaGraphDestroy(graph);
        if (ev0) cudaEventDestroy(ev0);
        if (ev1) cudaEventDestroy(ev1);
        if (cap) cudaStreamDestroy(cap);
        for (DevBuf *b : {&djobs, &dsegs, &status, &shell, &sums, &ctr, &scratch}) b->release();
    }
};

namespace {

wost_status validate(int32_t njobs, const wost_job *jobs, int32_t guided, const wost_exec &ex) {
    if (njobs <= 0 || !jobs) { set_error("wost_batch_create: no jobs"); return WOST_ERR_INVALID_ARG; }
    if (ex.rr_depth < 0 || (ex.rr_depth > 0 && !(ex.rr_survival > 0.f && ex.rr_survival <= 1.f))) {
        set_error("wost_batch_create: rr_depth must be >= 0 and rr_survival in (0, 1]");
        return WOST_ERR_INVALID_ARG;
    }
    if (!ws_walker_warps_valid(ex.walker_warps)) {
        set_error("wost_batch_create: walker_warps must be 0, 16 or 28");
        return WOST_ERR_INVALID_ARG;
    }
    const int dim = jobs[0].scene ? jobs[0].scene->dim : 0;
    std::unordered_set<const wost_field *> fields;
    for (int j = 0; j < njobs; ++j) {
        const wost_job &J = jobs[j];
        std::string at = "wost_batch_create: job " + std::to_string(j) + ": ";
        if (!J.scene) { set_error(at + "null scene"); return WOST_ERR_INVALID_ARG; }
        if (J.scene->dim != dim) { set_error(at + "all jobs of a batch must have the same dimension"); return WOST_ERR_INVALID_ARG; }
        if (wost_status dc = check_device(J.scene->device, "wost_batch_create (scene)")) return dc;
        if (J.npoints < 0 || J.npoints > (int64_t)UINT32_MAX || J.nwalks <= 0 || !(J.eps > 0) || J.maxsteps < 0) {
            set_error(at + "invalid npoints / nwalks / eps / maxsteps");
            return WOST_ERR_INVALID_ARG;
        }
        if (J.npoints > 0 && (!J.points || !J.out_mean)) { set_error(at + "null points or out_mean"); return WOST_ERR_INVALID_ARG; }
        if (guided) {
            if (!J.field) { set_error(at + "a guided batch needs a field per job"); return WOST_ERR_INVALID_ARG; }
            if (J.field->desc.dim != dim) { set_error(at + "field dimension differs from the scene"); return WOST_ERR_INVALID_ARG; }
            if (J.field->km != kMaxK) {
                set_error(at + "many-scene launches decode fields of at most 8 lobes");
                return WOST_ERR_UNSUPPORTED;
            }
            if (wost_status dc = check_device(J.field->device, "wost_batch_create (field)")) return dc;
            if (ex.train && !fields.insert(J.field).second) {
                set_error(at + "jobs that train need distinct fields");
                return WOST_ERR_INVALID_ARG;
            }
        }
    }
    return WOST_OK;
}

template <class T>
wost_status upload(DevBuf &buf, const std::vector<T> &v) {
    wost_status rc = buf.ensure(std::max<size_t>(v.size(), 1) * sizeof(T));
    if (rc != WOST_OK) return rc;
    if (!v.empty()) WOST_CUDA(cudaMemcpy(buf.ptr, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return WOST_OK;
}

wost_status build_plan(wost_batch *p) {
    const int nj = (int)p->jobs.size();
    const int D = p->dim;
    const wost_exec &ex = p->ex;
    // job table
    p->hjobs.assign(nj, DevJob{});
    int64_t off = 0;
    int max_steps = 1;
    for (int j = 0; j < nj; ++j) {
        const wost_job &J = p->jobs[j];
        DevJob &d = p->hjobs[j];
        d.sc = J.scene->dev;
        d.points = J.points;
        d.npoints = J.npoints;
        d.point_off = off;
        d.nwalks = J.nwalks;
        d.maxsteps = J.maxsteps;
        d.eps = (float)J.eps;
        d.eps64 = J.eps;
        d.key0 = (uint32_t)J.seed;
        d.key1 = (uint32_t)(J.seed >> 32) + J.scene->scene_id;
        d.rr_depth = p->ex.rr_depth;
        d.rr_q = p->ex.rr_survival;
        d.out_mean = J.out_mean;
        d.out_var = J.out_var;
        if (p->guided) d.f = J.field->dev();
        off += J.npoints;
        max_steps = std::max(max_steps, J.maxsteps);
    }
    p->total_points = off;
    // launches and their segments (job-major)
    std::vector<DevSeg> segs;
    auto add_launch = [&](bool record, auto walks_of) {
        wost_batch::Launch L;
        L.seg0 = (int)segs.size();
        L.record = record;
        for (int j = 0; j < nj; ++j) {
            int w0 = 0, nw = 0;
            walks_of(j, w0, nw);
            if (nw <= 0 || p->jobs[j].npoints == 0) continue;
            segs.push_back(DevSeg{L.total, j, w0});
            L.total += (unsigned long long)p->jobs[j].npoints * nw;
            if (record) L.train_jobs.push_back(j);
        }
        L.nseg = (int)segs.size() - L.seg0;
        return L;
    };
    int rounds = 0;
    if (p->guided && ex.train) {
        int maxw = 0;
        for (auto &J : p->jobs) maxw = std::max(maxw, J.nwalks);
        rounds = std::min(maxw, std::max(ex.train_until_wpp, 0));
    }
    for (int r = 0; r < rounds; ++r) {
        auto L = add_launch(true, [&](int j, int &w0, int &nw) { w0 = r; nw = p->jobs[j].nwalks > r ? 1 : 0; });
        if (L.total) p->launches.push_back(L);
    }
    {
        auto L = add_launch(false, [&](int j, int &w0, int &nw) {
            w0 = std::min(p->jobs[j].nwalks, rounds);
            nw = p->jobs[j].nwalks - w0;
        });
        if (L.total) p->launches.push_back(L);
    }
    p->calib = add_launch(false, [&](int, int &w0, int &nw) { w0 = 0; nw = 1; });
    p->record = false;
    for (auto &L : p->launches) p->record |= L.record;
    // device buffers
    wost_status rc;
    if ((rc = upload(p->djobs, p->hjobs)) != WOST_OK) return rc;
    if ((rc = upload(p->dsegs, segs)) != WOST_OK) return rc;
    const size_t np = (size_t)std::max<int64_t>(p->total_points, 1);
    if ((rc = p->status.ensure(np)) != WOST_OK) return rc;
    if ((rc = p->shell.ensure(np * sizeof(double))) != WOST_OK) return rc;
    if ((rc = p->sums.ensure(2 * np * sizeof(double))) != WOST_OK) return rc;
    if ((rc = p->ctr.ensure((kCtrWork + p->launches.size() + 1) * sizeof(unsigned long long))) != WOST_OK) return rc;
    if (p->record) {
        p->scratch_steps = max_steps;
        // walker lanes of the widest launch a plan may choose
        const int wmax = ex.walker_warps > 0 ? ex.walker_warps : kWsWalkersWide;
        size_t sb = (size_t)num_sms() * wmax * 32 * (size_t)max_steps * kRecFloats * sizeof(float);
        if ((rc = p->scratch.ensure(sb)) != WOST_OK) return rc;
        for (int j = 0; j < nj; ++j) {
            wost_field *f = p->jobs[j].field;
            int64_t cap = ex.max_train_records > 0 ? ex.max_train_records
                                                   : std::max<int64_t>(p->jobs[j].npoints * 64, 1 << 16);
            if ((rc = ensure_records(f, cap, 0)) != WOST_OK) return rc;
            f->t_c_mode = ex.c_mode;
            f->t_c_fixed = ex.c_fixed;
            f->t_reflect = ex.reflect;
            f->t_samples = ex.train_samples;
            p->hjobs[j].rd = RecDest{f->rec, f->rec_ctr, f->rec_cap};
        }
        if ((rc = upload(p->djobs, p->hjobs)) != WOST_OK) return rc;
        if ((rc = train_prepare(D)) != WOST_OK) return rc;
    }
    for (auto &L : p->launches) p->info.train_steps += (int)L.train_jobs.size();
    p->info.walk_launches = (int)p->launches.size();
    if (p->guided) {
        const cudaFuncAttribute at = cudaFuncAttributeMaxDynamicSharedMemorySize;
        if (D == 2) {
            WOST_CUDA(cudaFuncSetAttribute(batch_guided_kernel<2, kWsWalkerWarps>, at, kBatchGuidedSmem));
            WOST_CUDA(cudaFuncSetAttribute(batch_guided_kernel<2, kWsWalkersWide>, at, kBatchGuidedSmem));
        } else {
            WOST_CUDA(cudaFuncSetAttribute(batch_guided_kernel<3, kWsWalkerWarps>, at, kBatchGuidedSmem));
            WOST_CUDA(cudaFuncSetAttribute(batch_guided_kernel<3, kWsWalkersWide>, at, kBatchGuidedSmem));
        }
    }
    device_err_flag();   // created outside the capture
    WOST_CUDA(cudaStreamCreateWithFlags(&p->cap, cudaStreamNonBlocking));
    WOST_CUDA(cudaEventCreate(&p->ev0));
    WOST_CUDA(cudaEventCreate(&p->ev1));
    if ((rc = p->autotune()) != WOST_OK) return rc;
    p->info.ctas_per_sm = p->guided ? 1 : p->cps;
    p->info.flush_polls = (int)p->polls;
    p->info.walker_warps = p->guided ? p->walkers : 0;
    if (p->total_points == 0) return WOST_OK;
    // capture
    WOST_CUDA(cudaStreamSynchronize(p->cap));
    WOST_CUDA(cudaStreamBeginCapture(p->cap, cudaStreamCaptureModeThreadLocal));
    wost_status erc = p->enqueue(p->cap);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(p->cap, &g);
    if (erc != WOST_OK) {
        if (g) cudaGraphDestroy(g);
        return erc;
    }
    if (ce != cudaSuccess) return cuda_status(ce, "wost_batch_create: stream capture");
    p->graph = g;
    WOST_CUDA(cudaGraphInstantiate(&p->gexec, p->graph, 0));
    size_t nodes = 0;
    WOST_CUDA(cudaGraphGetNodes(p->graph, nullptr, &nodes));
    p->info.graph_nodes = (int64_t)nodes;
    return WOST_OK;
}

}  // namespace

extern "C" wost_status wost_batch_create(int32_t njobs, const wost_job *jobs, int32_t guided, const wost_exec *exec,
                                         wost_batch **out) {
    if (!out) { set_error("wost_batch_create: null out"); return WOST_ERR_INVALID_ARG; }
    *out = nullptr;
    wost_exec ex;
    if (exec) ex = *exec; else wost_exec_defaults(&ex);
    wost_status rc = validate(njobs, jobs, guided, ex);
    if (rc != WOST_OK) return rc;
    wost_batch *p = new wost_batch();
    p->dim = jobs[0].scene->dim;
    p->device = jobs[0].scene->device;
    p->guided = guided != 0;
    p->ex = ex;
    p->jobs.assign(jobs, jobs + njobs);
    rc = build_plan(p);
    if (rc != WOST_OK) { delete p; return rc; }
    *out = p;
    return WOST_OK;
}

extern "C" wost_status wost_batch_run(wost_batch *p, void *stream, wost_stats *stats) {
    if (!p) { set_error("wost_batch_run: null batch"); return WOST_ERR_INVALID_ARG; }
    if (stats) std::memset(stats, 0, sizeof(*stats));
    if (wost_status dc = check_device(p->device, "wost_batch_run")) return dc;
    if (!p->gexec) return WOST_OK;   // no points
    cudaStream_t st = (cudaStream_t)stream;
    WOST_CUDA(cudaEventRecord(p->ev0, st));
    WOST_CUDA(cudaGraphLaunch(p->gexec, st));
    WOST_CUDA(cudaEventRecord(p->ev1, st));
    unsigned long long hs[kCtrRec + 2 - kCtrStat];
    WOST_CUDA(cudaMemcpyAsync(hs, p->ctr_at(kCtrStat), sizeof(hs), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaStreamSynchronize(st));
    wost_status rc = device_check(st);
    if (rc != WOST_OK) return rc;
    if (stats) {
        float ms = 0;
        cudaEventElapsedTime(&ms, p->ev0, p->ev1);
        stats->walk_steps = (int64_t)hs[0];
        stats->truncated = (int64_t)hs[1];
        stats->walks = (int64_t)hs[2];
        stats->node_visits = (int64_t)hs[3];
        stats->prim_visits = (int64_t)(hs[4] + hs[5] + hs[6]);
        stats->dir_prim_visits = (int64_t)hs[4];
        stats->sil_prim_visits = (int64_t)hs[5];
        stats->neu_prim_visits = (int64_t)hs[6];
        stats->records = (int64_t)hs[kCtrRec - kCtrStat];
        stats->records_dropped = (int64_t)hs[kCtrRec + 1 - kCtrStat];
        stats->train_steps = p->info.train_steps;
        stats->ms_walk = ms;
        stats->ms_train = 0;
        stats->walk_launches = p->info.walk_launches;
        stats->kernel_launches = p->info.graph_nodes;
        stats->alg_bytes = walk_alg_bytes(p->dim, p->guided, hs, stats->records);
    }
    return WOST_OK;
}

extern "C" wost_status wost_batch_info_get(const wost_batch *p, wost_batch_info *info) {
    if (!p || !info) { set_error("wost_batch_info_get: null argument"); return WOST_ERR_INVALID_ARG; }
    *info = p->info;
    return WOST_OK;
}

extern "C" wost_status wost_batch_destroy(wost_batch *p) {
    delete p;
    return WOST_OK;
}

extern "C" wost_status wost_solve_batch(int32_t njobs, const wost_job *jobs, int32_t guided, const wost_exec *exec,
                                        wost_stats *stats) {
    wost_batch *p = nullptr;
    wost_status rc = wost_batch_create(njobs, jobs, guided, exec, &p);
    if (rc != WOST_OK) return rc;
    rc = wost_batch_run(p, exec ? exec->stream : nullptr, stats);
    wost_batch_destroy(p);
    return rc;
}
