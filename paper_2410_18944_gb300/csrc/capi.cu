// C ABI glue: errors, defaults, field lifetime and parameters, training-step
// entry points.
#include <cmath>
#include <cstring>
#include <random>
#include <string>

#include "field.cuh"
#include "internal.h"

namespace wost {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

wost_status cuda_status(cudaError_t e, const char *what) {
    g_last_error = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return e == cudaErrorMemoryAllocation ? WOST_ERR_OOM : WOST_ERR_CUDA;
}

wost_status check_device(int device, const char *who) {
    int cur = -1;
    cudaError_t e = cudaGetDevice(&cur);
    if (e != cudaSuccess) return cuda_status(e, who);
    if (cur != device) {
        g_last_error = std::string(who) + ": the handle belongs to CUDA device " + std::to_string(device) +
                       " but device " + std::to_string(cur) + " is current; make its device current first";
        return WOST_ERR_INVALID_ARG;
    }
    return WOST_OK;
}

wost_status refresh_inference_copy(wost_field *f, cudaStream_t st);
wost_status train_launch(wost_field *f, int dim, cudaStream_t st, bool apply_adam, float *loss_out_dev,
                         long long off = -1);
wost_status train_loss_launch(wost_field *f, int dim, cudaStream_t st, float *out_dev);
int *device_err_flag();
wost_status device_check(cudaStream_t st);

wost_status ensure_records(wost_field *f, int64_t cap, size_t scratch_bytes) {
    if (!f->rec_ctr) {
        WOST_CUDA(cudaMalloc(&f->rec_ctr, 4 * sizeof(unsigned long long)));
        WOST_CUDA(cudaMemset(f->rec_ctr, 0, 4 * sizeof(unsigned long long)));
    }
    if (cap > f->rec_cap) {
        if (f->rec) cudaFree(f->rec);
        f->rec = nullptr;
        f->rec_cap = 0;
        WOST_CUDA(cudaMalloc(&f->rec, (size_t)cap * 12 * sizeof(float)));
        f->rec_cap = cap;
    }
    if (scratch_bytes > f->scratch_bytes) {
        if (f->scratch) cudaFree(f->scratch);
        f->scratch = nullptr;
        f->scratch_bytes = 0;
        WOST_CUDA(cudaMalloc(&f->scratch, scratch_bytes));
        f->scratch_bytes = scratch_bytes;
    }
    return WOST_OK;
}

}  // namespace wost

using namespace wost;

wost::DevField wost_field::dev() const {
    DevField d{};
    d.dim = desc.dim;
    d.K = desc.K;
    d.L = desc.levels;
    d.log2T = desc.log2_table;
    d.nout = nout;
    d.dense_mask = dense_mask;
    for (int l = 0; l < 16; ++l) {
        d.res[l] = res[l];
        d.level_off[l] = (uint32_t)level_off[std::min(l, desc.levels)];
    }
    for (int k = 0; k < 3; ++k) {
        d.lo[k] = (float)desc.lo[k];
        double e = desc.hi[k] - desc.lo[k];
        d.inv_ext[k] = e > 0 ? (float)(1.0 / e) : 0.f;
    }
    d.grid16 = grid16;
    d.wimg = reinterpret_cast<const uint4 *>(wimg);
    d.b3 = b3pad;
    return d;
}

wost_field::~wost_field() {
    void *ps[] = {grid32, grid_m, grid_v, grid_g, grid16, mlp32, mlp_m, mlp_v, mlp_g, wimg, b3pad, rec, rec_ctr, scratch, loss_acc};
    for (void *p : ps)
        if (p) cudaFree(p);
}

extern "C" const char *wost_last_error(void) { return g_last_error.c_str(); }

extern "C" void wost_exec_defaults(wost_exec *e) {
    if (!e) return;
    std::memset(e, 0, sizeof(*e));
    e->seed = 1;
    e->reflect = 1;
    e->c_fixed = 0.5f;
    e->train_until_wpp = 256;
    e->rr_survival = 0.995f;
}

extern "C" void wost_field_desc_defaults(wost_field_desc *d, int32_t dim) {
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->dim = dim;
    d->K = 8;
    d->levels = 16;
    d->log2_table = dim == 3 ? 19 : 16;
    d->features = 2;
    d->hidden = 64;
    d->base_res = 16;
    d->max_res = dim == 3 ? 512 : 2048;
    for (int k = 0; k < 3; ++k) { d->lo[k] = -1.0; d->hi[k] = 1.0; }
    d->seed = 1;
    d->lr_grid = 1e-2f;
    d->lr_mlp = 1e-3f;
    d->beta1 = 0.9f;
    d->beta2 = 0.99f;
    d->adam_eps = 1e-8f;
    d->e_sel = 0.2f;
}

namespace {

wost_status alloc(void **p, size_t bytes) {
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) return cuda_status(e, "field allocation");
    return WOST_OK;
}

// Initial parameters (the paper's Appendix D is not available): grid
// U(-1e-4, 1e-4); He-uniform hidden layers; output layer U(+-0.1 sqrt(6/H));
// output bias spreading the K lobe directions evenly (circle / Fibonacci
// sphere), kappa' = 0 (kappa = 1), uniform lambda, c' = 0 (c = 0.5).
void init_params(const wost_field_desc &d, int nout, int64_t ngrid, std::vector<float> &grid, std::vector<float> &mlp) {
    std::mt19937_64 rng(d.seed);
    std::uniform_real_distribution<float> U(-1.f, 1.f);
    grid.resize(ngrid);
    for (auto &g : grid) g = 1e-4f * U(rng);
    const int H = d.hidden, nin = d.levels * d.features;
    mlp.assign((size_t)H * nin + (size_t)H * H + (size_t)nout * H + nout, 0.f);
    float *W1 = mlp.data(), *W2 = W1 + H * nin, *W3 = W2 + H * H, *b3 = W3 + nout * H;
    for (int i = 0; i < H * nin; ++i) W1[i] = std::sqrt(6.f / nin) * U(rng);
    for (int i = 0; i < H * H; ++i) W2[i] = std::sqrt(6.f / H) * U(rng);
    for (int i = 0; i < nout * H; ++i) W3[i] = 0.1f * std::sqrt(6.f / H) * U(rng);
    const int K = d.K, D = d.dim;
    for (int i = 0; i < K; ++i) {
        if (D == 2) {
            double th = 2 * M_PI * (i + 0.5) / K;
            b3[i * 2] = (float)std::cos(th);
            b3[i * 2 + 1] = (float)std::sin(th);
        } else {
            double z = 1 - (2.0 * i + 1) / K, r = std::sqrt(std::max(0.0, 1 - z * z));
            double ph = i * M_PI * (3 - std::sqrt(5.0));
            b3[i * 3] = (float)(r * std::cos(ph));
            b3[i * 3 + 1] = (float)(r * std::sin(ph));
            b3[i * 3 + 2] = (float)z;
        }
    }
}

}  // namespace

extern "C" wost_status wost_create_field(const wost_field_desc *desc, wost_field **out) {
    if (!desc || !out) { set_error("wost_create_field: null argument"); return WOST_ERR_INVALID_ARG; }
    *out = nullptr;
    const wost_field_desc &d = *desc;
    if ((d.dim != 2 && d.dim != 3) || d.K < 1 || d.K > kMaxKWide || d.levels != 16 || d.features != 2 || d.hidden != 64) {
        set_error("wost_create_field: this library supports dim 2/3, K = 1..16, L = 16, F = 2, H = 64");
        return WOST_ERR_UNSUPPORTED;
    }
    if (d.log2_table < 8 || d.log2_table > 24 || d.base_res < 2 || d.max_res < d.base_res ||
        (d.grid_type != 0 && d.grid_type != 1)) {
        set_error("wost_create_field: bad table size, resolutions or grid type");
        return WOST_ERR_INVALID_ARG;
    }
    for (int k = 0; k < d.dim; ++k)
        if (!(d.hi[k] > d.lo[k])) { set_error("wost_create_field: empty box"); return WOST_ERR_INVALID_ARG; }
    int dev = -1;
    WOST_CUDA(cudaGetDevice(&dev));
    auto *f = new wost_field();
    f->desc = d;
    f->device = dev;
    f->nout = (d.dim + 2) * d.K + 1;
    f->km = field_km(d.K);
    f->T = (int64_t)1 << d.log2_table;
    double b = d.levels > 1 ? std::exp((std::log((double)d.max_res) - std::log((double)d.base_res)) / (d.levels - 1)) : 1.0;
    // level l's entries start at level_off[l]: l 2^log2T in the hash grid;
    // in the dense grid every level is dense with its own (N_l + 1)^d
    // vertices, the levels one after the other
    for (int l = 0; l < d.levels; ++l) {
        f->res[l] = (int)std::floor(d.base_res * std::pow(b, l) + 1e-6);
        double side = f->res[l] + 1.0;
        const double nv = std::pow(side, d.dim);
        if (d.grid_type == 1 || nv <= (double)f->T) f->dense_mask |= 1u << l;
        f->level_off[l + 1] = f->level_off[l] + (d.grid_type == 1 ? (int64_t)nv : f->T);
    }
    if (f->level_off[d.levels] >= ((int64_t)1 << 31)) {
        delete f;
        set_error("wost_create_field: the dense grid needs more than 2^31 entries; lower max_res");
        return WOST_ERR_INVALID_ARG;
    }
    const int64_t ng = f->n_grid(), nm = f->n_mlp();
    wost_status rc = WOST_OK;
    void **bufs[] = {(void **)&f->grid32, (void **)&f->grid_m, (void **)&f->grid_v, (void **)&f->grid_g};
    for (void **p : bufs) if (rc == WOST_OK) rc = alloc(p, ng * sizeof(float));
    void **mbufs[] = {(void **)&f->mlp32, (void **)&f->mlp_m, (void **)&f->mlp_v, (void **)&f->mlp_g};
    for (void **p : mbufs) if (rc == WOST_OK) rc = alloc(p, nm * sizeof(float));
    if (rc == WOST_OK) rc = alloc((void **)&f->grid16, (ng / 2) * sizeof(__half2));
    if (rc == WOST_OK) rc = alloc((void **)&f->wimg, wimg_bytes(f->km));
    if (rc == WOST_OK) rc = alloc((void **)&f->b3pad, out_pad(f->km) * sizeof(float));
    if (rc == WOST_OK) rc = alloc((void **)&f->loss_acc, 3 * sizeof(double));
    if (rc != WOST_OK) { delete f; return rc; }
    std::vector<float> grid, mlp;
    init_params(d, f->nout, ng, grid, mlp);
    cudaError_t e = cudaMemcpy(f->grid32, grid.data(), ng * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(f->mlp32, mlp.data(), nm * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(f->grid_m, 0, ng * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(f->grid_v, 0, ng * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(f->mlp_m, 0, nm * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(f->mlp_v, 0, nm * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(f->wimg, 0, wimg_bytes(f->km));
    if (e == cudaSuccess) e = cudaMemset(f->loss_acc, 0, 3 * sizeof(double));
    if (e != cudaSuccess) { delete f; return cuda_status(e, "wost_create_field"); }
    if ((rc = refresh_inference_copy(f, 0)) != WOST_OK) { delete f; return rc; }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) { delete f; return cuda_status(e, "wost_create_field"); }
    *out = f;
    return WOST_OK;
}

extern "C" wost_status wost_field_grid_entries(const wost_field *f, int64_t *entries) {
    if (!f || !entries) { set_error("wost_field_grid_entries: null argument"); return WOST_ERR_INVALID_ARG; }
    *entries = f->level_off[f->desc.levels];
    return WOST_OK;
}

extern "C" wost_status wost_destroy_field(wost_field *f) {
    delete f;
    return WOST_OK;
}

extern "C" wost_status wost_field_set_params(wost_field *f, const float *grid, const float *W1, const float *W2,
                                             const float *W3, const float *b3) {
    if (!f || !grid || !W1 || !W2 || !W3 || !b3) { set_error("wost_field_set_params: null argument"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(f->device, "wost_field_set_params")) return dc;
    const int H = f->desc.hidden, nin = f->desc.levels * f->desc.features;
    float *d = f->mlp32;
    WOST_CUDA(cudaMemcpy(f->grid32, grid, f->n_grid() * sizeof(float), cudaMemcpyDefault));
    WOST_CUDA(cudaMemcpy(d, W1, (size_t)H * nin * sizeof(float), cudaMemcpyDefault));
    WOST_CUDA(cudaMemcpy(d + H * nin, W2, (size_t)H * H * sizeof(float), cudaMemcpyDefault));
    WOST_CUDA(cudaMemcpy(d + H * nin + H * H, W3, (size_t)f->nout * H * sizeof(float), cudaMemcpyDefault));
    WOST_CUDA(cudaMemcpy(d + H * nin + H * H + f->nout * H, b3, f->nout * sizeof(float), cudaMemcpyDefault));
    WOST_CUDA(cudaMemset(f->grid_m, 0, f->n_grid() * sizeof(float)));
    WOST_CUDA(cudaMemset(f->grid_v, 0, f->n_grid() * sizeof(float)));
    WOST_CUDA(cudaMemset(f->mlp_m, 0, f->n_mlp() * sizeof(float)));
    WOST_CUDA(cudaMemset(f->mlp_v, 0, f->n_mlp() * sizeof(float)));
    WOST_CUDA(cudaMemset(f->adam_step(), 0, sizeof(unsigned long long)));
    wost_status rc = refresh_inference_copy(f, 0);
    if (rc != WOST_OK) return rc;
    WOST_CUDA(cudaDeviceSynchronize());
    return WOST_OK;
}

extern "C" wost_status wost_field_get_params(const wost_field *f, float *grid, float *W1, float *W2, float *W3,
                                             float *b3) {
    if (!f) { set_error("wost_field_get_params: null field"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(f->device, "wost_field_get_params")) return dc;
    const int H = f->desc.hidden, nin = f->desc.levels * f->desc.features;
    const float *d = f->mlp32;
    WOST_CUDA(cudaDeviceSynchronize());
    if (grid) WOST_CUDA(cudaMemcpy(grid, f->grid32, f->n_grid() * sizeof(float), cudaMemcpyDefault));
    if (W1) WOST_CUDA(cudaMemcpy(W1, d, (size_t)H * nin * sizeof(float), cudaMemcpyDefault));
    if (W2) WOST_CUDA(cudaMemcpy(W2, d + H * nin, (size_t)H * H * sizeof(float), cudaMemcpyDefault));
    if (W3) WOST_CUDA(cudaMemcpy(W3, d + H * nin + H * H, (size_t)f->nout * H * sizeof(float), cudaMemcpyDefault));
    if (b3) WOST_CUDA(cudaMemcpy(b3, d + H * nin + H * H + f->nout * H, f->nout * sizeof(float), cudaMemcpyDefault));
    return WOST_OK;
}

extern "C" wost_status wost_train_records(wost_field *f, const float *records, int64_t n, const wost_exec *exec) {
    if (!f || n < 0 || (n > 0 && !records)) { set_error("wost_train_records: invalid argument"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(f->device, "wost_train_records")) return dc;
    wost_exec ex;
    if (exec) ex = *exec; else wost_exec_defaults(&ex);
    wost_status rc = ensure_records(f, std::max<int64_t>(n, 1), 0);
    if (rc != WOST_OK) return rc;
    if (n > 0)
        WOST_CUDA(cudaMemcpy(f->rec, records, n * 12 * sizeof(float),
                             ex.points_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice));
    unsigned long long c[2] = {(unsigned long long)n, 0ull};
    WOST_CUDA(cudaMemcpy(f->rec_ctr, c, sizeof(c), cudaMemcpyHostToDevice));
    f->t_c_mode = ex.c_mode;
    f->t_c_fixed = ex.c_fixed;
    f->t_reflect = ex.reflect;
    f->t_samples = ex.train_samples;
    return WOST_OK;
}

extern "C" wost_status wost_get_records(const wost_field *f, float *records, int64_t cap, int64_t *n) {
    if (!f || !n || cap < 0 || (cap > 0 && !records)) { set_error("wost_get_records: invalid argument"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(f->device, "wost_get_records")) return dc;
    *n = 0;
    if (!f->rec_ctr) return WOST_OK;
    unsigned long long c[2];
    WOST_CUDA(cudaDeviceSynchronize());
    WOST_CUDA(cudaMemcpy(c, f->rec_ctr, sizeof(c), cudaMemcpyDeviceToHost));
    int64_t have = (int64_t)std::min<unsigned long long>(c[0], (unsigned long long)f->rec_cap);
    int64_t m = std::min(have, cap);
    if (m > 0) WOST_CUDA(cudaMemcpy(records, f->rec, m * 12 * sizeof(float), cudaMemcpyDeviceToHost));
    *n = have;
    return WOST_OK;
}

static wost_status read_loss(wost_field *f, cudaStream_t st, float *out_loss) {
    double acc[3] = {0, 0, 0};
    WOST_CUDA(cudaMemcpyAsync(acc, f->loss_acc, sizeof(acc), cudaMemcpyDeviceToHost, st));
    WOST_CUDA(cudaStreamSynchronize(st));
    unsigned long long n;
    std::memcpy(&n, &acc[2], sizeof(n));
    if (out_loss) *out_loss = n > 0 ? (float)(acc[0] / (double)n) : 0.f;
    return WOST_OK;
}

extern "C" wost_status wost_train_step(wost_scene *s, wost_field *f, const wost_exec *exec, float *out_loss) {
    if (!f) { set_error("wost_train_step: null field"); return WOST_ERR_INVALID_ARG; }
    if (s && s->dim != f->desc.dim) { set_error("wost_train_step: dimension mismatch"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(f->device, "wost_train_step")) return dc;
    if (!f->rec || !f->rec_ctr) { set_error("wost_train_step: no training records"); return WOST_ERR_INVALID_ARG; }
    cudaStream_t st = exec ? (cudaStream_t)exec->stream : 0;
    if (exec) f->t_samples = exec->train_samples;
    wost_status rc = train_launch(f, f->desc.dim, st, true, nullptr);
    if (rc != WOST_OK) return rc;
    if ((rc = read_loss(f, st, out_loss)) != WOST_OK) return rc;
    return device_check(st);
}

extern "C" wost_status wost_train_loss(wost_field *f, const wost_exec *exec, float *out_loss) {
    if (!f || !out_loss) { set_error("wost_train_loss: invalid argument"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(f->device, "wost_train_loss")) return dc;
    if (!f->rec || !f->rec_ctr) { set_error("wost_train_loss: no training records"); return WOST_ERR_INVALID_ARG; }
    wost_exec ex;
    if (exec) ex = *exec; else wost_exec_defaults(&ex);
    cudaStream_t st = (cudaStream_t)ex.stream;
    f->t_samples = ex.train_samples;
    if (ex.out_on_device) {
        // stays on the stream: no synchronisation
        return train_loss_launch(f, f->desc.dim, st, out_loss);
    }
    wost_status rc = train_loss_launch(f, f->desc.dim, st, nullptr);
    if (rc != WOST_OK) return rc;
    if ((rc = read_loss(f, st, out_loss)) != WOST_OK) return rc;
    return device_check(st);
}

extern "C" wost_status wost_train_grad(wost_field *f, const wost_exec *exec, float *out_loss, float *g_grid,
                                       float *g_W1, float *g_W2, float *g_W3, float *g_b3) {
    if (!f) { set_error("wost_train_grad: null field"); return WOST_ERR_INVALID_ARG; }
    if (wost_status dc = check_device(f->device, "wost_train_grad")) return dc;
    if (!f->rec || !f->rec_ctr) { set_error("wost_train_grad: no training records"); return WOST_ERR_INVALID_ARG; }
    cudaStream_t st = exec ? (cudaStream_t)exec->stream : 0;
    if (exec) f->t_samples = exec->train_samples;
    wost_status rc = train_launch(f, f->desc.dim, st, false, nullptr);
    if (rc != WOST_OK) return rc;
    if ((rc = read_loss(f, st, out_loss)) != WOST_OK) return rc;
    if ((rc = device_check(st)) != WOST_OK) return rc;
    const int H = f->desc.hidden, nin = f->desc.levels * f->desc.features;
    const float *d = f->mlp_g;
    if (g_grid) WOST_CUDA(cudaMemcpy(g_grid, f->grid_g, f->n_grid() * sizeof(float), cudaMemcpyDefault));
    if (g_W1) WOST_CUDA(cudaMemcpy(g_W1, d, (size_t)H * nin * sizeof(float), cudaMemcpyDefault));
    if (g_W2) WOST_CUDA(cudaMemcpy(g_W2, d + H * nin, (size_t)H * H * sizeof(float), cudaMemcpyDefault));
    if (g_W3) WOST_CUDA(cudaMemcpy(g_W3, d + H * nin + H * H, (size_t)f->nout * H * sizeof(float), cudaMemcpyDefault));
    if (g_b3) WOST_CUDA(cudaMemcpy(g_b3, d + H * nin + H * H + f->nout * H, f->nout * sizeof(float), cudaMemcpyDefault));
    return WOST_OK;
}
