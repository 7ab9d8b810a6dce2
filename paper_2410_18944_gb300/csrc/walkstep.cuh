// One walk-on-stars step, shared by the plain and the guided persistent
// kernels (Sec. 3.2 Eq. wost_estm, reparameterised as in Sec. 4.1):
//   1. closest Dirichlet point; stop inside the epsilon-shell (FP64 re-test)
//      or at the step cap, adding T g(xbar) to the point's FP64 sums;
//   2. star radius r = max(min(R_D, R_S), eps) from the closest silhouette;
//   0. Russian roulette from step rr_depth on (after the epsilon-shell test):
//      go on with probability q (throughput / q), else end with value 0;
//   3. source term -(r^2 / 2d) f(y), y ~ Green-function density, if visible,
//      and the Neumann term -<N> when the flux is nonzero;
//   4. (caller) direction nu and step weight;
//   5. first Neumann hit within r (FP64 re-test of the winner) or x + r nu.
// Random numbers: Philox4x32-10, counter (point, walk, step, purpose).
#pragma once
#include "geom.cuh"

namespace wost {

// width of the band (relative to the scene scale) inside which an FP32
// distance or hit parameter may be on the wrong side of its threshold:
// 16 units of 2^-24
constexpr float kRoundBand = 16.f * 5.9604645e-8f;

struct WalkArgs {
    DevScene sc;
    const double *points;      // npoints * D
    const uint8_t *status;     // 0 walk, 1 shell, 2 outside
    int64_t npoints;
    int walk_begin;
    unsigned long long total;  // work items = npoints * walks in this launch
    unsigned long long *work_ctr;
    double *sum, *sum2;
    float eps;
    double eps64;
    int maxsteps;
    uint32_t key0, key1;
    unsigned long long *stat;  // [0] walk-steps, [1] truncated, [2] walks, [3..6] node/Dirichlet/silhouette/Neumann visits
    int *err;
    int rr_depth;              // Russian roulette from this step on (0 = off)
    float rr_q;                // survival probability of a roulette step
    // single-scene guided launches only (nullptr elsewhere): the order in
    // which a launch hands out the points of each walk index (a
    // permutation of [0, npoints)), and per point the walk-steps its walks
    // take in this launch
    const uint32_t *order;
    unsigned *plen;
};

// what one step needs besides the walk state: the walk's scene and the
// solve's scalars (scene and keys differ per job in a multi-scene batch)
struct StepEnv {
    const DevScene &sc;
    float eps;
    double eps64;
    int maxsteps;
    uint32_t key0, key1;
    int *err;
    int rr_depth;
    float rr_q;
};

__device__ __forceinline__ StepEnv env_of(const WalkArgs &a) {
    return StepEnv{a.sc, a.eps, a.eps64, a.maxsteps, a.key0, a.key1, a.err, a.rr_depth, a.rr_q};
}

// Russian roulette (Sec. 6.1 enables it beyond 128 steps; the survival rule
// is a reading: a fixed probability q).  A step k >= rr_depth that survives
// divides the throughput by q, and for the suffix pass its weight and
// non-recursive terms carry the same 1 / q: roulette_scale(k).
__device__ __forceinline__ bool roulette_on(const StepEnv &a, int k) { return a.rr_depth > 0 && k >= a.rr_depth; }
__device__ __forceinline__ float roulette_scale(const StepEnv &a, int k) {
    return roulette_on(a, k) ? 1.f / a.rr_q : 1.f;
}
// the step's roulette draw (counter purpose P_RR): true if the walk goes on
__device__ __forceinline__ bool roulette_survives(const StepEnv &a, uint32_t pid, uint32_t wid, int k) {
    U4 u = philox(pid, wid, (uint32_t)k, P_RR, a.key0, a.key1);
    return u01(u.x) < a.rr_q;
}

template <int D>
struct Walk {
    float x[D], n[D];
    float T, acc;
    uint32_t pid, wid;
    int k, prim;     // prim: Neumann leaf slot the walker stands on, -1 if interior
    int job;         // job of a multi-scene batch (unused by single solves)
};

template <int D>
__device__ __forceinline__ void uniform_dir(float u0, float u1, float *v) {
    if (D == 2) {
        float s, c;
        sincospif(2.f * u0, &s, &c);
        v[0] = c;
        v[1] = s;
    } else {
        float z = 1.f - 2.f * u0, s, c;
        float st = sqrtf(fmaxf(0.f, 1.f - z * z));
        sincospif(2.f * u1, &s, &c);
        v[0] = st * c;
        v[1] = st * s;
        v[2] = z;
    }
}

template <int D>
__device__ __forceinline__ float dotv(const float *a, const float *b) {
    float s = a[0] * b[0] + a[1] * b[1];
    if (D == 3) s += a[2] * b[2];
    return s;
}

template <int D>
__device__ __forceinline__ void reflect(float *v, const float *n) {
    float t = 2.f * dotv<D>(v, n);
#pragma unroll
    for (int i = 0; i < D; ++i) v[i] -= t * n[i];
}

// Beta(2,2) by inversion of F(s) = 3 s^2 - 2 s^3 (trigonometric root)
__device__ __forceinline__ float beta22_inv(float u) {
    return 0.5f + cosf((acosf(1.f - 2.f * u) + 4.f * WOST_PI) / 3.f);
}

template <int D>
__device__ __forceinline__ void start_walk(Walk<D> &w, const WalkArgs &a, unsigned long long item) {
    w.pid = (uint32_t)(item % (unsigned long long)a.npoints);
    w.wid = (uint32_t)(a.walk_begin + item / (unsigned long long)a.npoints);
#pragma unroll
    for (int i = 0; i < D; ++i) { w.x[i] = (float)a.points[(size_t)w.pid * D + i]; w.n[i] = 0.f; }
    w.T = 1.f;
    w.acc = 0.f;
    w.k = 0;
    w.prim = -1;
}

__device__ __forceinline__ void finish_walk(const WalkArgs &a, uint32_t pid, float value) {
    atomicAdd(a.sum + pid, (double)value);
    atomicAdd(a.sum2 + pid, (double)value * (double)value);
}

// Neumann contribution <N> of a step (Sec. 3.2, Eq. wost_estm), entering the
// estimate with a minus sign: z on the Neumann boundary inside B(x, r) with
// density 1 / W (neumann_pick, then uniform on the chosen primitive), counted
// when it faces x (inside B there is no silhouette, so every Neumann point
// there that faces x is on the star's boundary).
//   <N> = G(x, z) h(z) W / alpha,  G = ln(r / |z - x|) / 2 pi  (2D),
//                                      (1 / |z - x| - 1 / r) / 4 pi  (3D),
// h the flux along the normal into the domain, alpha = 1/2 on a Neumann point.
template <int D>
__device__ __forceinline__ float neumann_term(const Walk<D> &w, const DevScene &sc, float r, uint32_t k0,
                                              uint32_t k1, int *err, Visits *vis) {
    float W;
    const int js = neumann_pick<D>(sc.neu, w.x, r, w.pid, w.wid, (uint32_t)w.k, k0, k1, W, err, vis);
    if (js < 0) return 0.f;
    U4 u = philox(w.pid, w.wid, (uint32_t)w.k, P_NEU, k0, k1);
    const float u0 = u01(u.x), u1 = u01(u.y);
    float z[3];
    if (D == 2) {
        const float4 p = ldn(sc.neu.prims + js);
        z[0] = (1.f - u0) * p.x + u0 * p.z;
        z[1] = (1.f - u0) * p.y + u0 * p.w;
    } else {
        float a[3], b[3], c[3];
        load_tri(sc.neu.prims, js, a, b, c);
        const float su = sqrtf(u0);
#pragma unroll
        for (int i = 0; i < 3; ++i) z[i] = (1.f - su) * a[i] + su * (1.f - u1) * b[i] + su * u1 * c[i];
    }
    float dz[D], dd2 = 0.f, facing = 0.f;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        dz[i] = z[i] - w.x[i];
        dd2 += dz[i] * dz[i];
        facing += dz[i] * __ldg(sc.nin_neu + (size_t)js * D + i);   // normals by leaf slot
    }
    const float dd = sqrtf(dd2);
    if (!(dd > 0.f) || !(dd < r) || !(facing < 0.f)) return 0.f;
    const float G = D == 2 ? logf(r / dd) * (0.5f / WOST_PI) : (1.f / dd - 1.f / r) * (0.25f / WOST_PI);
    return G * eval_fn<D>(sc.h, z) * W * (w.prim >= 0 ? 2.f : 1.f);
}

// Steps 1-3.  Returns true if the walk ended (its value already added;
// term_value 0 after a lost roulette draw).  On return false: r (star
// radius) and S (this step's source and Neumann terms, times the step's
// roulette scale, as the suffix pass of a recorded walk takes them).
template <int D>
__device__ __forceinline__ bool step_geometry(Walk<D> &w, const StepEnv &a, float &r, float &S,
                                              float &term_value, bool &truncated, Visits *vis) {
    const DevScene &sc = a.sc;
    float bd2;
    int slot = closest_dirichlet<D>(sc.dir, w.x, bd2, a.err, vis);
    float RD = sqrtf(bd2);
    // eps-shell decision: in FP64 when the FP32 distance lies within its
    // rounding band around eps (elsewhere both precisions agree)
    double q64[3];
    bool have64 = false, shell;
    if (fabsf(RD - a.eps) <= kRoundBand * (sc.scale + RD)) {
        shell = dirichlet_dist64<D>(sc.dir, slot, w.x, q64) <= a.eps64;
        have64 = true;
    } else {
        shell = RD <= a.eps;
    }
    if (shell || w.k >= a.maxsteps) {
        if (!have64) dirichlet_dist64<D>(sc.dir, slot, w.x, q64);
        float xb[3] = {(float)q64[0], (float)q64[1], D == 3 ? (float)q64[2] : 0.f};
        term_value = eval_fn<D>(sc.g, xb);
        w.acc += w.T * term_value;
        truncated = !shell;
        return true;
    }
    if (roulette_on(a, w.k)) {
        if (!roulette_survives(a, w.pid, w.wid, w.k)) {
            term_value = 0.f;
            truncated = false;
            return true;
        }
        w.T *= 1.f / a.rr_q;
    }
    float bs = RD * RD;
    closest_silhouette<D>(sc.sil, w.x, sc.tau, bs, a.err, vis, sc.sil_cones);
    float R = fminf(sqrtf(bs), RD);
    r = fmaxf(R, a.eps);
    S = 0.f;
    if (sc.has_source) {
        U4 u = philox(w.pid, w.wid, (uint32_t)w.k, P_SRC, a.key0, a.key1);
        float vs[D];
        uniform_dir<D>(u01(u.x), u01(u.y), vs);
        if (w.prim >= 0 && dotv<D>(vs, w.n) < 0.f) reflect<D>(vs, w.n);
        float rho = D == 2 ? r * sqrtf(u01(u.z) * u01(u.w)) : r * beta22_inv(u01(u.z));
        float th;
        const float tneg = kRoundBand * sc.scale;
        int hs = ray_neumann<D, true>(sc.neu, w.x, vs, rho, w.prim, th, a.err, vis, tneg);
        if (hs >= 0 && rho - th <= kRoundBand * (sc.scale + rho)) {
            double t64;
            if (!ray_prim64<D, true>(sc.neu, hs, w.x, vs, t64, tneg) || t64 > (double)rho) hs = -1;
        }
        if (hs < 0) {
            float y[3];
#pragma unroll
            for (int i = 0; i < D; ++i) y[i] = w.x[i] + rho * vs[i];
            S = -(r * r / (2.f * D)) * eval_fn<D>(sc.f, y);
        }
        if (!sc.has_flux) w.acc += w.T * S;
    }
    if (sc.has_flux) {
        S -= neumann_term<D>(w, sc, r, a.key0, a.key1, a.err, vis);
        w.acc += w.T * S;
    }
    S *= roulette_scale(a, w.k);
    return false;
}

// Step 5: ray cast within r and move.
template <int D>
__device__ __forceinline__ void step_move(Walk<D> &w, const StepEnv &a, const float *nu, float r, Visits *vis) {
    const DevScene &sc = a.sc;
    float th;
    // the first exit through the Neumann boundary (ray_prim, kExit), from
    // t > -(rounding band of a position)
    const float tneg = kRoundBand * sc.scale;
    int hit = ray_neumann<D, true>(sc.neu, w.x, nu, r, w.prim, th, a.err, vis, tneg);
    // hit-or-reach-r decision: in FP64 when the FP32 hit lies within its
    // rounding band below r
    if (hit >= 0 && r - th <= kRoundBand * (sc.scale + r)) {
        double t64;
        if (!ray_prim64<D, true>(sc.neu, hit, w.x, nu, t64, tneg) || t64 > (double)r) hit = -1;
    }
    if (hit >= 0) {
        // an exit hit arrives from the inside, the side the walk is on, so
        // the walker's normal is the primitive's inward normal (Sec. 4.1,
        // normal convention at Eq. angular_req).  The walker stands at the
        // hit point moved tneg along that normal: a rounded hit point may lie
        // on either side of the boundary, and every later query (silhouettes,
        // exit casts near a vertex) needs a start point inside the domain.
        th = fmaxf(th, 0.f);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            w.n[i] = __ldg(sc.nin_neu + (size_t)hit * D + i);
            w.x[i] += th * nu[i] + tneg * w.n[i];
        }
        w.prim = hit;
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) w.x[i] += r * nu[i];
        w.prim = -1;
    }
    w.k++;
}

// Status of a query point: 2 outside (odd/even crossing count of a fixed
// ray against all primitives), 1 inside the epsilon-shell (val = g at the
// closest Dirichlet point, FP64 distance test), 0 to be walked.
template <int D>
__device__ __forceinline__ uint8_t classify_point(const DevScene &sc, double eps64, const double *p, int *err,
                                                  double &val) {
    float x[D];
    for (int k = 0; k < D; ++k) x[k] = (float)p[k];
    const float dir[3] = {0.5377844f, 0.7924136f, 0.2876523f};
    float v[D], nn = 0.f;
    for (int k = 0; k < D; ++k) { v[k] = dir[k]; nn += v[k] * v[k]; }
    for (int k = 0; k < D; ++k) v[k] *= rsqrtf(nn);
    int c = ray_count<D>(sc.dir, x, v, err) + ray_count<D>(sc.neu, x, v, err);
    val = 0.0;
    if ((c & 1) == 0) {
        val = __longlong_as_double(0x7ff8000000000000LL);
        return 2;
    }
    float bd2;
    int slot = closest_dirichlet<D>(sc.dir, x, bd2, err);
    double q[3];
    if (dirichlet_dist64<D>(sc.dir, slot, x, q) <= eps64) {
        float xb[3] = {(float)q[0], (float)q[1], D == 3 ? (float)q[2] : 0.f};
        val = eval_fn<D>(sc.g, xb);
        return 1;
    }
    return 0;
}

// mean and variance of the mean of one point from its FP64 sums (Sec. 3.2);
// shell / outside points take their classification value
__device__ __forceinline__ void finalize_point(uint8_t status, double shell, double sum, double sum2, int nw,
                                               double *mean, double *var) {
    if (status != 0) {
        *mean = shell;
        if (var) *var = status == 1 ? 0.0 : shell;
        return;
    }
    double m = sum / nw;
    *mean = m;
    if (var) {
        double v = nw > 1 ? (sum2 - nw * m * m) / ((double)nw * (nw - 1)) : 0.0;
        *var = v > 0 ? v : 0.0;
    }
}

// block-level sum of the per-thread counters into the launch statistics
// stat[0..6]: walk-steps, truncated, walks, node / Dirichlet / silhouette /
// Neumann visits
__device__ __forceinline__ void flush_stats(unsigned long long *stat, unsigned long long steps,
                                            unsigned long long trunc, unsigned long long walks, const Visits &v) {
    __shared__ unsigned long long red[7];
    if (threadIdx.x < 7) red[threadIdx.x] = 0;
    __syncthreads();
    atomicAdd(&red[0], steps);
    atomicAdd(&red[1], trunc);
    atomicAdd(&red[2], walks);
    atomicAdd(&red[3], (unsigned long long)v.nodes);
    atomicAdd(&red[4], (unsigned long long)v.dprims);
    atomicAdd(&red[5], (unsigned long long)v.sprims);
    atomicAdd(&red[6], (unsigned long long)v.nprims);
    __syncthreads();
    if (threadIdx.x < 7 && red[threadIdx.x]) atomicAdd(stat + threadIdx.x, red[threadIdx.x]);
}

}  // namespace wost
