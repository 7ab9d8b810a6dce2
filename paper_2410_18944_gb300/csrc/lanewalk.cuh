// Plain walk loop as a per-lane state machine over the three boundary
// queries of a walk-on-stars step (Sec. 3.2): closest Dirichlet point,
// closest silhouette, first Neumann exit along a ray (source visibility and
// the step itself).
//
// The query functions of geom.cuh run one query for the whole warp: the
// warp leaves a query only when its slowest lane has finished it, so on
// incoherent walks most lanes sit idle through the tail of every query.
// Here every lane carries its own query (kind, BVH cursor, stack, best
// result) through one loop:
//   logic phase  - lanes whose query finished take the step logic that
//                  follows it and set up their next query (or end the walk
//                  and fetch the next one);
//   node phase   - lanes at an inner node visit it, until every lane that
//                  is still searching holds a leaf (while-while);
//   leaf phase   - lanes at a leaf test its primitives.
// A lane that finishes its query early starts its next one at the next
// logic phase instead of waiting for the rest of the warp; over many walks
// per lane the lanes' total work evens out.  Results are those of the
// warp-synchronous queries: each query returns the minimum (distance or hit
// parameter, ties to the smaller primitive id), which does not depend on the
// order of visits.
#pragma once
#include "walkstep.cuh"

namespace wost {

enum : int { kQNone = 0, kQDir = 1, kQSil = 2, kQSrc = 3, kQMove = 4 };

template <int D>
struct LaneQuery {
    int q = kQNone;   // query kind
    bool fin = true;  // traversal finished: result in best / slot
    int ref = 0, sp = 0;
    float best = 0.f; // squared distance (Dirichlet, silhouette) or hit parameter (rays)
    int slot = -1, id = 0x7fffffff;
    float v[D], inv[D];
    int stack[kStack];
    float key[kStack];
};

template <int D>
__device__ __forceinline__ const DevBVH &query_bvh(const DevScene &sc, int q) {
    return q == kQDir ? sc.dir : (q == kQSil ? sc.sil : sc.neu);
}

// start a traversal of kind q from the root with initial bound best0
template <int D>
__device__ __forceinline__ void query_begin(LaneQuery<D> &Q, const DevScene &sc, int q, float best0) {
    Q.q = q;
    Q.ref = 0;
    Q.sp = 0;
    Q.best = best0;
    Q.slot = -1;
    Q.id = 0x7fffffff;
    Q.fin = query_bvh<D>(sc, q).nprims == 0;
}

template <int D>
__device__ __forceinline__ void query_ray(LaneQuery<D> &Q, const DevScene &sc, int q, const float *v, float tmax) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
        Q.v[k] = v[k];
        Q.inv[k] = 1.f / v[k];
    }
    query_begin<D>(Q, sc, q, tmax);
}

template <int D>
__device__ __forceinline__ void query_pop(LaneQuery<D> &Q) {
    while (Q.sp > 0) {
        --Q.sp;
        if (Q.key[Q.sp] <= Q.best) {
            Q.ref = Q.stack[Q.sp];
            return;
        }
    }
    Q.fin = true;
}

// one inner node: order and keep the children within the bound
template <int D>
__device__ __forceinline__ void query_node(LaneQuery<D> &Q, const DevScene &sc, const float *x, float tneg,
                                           int *err, Visits &vis) {
    constexpr int kBW = bvh_width(D);
    const DevBVH &bv = query_bvh<D>(sc, Q.q);
    float k[kBW];
    int r[kBW];
    bool h[kBW];
    if (Q.q == kQDir || Q.q == kQSil) node_keys_d2<D>(bv.nodes, Q.ref, x, k, r);
    else node_keys_ray<D>(bv.nodes, Q.ref, x, Q.inv, Q.best, k, r, tneg);
    vis.nodes++;
#pragma unroll
    for (int c = 0; c < kBW; ++c) {
        h[c] = r[c] != kEmptyRef && k[c] <= Q.best;
        if (Q.q == kQSil && sc.sil_cones && h[c]) {
            float lo[3], hi[3];
            node_child_box<D>(bv.nodes, Q.ref, c, lo, hi);
            if (cone_prunes<D>(ldn(sc.sil_cones + kBW * Q.ref + c), lo, hi, x, k[c], sc.tau)) h[c] = false;
        }
    }
    if (!take_children<kBW>(k, r, h, Q.ref, Q.stack, Q.key, Q.sp, err)) query_pop<D>(Q);
}

// one leaf: test its primitives, then continue from the stack
template <int D>
__device__ __forceinline__ void query_leaf(LaneQuery<D> &Q, const DevScene &sc, const float *x, int skip,
                                           float tneg, Visits &vis) {
    const int s0 = leaf_start(Q.ref), cnt = leaf_count(Q.ref);
    if (Q.q == kQDir) {
        const DevBVH &bv = sc.dir;
        vis.dprims += cnt;
        for (int s = s0; s < s0 + cnt; ++s) {
            float d2;
            if (D == 2) {
                float4 p = ldn(bv.prims + s);
                float qx, qy;
                d2 = seg_d2<float>(p.x, p.y, p.z, p.w, x[0], x[1], qx, qy);
            } else {
                float a[3], b[3], c[3], q[3];
                load_tri(bv.prims, s, a, b, c);
                d2 = tri_d2<float>(a, b, c, x, q);
            }
            if (d2 <= Q.best) {
                int id = __ldg(bv.ids + s);
                if (d2 < Q.best || id < Q.id) { Q.best = d2; Q.slot = s; Q.id = id; }
            }
        }
    } else if (Q.q == kQSil) {
        const DevBVH &bv = sc.sil;
        vis.sprims += cnt;
        for (int s = s0; s < s0 + cnt; ++s) {
            float d2, o0, o1;
            bool always;
            if (D == 2) {
                float4 e0 = ldn(bv.prims + 2 * s), e1 = ldn(bv.prims + 2 * s + 1);
                float rx = x[0] - e0.x, ry = x[1] - e0.y;
                d2 = rx * rx + ry * ry;
                o0 = e0.z * rx + e0.w * ry;
                o1 = e1.x * rx + e1.y * ry;
                always = e1.z != 0.f;
            } else {
                float4 e0 = ldn(bv.prims + 4 * s), e1 = ldn(bv.prims + 4 * s + 1);
                float4 e2 = ldn(bv.prims + 4 * s + 2), e3 = ldn(bv.prims + 4 * s + 3);
                float a[3] = {e0.x, e0.y, e0.z}, b[3] = {e0.w, e1.x, e1.y};
                d2 = seg3_d2<float>(a, b, x);
                float r[3] = {x[0] - a[0], x[1] - a[1], x[2] - a[2]};
                o0 = e1.z * r[0] + e1.w * r[1] + e2.x * r[2];
                o1 = e2.y * r[0] + e2.z * r[1] + e2.w * r[2];
                always = e3.x != 0.f;
            }
            if (d2 <= Q.best && (always || sil_rule(o0, o1, sc.tau))) {
                int id = __ldg(bv.ids + s);
                if (d2 < Q.best || id < Q.id) { Q.best = d2; Q.slot = s; Q.id = id; }
            }
        }
    } else {
        const DevBVH &bv = sc.neu;
        vis.nprims += cnt;
        for (int s = s0; s < s0 + cnt; ++s) {
            float t;
            if (s != skip && ray_prim<D, true>(bv.prims, s, x, Q.v, t, tneg) && t <= Q.best) {
                int id = __ldg(bv.ids + s);
                if (t < Q.best || id < Q.id) { Q.best = t; Q.slot = s; Q.id = id; }
            }
        }
    }
    query_pop<D>(Q);
}

// Step values a lane carries between its queries.
struct LaneStep {
    float RD = 0.f;    // distance to the closest Dirichlet point
    float r = 0.f;     // star radius
    float rho = 0.f;   // source sample radius
    float S = 0.f;     // source term of the step
    int dslot = -1;    // closest Dirichlet leaf slot
};

enum : int {
    kLaneGo = 0,      // the next query is set up
    kLaneEnded = 1,   // the walk ended: value in w.acc, terminal value in gv
    kLaneDirection = 2  // the step needs its direction (r and S are set)
};

// The step logic that follows a finished query (the walk-on-stars step of
// walkstep.cuh, split at its queries):
//   Dirichlet  -> epsilon-shell or step cap: end with T g(xbar); else the
//                 silhouette query bounded by R_D;
//   silhouette -> r = max(min(R_D, R_S), eps); the source-visibility ray, or
//                 the direction;
//   source ray -> source term -(r^2 / 2d) f(y) if visible; the direction;
//   step ray   -> move (to the exit hit, tneg inside, or x + r nu); the next
//                 step's Dirichlet query.
template <int D>
__device__ __forceinline__ int lane_after_query(Walk<D> &w, LaneQuery<D> &Q, LaneStep &L, const StepEnv &env,
                                                float &gv, bool &trunc, unsigned long long &nsteps) {
    const DevScene &sc = env.sc;
    const float tneg = kRoundBand * sc.scale;
    if (Q.q == kQDir) {
        L.dslot = Q.slot;
        L.RD = sqrtf(Q.best);
        double q64[3];
        bool have64 = false, shell;
        if (fabsf(L.RD - env.eps) <= kRoundBand * (sc.scale + L.RD)) {
            shell = dirichlet_dist64<D>(sc.dir, L.dslot, w.x, q64) <= env.eps64;
            have64 = true;
        } else {
            shell = L.RD <= env.eps;
        }
        if (shell || w.k >= env.maxsteps) {
            if (!have64) dirichlet_dist64<D>(sc.dir, L.dslot, w.x, q64);
            float xb[3] = {(float)q64[0], (float)q64[1], D == 3 ? (float)q64[2] : 0.f};
            gv = eval_fn<D>(sc.g, xb);
            w.acc += w.T * gv;
            trunc = !shell;
            Q.q = kQNone;
            return kLaneEnded;
        }
        if (roulette_on(env, w.k)) {
            if (!roulette_survives(env, w.pid, w.wid, w.k)) {
                gv = 0.f;
                trunc = false;
                Q.q = kQNone;
                return kLaneEnded;
            }
            w.T *= 1.f / env.rr_q;
        }
        query_begin<D>(Q, sc, kQSil, L.RD * L.RD);
        return kLaneGo;
    }
    if (Q.q == kQSil) {
        const float R = fminf(sqrtf(Q.best), L.RD);
        L.r = fmaxf(R, env.eps);
        L.S = 0.f;
        if (!sc.has_source) {
            if (sc.has_flux) {
                L.S = -neumann_term<D>(w, sc, L.r, env.key0, env.key1, env.err, nullptr);
                w.acc += w.T * L.S;
            }
            return kLaneDirection;
        }
        U4 u = philox(w.pid, w.wid, (uint32_t)w.k, P_SRC, env.key0, env.key1);
        float vs[D];
        uniform_dir<D>(u01(u.x), u01(u.y), vs);
        if (w.prim >= 0 && dotv<D>(vs, w.n) < 0.f) reflect<D>(vs, w.n);
        L.rho = D == 2 ? L.r * sqrtf(u01(u.z) * u01(u.w)) : L.r * beta22_inv(u01(u.z));
        query_ray<D>(Q, sc, kQSrc, vs, L.rho);
        return kLaneGo;
    }
    if (Q.q == kQSrc) {
        int hs = Q.slot;
        const float th = Q.best;
        if (hs >= 0 && L.rho - th <= kRoundBand * (sc.scale + L.rho)) {
            double t64;
            if (!ray_prim64<D, true>(sc.neu, hs, w.x, Q.v, t64, tneg) || t64 > (double)L.rho) hs = -1;
        }
        L.S = 0.f;
        if (hs < 0) {
            float y[3];
#pragma unroll
            for (int i = 0; i < D; ++i) y[i] = w.x[i] + L.rho * Q.v[i];
            L.S = -(L.r * L.r / (2.f * D)) * eval_fn<D>(sc.f, y);
        }
        if (sc.has_flux) L.S -= neumann_term<D>(w, sc, L.r, env.key0, env.key1, env.err, nullptr);
        w.acc += w.T * L.S;
        return kLaneDirection;
    }
    // kQMove
    int hit = Q.slot;
    float th = Q.best;
    if (hit >= 0 && L.r - th <= kRoundBand * (sc.scale + L.r)) {
        double t64;
        if (!ray_prim64<D, true>(sc.neu, hit, w.x, Q.v, t64, tneg) || t64 > (double)L.r) hit = -1;
    }
    if (hit >= 0) {
        // exit hit: stand tneg inside along the primitive's inward normal
        th = fmaxf(th, 0.f);
#pragma unroll
        for (int i = 0; i < D; ++i) {
            w.n[i] = __ldg(sc.nin_neu + (size_t)hit * D + i);
            w.x[i] += th * Q.v[i] + tneg * w.n[i];
        }
        w.prim = hit;
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) w.x[i] += L.r * Q.v[i];
        w.prim = -1;
    }
    w.k++;
    nsteps++;
    query_begin<D>(Q, sc, kQDir, __int_as_float(0x7f800000));
    return kLaneGo;
}

// One node or leaf phase of the lanes that are searching (all lanes of the
// warp take part).
template <int D, class Src>
__device__ __forceinline__ void lanes_traverse(const Src &src, const Walk<D> &w, LaneQuery<D> &Q, bool searching,
                                               Visits &vis) {
    const StepEnv env = src.env(w);
    const float tneg = kRoundBand * env.sc.scale;
    while (__any_sync(0xffffffffu, searching && !Q.fin && Q.ref >= 0)) {
        if (searching && !Q.fin && Q.ref >= 0) query_node<D>(Q, env.sc, w.x, tneg, env.err, vis);
    }
    if (searching && !Q.fin) query_leaf<D>(Q, env.sc, w.x, w.prim, tneg, vis);
}

// The plain walk (uniform directions, reflection at Neumann points) over a
// job source, step for step the computation of plain_loop: the same random
// numbers, tests and updates in the same order per walk.
template <int D, class Src>
__device__ __forceinline__ void plain_loop_lanes(const Src &src, unsigned long long *stat) {
    Walk<D> w;
    w.job = 0;        // a lane without a walk still names a valid job
    w.prim = -1;
    LaneQuery<D> Q;
    LaneStep L;
    Visits vis;
    bool active = false, exhausted = false;
    unsigned long long nsteps = 0, ntrunc = 0, nwalks = 0;
    for (;;) {
        // ---- logic phase ----
        if (Q.fin && Q.q != kQNone) {
            const StepEnv env = src.env(w);
            float gv = 0.f;
            bool trunc = false;
            const int res = lane_after_query<D>(w, Q, L, env, gv, trunc, nsteps);
            if (res == kLaneEnded) {
                src.finish(w);
                ntrunc += trunc;
                active = false;
            } else if (res == kLaneDirection) {
                U4 u = philox(w.pid, w.wid, (uint32_t)w.k, P_DIR, env.key0, env.key1);
                float nu[D];
                uniform_dir<D>(u01(u.x), u01(u.y), nu);
                bool ended = false;
                if (w.prim >= 0) {
                    float dn = dotv<D>(nu, w.n);
                    if (dn < 0.f) reflect<D>(nu, w.n);
                    ended = dn == 0.f;   // zero density at the tangent plane (Eq. angular_req)
                }
                if (ended) {
                    src.finish(w);
                    active = false;
                    Q.q = kQNone;
                } else {
                    query_ray<D>(Q, env.sc, kQMove, nu, L.r);
                }
            }
        }
        if (!active && !exhausted) {
            unsigned long long item = warp_fetch_add(src.work_ctr(), true);
            if (item >= src.total()) {
                exhausted = true;
            } else if (src.start(w, item)) {
                active = true;
                nwalks++;
                nsteps++;
                query_begin<D>(Q, src.env(w).sc, kQDir, __int_as_float(0x7f800000));
            }
        }
        if (!__any_sync(0xffffffffu, active || !exhausted)) break;
        __syncwarp();
        const bool searching = active && !Q.fin;
        if (!__any_sync(0xffffffffu, searching)) continue;
        // ---- node and leaf phases ----
        lanes_traverse<D>(src, w, Q, searching, vis);
    }
    flush_stats(stat, nsteps, ntrunc, nwalks, vis);
}

}  // namespace wost
