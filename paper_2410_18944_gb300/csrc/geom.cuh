// Boundary queries of one walk step (Sec. 3.2, Sec. 5.3): closest Dirichlet
// point (epsilon-shell test, R_D), closest Neumann silhouette (R_S), first
// Neumann hit along a ray (next point on the star boundary).  Stack-based
// traversal of a binary BVH with child boxes in the parent; node and
// primitive loads are 16-byte vector loads through the read-only path.
// Ties between equal distances go to the smaller original primitive id.
#pragma once
#include <climits>

#include "common.cuh"

namespace wost {

constexpr int kStack = 64;

// The closest-point, closest-silhouette and ray queries compiled out of line
// (a call per query; the caller's live registers no longer add to the
// traversal's), or inlined into the walk step.  Measured on one GB300,
// guided training batches: out of line the icosphere took 317 against 342
// ms, but genus-3 724 against 686, the star 58.5 against 55.0, and plain 2D
// walks ran 16% slower; inlined is the default.
#ifndef WOST_QUERY_NOINLINE
#define WOST_QUERY_NOINLINE 0
#endif
#if WOST_QUERY_NOINLINE
#define WOST_QUERY_FN __noinline__
#else
#define WOST_QUERY_FN
#endif

// Children per BVH node, by dimension: 2 (binary, child boxes in the
// parent) or 4 (the binary tree collapsed one level: four child boxes per
// node, stored one coordinate of all four children per float4).  Width 4
// halves the chain of dependent node loads from the root to a leaf.
// Measured on one GB300: 3D walks 8-10% faster with width 4 (L2-resident
// BVHs of 82k and 994k triangles); 2D walks 25-31% slower (the 4096-segment
// scene's BVH sits in L1 or shared memory, and the wider visit costs more
// instructions and registers than the shorter chain saves).
#ifndef WOST_BVH_WIDTH_2D
#define WOST_BVH_WIDTH_2D 2
#endif
#ifndef WOST_BVH_WIDTH_3D
#define WOST_BVH_WIDTH_3D 4
#endif
__host__ __device__ constexpr int bvh_width(int d) { return d == 2 ? WOST_BVH_WIDTH_2D : WOST_BVH_WIDTH_3D; }
static_assert((bvh_width(2) == 2 || bvh_width(2) == 4) && (bvh_width(3) == 2 || bvh_width(3) == 4),
              "BVH width must be 2 or 4");
constexpr int kEmptyRef = INT_MIN;   // child slot without a child (width 4)

// float4 per node: width 2: 2D 3, 3D 4; width 4: 2D 5, 3D 7
template <int D>
__host__ __device__ constexpr int node_f4() {
    return bvh_width(D) == 2 ? (D == 2 ? 3 : 4) : (D == 2 ? 5 : 7);
}

// per-thread visit counts of the traversals (algorithmic-traffic accounting)
struct Visits {
    uint32_t nodes = 0, dprims = 0, sprims = 0, nprims = 0;
};

// squared distance from x to the two child boxes of a node
template <int D>
__device__ __forceinline__ void node_box_d2(const float4 *nodes, int node, const float *x,
                                            float &d0, float &d1, int &r0, int &r1) {
    if (D == 2) {
        const float4 a = ldn(nodes + 3 * node), b = ldn(nodes + 3 * node + 1), r = ldn(nodes + 3 * node + 2);
        float ax = fmaxf(fmaxf(a.x - x[0], x[0] - a.z), 0.f), ay = fmaxf(fmaxf(a.y - x[1], x[1] - a.w), 0.f);
        float bx = fmaxf(fmaxf(b.x - x[0], x[0] - b.z), 0.f), by = fmaxf(fmaxf(b.y - x[1], x[1] - b.w), 0.f);
        d0 = ax * ax + ay * ay;
        d1 = bx * bx + by * by;
        r0 = __float_as_int(r.x);
        r1 = __float_as_int(r.y);
    } else {
        const float4 a = ldn(nodes + 4 * node), b = ldn(nodes + 4 * node + 1);
        const float4 c = ldn(nodes + 4 * node + 2), r = ldn(nodes + 4 * node + 3);
        // child 0: lo = (a.x, a.y, a.z) hi = (a.w, b.x, b.y); child 1: lo = (b.z, b.w, c.x) hi = (c.y, c.z, c.w)
        float ax = fmaxf(fmaxf(a.x - x[0], x[0] - a.w), 0.f);
        float ay = fmaxf(fmaxf(a.y - x[1], x[1] - b.x), 0.f);
        float az = fmaxf(fmaxf(a.z - x[2], x[2] - b.y), 0.f);
        float bx = fmaxf(fmaxf(b.z - x[0], x[0] - c.y), 0.f);
        float by = fmaxf(fmaxf(b.w - x[1], x[1] - c.z), 0.f);
        float bz = fmaxf(fmaxf(c.x - x[2], x[2] - c.w), 0.f);
        d0 = ax * ax + ay * ay + az * az;
        d1 = bx * bx + by * by + bz * bz;
        r0 = __float_as_int(r.x);
        r1 = __float_as_int(r.y);
    }
}

// entry/exit of the ray o + t v (inv = 1/v) with the two child boxes
// (exit casts: from t > -pad, boxes grown by pad on every side, so that
// crossings within the rounding band of a primitive are not pruned)
template <int D>
__device__ __forceinline__ void node_box_ray(const float4 *nodes, int node, const float *o,
                                             const float *inv, float tmax, float &t0, float &t1,
                                             int &r0, int &r1, float pad = 0.f) {
    float lo0[3], hi0[3], lo1[3], hi1[3];
    if (D == 2) {
        const float4 a = ldn(nodes + 3 * node), b = ldn(nodes + 3 * node + 1), r = ldn(nodes + 3 * node + 2);
        lo0[0] = a.x; lo0[1] = a.y; hi0[0] = a.z; hi0[1] = a.w;
        lo1[0] = b.x; lo1[1] = b.y; hi1[0] = b.z; hi1[1] = b.w;
        r0 = __float_as_int(r.x);
        r1 = __float_as_int(r.y);
    } else {
        const float4 a = ldn(nodes + 4 * node), b = ldn(nodes + 4 * node + 1);
        const float4 c = ldn(nodes + 4 * node + 2), r = ldn(nodes + 4 * node + 3);
        lo0[0] = a.x; lo0[1] = a.y; lo0[2] = a.z; hi0[0] = a.w; hi0[1] = b.x; hi0[2] = b.y;
        lo1[0] = b.z; lo1[1] = b.w; lo1[2] = c.x; hi1[0] = c.y; hi1[1] = c.z; hi1[2] = c.w;
        r0 = __float_as_int(r.x);
        r1 = __float_as_int(r.y);
    }
    float e0 = -pad, x0 = tmax, e1 = -pad, x1 = tmax;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float a0 = (lo0[k] - pad - o[k]) * inv[k], b0 = (hi0[k] + pad - o[k]) * inv[k];
        float a1 = (lo1[k] - pad - o[k]) * inv[k], b1 = (hi1[k] + pad - o[k]) * inv[k];
        e0 = fmaxf(e0, fminf(a0, b0));
        x0 = fminf(x0, fmaxf(a0, b0));
        e1 = fmaxf(e1, fminf(a1, b1));
        x1 = fminf(x1, fmaxf(a1, b1));
    }
    t0 = e0 <= x0 ? e0 : __int_as_float(0x7f800000);
    t1 = e1 <= x1 ? e1 : __int_as_float(0x7f800000);
}

// ---- node visits of either width ---------------------------------------------
// keys of the children: squared distance from x to the child box
template <int D>
__device__ __forceinline__ void node_keys_d2(const float4 *nodes, int node, const float *x, float *k, int *r) {
    constexpr int kBW = bvh_width(D);
    if (kBW == 2) {
        node_box_d2<D>(nodes, node, x, k[0], k[1], r[0], r[1]);
        return;
    }
    const float4 *p = nodes + (size_t)node_f4<D>() * node;
    const float4 lx = ldn(p), ly = ldn(p + 1);
    const float4 lz = D == 3 ? ldn(p + 2) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 hx = ldn(p + (D == 3 ? 3 : 2)), hy = ldn(p + (D == 3 ? 4 : 3));
    const float4 hz = D == 3 ? ldn(p + 5) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 rr = ldn(p + (D == 3 ? 6 : 4));
    const float LX[4] = {lx.x, lx.y, lx.z, lx.w}, LY[4] = {ly.x, ly.y, ly.z, ly.w}, LZ[4] = {lz.x, lz.y, lz.z, lz.w};
    const float HX[4] = {hx.x, hx.y, hx.z, hx.w}, HY[4] = {hy.x, hy.y, hy.z, hy.w}, HZ[4] = {hz.x, hz.y, hz.z, hz.w};
    const float RR[4] = {rr.x, rr.y, rr.z, rr.w};
#pragma unroll
    for (int c = 0; c < kBW; ++c) {
        float dx = fmaxf(fmaxf(LX[c] - x[0], x[0] - HX[c]), 0.f);
        float dy = fmaxf(fmaxf(LY[c] - x[1], x[1] - HY[c]), 0.f);
        float d2 = dx * dx + dy * dy;
        if (D == 3) {
            float dz = fmaxf(fmaxf(LZ[c] - x[2], x[2] - HZ[c]), 0.f);
            d2 += dz * dz;
        }
        k[c] = d2;
        r[c] = __float_as_int(RR[c]);
    }
}

// keys of the children: entry parameter of the ray o + t v (inv = 1/v) into
// the child box grown by pad, from t > -pad, +inf if it misses within tmax
template <int D>
__device__ __forceinline__ void node_keys_ray(const float4 *nodes, int node, const float *o, const float *inv,
                                              float tmax, float *k, int *r, float pad) {
    constexpr int kBW = bvh_width(D);
    if (kBW == 2) {
        node_box_ray<D>(nodes, node, o, inv, tmax, k[0], k[1], r[0], r[1], pad);
        return;
    }
    const float4 *p = nodes + (size_t)node_f4<D>() * node;
    float4 lo4[3], hi4[3];
    lo4[0] = ldn(p);
    lo4[1] = ldn(p + 1);
    lo4[2] = D == 3 ? ldn(p + 2) : make_float4(0.f, 0.f, 0.f, 0.f);
    hi4[0] = ldn(p + (D == 3 ? 3 : 2));
    hi4[1] = ldn(p + (D == 3 ? 4 : 3));
    hi4[2] = D == 3 ? ldn(p + 5) : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 rr = ldn(p + (D == 3 ? 6 : 4));
    const float RR[4] = {rr.x, rr.y, rr.z, rr.w};
    float e[4] = {-pad, -pad, -pad, -pad}, xm[4] = {tmax, tmax, tmax, tmax};
#pragma unroll
    for (int a = 0; a < D; ++a) {
        const float L[4] = {lo4[a].x, lo4[a].y, lo4[a].z, lo4[a].w};
        const float H[4] = {hi4[a].x, hi4[a].y, hi4[a].z, hi4[a].w};
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            float t0 = (L[c] - pad - o[a]) * inv[a], t1 = (H[c] + pad - o[a]) * inv[a];
            e[c] = fmaxf(e[c], fminf(t0, t1));
            xm[c] = fminf(xm[c], fmaxf(t0, t1));
        }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        k[c] = e[c] <= xm[c] ? e[c] : __int_as_float(0x7f800000);
        r[c] = __float_as_int(RR[c]);
    }
}

// box of child c (cone tests)
template <int D>
__device__ __forceinline__ void node_child_box(const float4 *nodes, int node, int c, float *lo, float *hi);

// Continue at the nearest child with h[c] (ties: the lower child index) and
// push the others, farthest first.  Returns false if no child is taken.
template <int kBW>
__device__ __forceinline__ bool take_children(const float *k, const int *r, const bool *h, int &ref, int *stack,
                                              float *skey, int &sp, int *err) {
    float kk[kBW];
    int rr[kBW], n = 0;
#pragma unroll
    for (int c = 0; c < kBW; ++c) {
        kk[c] = h[c] ? k[c] : __int_as_float(0x7f800000);
        rr[c] = r[c];
        n += h[c] ? 1 : 0;
    }
    if (n == 0) return false;
    auto cs = [&](int i, int j) {
        if (kk[j] < kk[i]) {
            float tk = kk[i]; kk[i] = kk[j]; kk[j] = tk;
            int tr = rr[i]; rr[i] = rr[j]; rr[j] = tr;
        }
    };
    if (kBW == 2) {
        cs(0, 1);
    } else {
        cs(0, 1); cs(2, 3); cs(0, 2); cs(1, 3); cs(1, 2);
    }
#pragma unroll
    for (int i = kBW - 1; i >= 1; --i) {
        if (i < n) {
            if (sp < kStack) {
                stack[sp] = rr[i];
                skey[sp] = kk[i];
                ++sp;
            } else {
                atomicOr(err, 1);
            }
        }
    }
    ref = rr[0];
    return true;
}

// ---- primitive distances ----------------------------------------------------
template <typename R>
__device__ __forceinline__ R seg_d2(R ax, R ay, R bx, R by, R px, R py, R &qx, R &qy) {
    R ex = bx - ax, ey = by - ay;
    R ee = ex * ex + ey * ey;
    R t = ee > R(0) ? ((px - ax) * ex + (py - ay) * ey) / ee : R(0);
    t = t < R(0) ? R(0) : (t > R(1) ? R(1) : t);
    qx = ax + t * ex;
    qy = ay + t * ey;
    R dx = px - qx, dy = py - qy;
    return dx * dx + dy * dy;
}

template <typename R>
__device__ __forceinline__ R seg3_d2(const R *a, const R *b, const R *p) {
    R e[3], ap[3], ee = 0, t = 0;
    for (int i = 0; i < 3; ++i) { e[i] = b[i] - a[i]; ap[i] = p[i] - a[i]; ee += e[i] * e[i]; t += ap[i] * e[i]; }
    t = ee > R(0) ? t / ee : R(0);
    t = t < R(0) ? R(0) : (t > R(1) ? R(1) : t);
    R s = 0;
    for (int i = 0; i < 3; ++i) { R d = ap[i] - t * e[i]; s += d * d; }
    return s;
}

// closest point on a triangle by Voronoi regions (Ericson 2004, Sec. 5.1.5)
template <typename R>
__device__ __forceinline__ R tri_d2(const R *a, const R *b, const R *c, const R *p, R *q) {
    R ab[3], ac[3], ap[3], bp[3], cp[3];
    for (int i = 0; i < 3; ++i) { ab[i] = b[i] - a[i]; ac[i] = c[i] - a[i]; ap[i] = p[i] - a[i]; bp[i] = p[i] - b[i]; cp[i] = p[i] - c[i]; }
    auto dot = [](const R *u, const R *v) { return u[0] * v[0] + u[1] * v[1] + u[2] * v[2]; };
    R d1 = dot(ab, ap), d2 = dot(ac, ap);
    R d3 = dot(ab, bp), d4 = dot(ac, bp);
    R d5 = dot(ab, cp), d6 = dot(ac, cp);
    R vc = d1 * d4 - d3 * d2, vb = d5 * d2 - d1 * d6, va = d3 * d6 - d5 * d4;
    if (d1 <= R(0) && d2 <= R(0)) {
        for (int i = 0; i < 3; ++i) q[i] = a[i];
    } else if (d3 >= R(0) && d4 <= d3) {
        for (int i = 0; i < 3; ++i) q[i] = b[i];
    } else if (vc <= R(0) && d1 >= R(0) && d3 <= R(0)) {
        R v = d1 / (d1 - d3);
        for (int i = 0; i < 3; ++i) q[i] = a[i] + v * ab[i];
    } else if (d6 >= R(0) && d5 <= d6) {
        for (int i = 0; i < 3; ++i) q[i] = c[i];
    } else if (vb <= R(0) && d2 >= R(0) && d6 <= R(0)) {
        R w = d2 / (d2 - d6);
        for (int i = 0; i < 3; ++i) q[i] = a[i] + w * ac[i];
    } else if (va <= R(0) && (d4 - d3) >= R(0) && (d5 - d6) >= R(0)) {
        R w = (d4 - d3) / ((d4 - d3) + (d5 - d6));
        for (int i = 0; i < 3; ++i) q[i] = b[i] + w * (c[i] - b[i]);
    } else {
        R den = R(1) / (va + vb + vc);
        R v = vb * den, w = vc * den;
        for (int i = 0; i < 3; ++i) q[i] = a[i] + v * ab[i] + w * ac[i];
    }
    R s = 0;
    for (int i = 0; i < 3; ++i) { R d = p[i] - q[i]; s += d * d; }
    return s;
}

__device__ __forceinline__ void load_tri(const float4 *__restrict__ P, int s, float *a, float *b, float *c) {
    float4 u = ldn(P + 3 * s), v = ldn(P + 3 * s + 1), w = ldn(P + 3 * s + 2);
    a[0] = u.x; a[1] = u.y; a[2] = u.z; b[0] = u.w; b[1] = v.x; b[2] = v.y; c[0] = v.z; c[1] = v.w; c[2] = w.x;
}

// ---- warp-synchronous traversal ------------------------------------------------
// Every traversal below runs as a loop whose iterations are taken together by
// all lanes of the warp that entered it (a warp vote at the loop head): in one
// iteration each unfinished lane processes one inner node or one leaf, then
// pops its stack if needed.  Lanes that diverge inside an iteration
// re-converge at its end, instead of drifting apart for the rest of the
// traversal.
#define WOST_POP(stack, sd, sp, ref, done, best)               \
    do {                                                       \
        bool found_ = false;                                   \
        while (sp > 0) {                                       \
            --sp;                                              \
            if (sd[sp] <= best) { ref = stack[sp]; found_ = true; break; } \
        }                                                      \
        if (!found_) done = true;                              \
    } while (0)

// ---- closest Dirichlet primitive -------------------------------------------
// returns the leaf slot of the closest primitive (-1 if none); best = squared distance
template <int D>
__device__ WOST_QUERY_FN int closest_dirichlet(const DevBVH &bv, const float *x, float &best, int *err, Visits *vis = nullptr) {
    constexpr int kBW = bvh_width(D);
    best = __int_as_float(0x7f800000);
    if (bv.nprims == 0) return -1;
    const unsigned mask = __activemask();
    int best_slot = -1, best_id = 0x7fffffff;
    int stack[kStack];
    float sd[kStack];
    int sp = 0, ref = 0;
    bool done = false;
    // while-while: descend inner nodes together until every lane holds a
    // leaf (or is done), then test the leaves together
    while (__any_sync(mask, !done)) {
        while (__any_sync(mask, !done && ref >= 0)) {
            if (done || ref < 0) continue;
            float k[kBW];
            int r[kBW];
            bool h[kBW];
            node_keys_d2<D>(bv.nodes, ref, x, k, r);
            if (vis) vis->nodes++;
#pragma unroll
            for (int c = 0; c < kBW; ++c) h[c] = r[c] != kEmptyRef && k[c] <= best;
            if (!take_children<kBW>(k, r, h, ref, stack, sd, sp, err)) WOST_POP(stack, sd, sp, ref, done, best);
        }
        if (!done && ref < 0) {
            int s0 = leaf_start(ref), cnt = leaf_count(ref);
            if (vis) vis->dprims += cnt;
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
                if (d2 <= best) {
                    int id = __ldg(bv.ids + s);
                    if (d2 < best || id < best_id) { best = d2; best_slot = s; best_id = id; }
                }
            }
            WOST_POP(stack, sd, sp, ref, done, best);
        }
    }
    return best_slot;
}

// FP64 distance (and closest point) from x to Dirichlet leaf slot s
template <int D>
__device__ __forceinline__ double dirichlet_dist64(const DevBVH &bv, int s, const float *x, double *q) {
    double p[3] = {x[0], x[1], D == 3 ? x[2] : 0.0};
    if (D == 2) {
        const double *v = bv.prims64 + 4 * (size_t)s;
        double d2 = seg_d2<double>(v[0], v[1], v[2], v[3], p[0], p[1], q[0], q[1]);
        return sqrt(d2);
    } else {
        const double *v = bv.prims64 + 9 * (size_t)s;
        return sqrt(tri_d2<double>(v, v + 3, v + 6, p, q));
    }
}

// ---- closest silhouette ------------------------------------------------------
// Silhouette rule: o = signed distance of x to the plane of an adjacent
// Neumann primitive (positive on the domain side); front o > tau, back
// o < -tau, edge-on otherwise; a silhouette has one neighbour seen from the
// back and the other from the front or edge-on.  Elements flagged "always"
// border the Neumann set.  Search radius starts at sqrt(best) (cap).
__device__ __forceinline__ bool sil_rule(float o0, float o1, float tau) {
    int c0 = o0 > tau ? 1 : (o0 < -tau ? -1 : 0);
    int c1 = o1 > tau ? 1 : (o1 < -tau ? -1 : 0);
    return (c0 == -1 && c1 >= 0) || (c1 == -1 && c0 >= 0);
}

// Normal-cone test of a silhouette-BVH child: no element below it can be a
// silhouette from x when every normal in its cone (axis a, half-angle t) is
// strictly front- or strictly back-facing from every point of its box.  With
// c = x - (box centre), view half-angle p = asin(R / |c|) (R = box
// half-diagonal), that holds when |a . c/|c|| > sin(t + p); the margin
// tau / dist keeps every |o| above the edge-on tolerance.
template <int D>
__device__ __forceinline__ bool cone_prunes(float4 cone, const float *lo, const float *hi, const float *x,
                                            float dist2, float tau) {
    if (cone.w <= 0.f || dist2 <= 0.f) return false;
    float c[3], r2 = 0.f, cl2 = 0.f, ac = 0.f;
    const float ax[3] = {cone.x, cone.y, cone.z};
#pragma unroll
    for (int k = 0; k < D; ++k) {
        float h = 0.5f * (hi[k] - lo[k]);
        c[k] = x[k] - 0.5f * (hi[k] + lo[k]);
        r2 += h * h;
        cl2 += c[k] * c[k];
        ac += ax[k] * c[k];
    }
    if (cl2 <= r2) return false;
    float inv = rsqrtf(cl2);
    float sp = sqrtf(r2) * inv, cp = sqrtf(fmaxf(0.f, 1.f - sp * sp));
    float ct = cone.w, st = sqrtf(fmaxf(0.f, 1.f - ct * ct));
    if (ct * cp - st * sp <= 0.f) return false;          // t + p >= 90 degrees
    float s_tp = st * cp + ct * sp;                      // sin(t + p)
    return fabsf(ac) * inv > s_tp + 2.f * tau * rsqrtf(dist2) + 1e-6f;
}

template <int D>
__device__ __forceinline__ void child_boxes(const float4 *nodes, int node, float *lo0, float *hi0,
                                            float *lo1, float *hi1) {
    if (D == 2) {
        const float4 a = ldn(nodes + 3 * node), b = ldn(nodes + 3 * node + 1);
        lo0[0] = a.x; lo0[1] = a.y; hi0[0] = a.z; hi0[1] = a.w;
        lo1[0] = b.x; lo1[1] = b.y; hi1[0] = b.z; hi1[1] = b.w;
    } else {
        const float4 a = ldn(nodes + 4 * node), b = ldn(nodes + 4 * node + 1), c = ldn(nodes + 4 * node + 2);
        lo0[0] = a.x; lo0[1] = a.y; lo0[2] = a.z; hi0[0] = a.w; hi0[1] = b.x; hi0[2] = b.y;
        lo1[0] = b.z; lo1[1] = b.w; lo1[2] = c.x; hi1[0] = c.y; hi1[1] = c.z; hi1[2] = c.w;
    }
}

template <int D>
__device__ __forceinline__ void node_child_box(const float4 *nodes, int node, int c, float *lo, float *hi) {
    if (bvh_width(D) == 2) {
        float lo1[3], hi1[3];
        if (c == 0) child_boxes<D>(nodes, node, lo, hi, lo1, hi1);
        else child_boxes<D>(nodes, node, lo1, hi1, lo, hi);
        return;
    }
    const float *p = reinterpret_cast<const float *>(nodes + (size_t)node_f4<D>() * node);
#pragma unroll
    for (int a = 0; a < D; ++a) {
        lo[a] = p[4 * a + c];
        hi[a] = p[4 * (D + a) + c];
    }
}

template <int D>
__device__ WOST_QUERY_FN int closest_silhouette(const DevBVH &bv, const float *x, float tau, float &best, int *err,
                                   Visits *vis = nullptr, const float4 *cones = nullptr) {
    constexpr int kBW = bvh_width(D);
    if (bv.nprims == 0) return -1;
    const unsigned mask = __activemask();
    int best_slot = -1, best_id = 0x7fffffff;
    int stack[kStack];
    float sd[kStack];
    int sp = 0, ref = 0;
    bool done = false;
    // while-while: descend inner nodes together until every lane holds a
    // leaf (or is done), then test the leaves together
    while (__any_sync(mask, !done)) {
        while (__any_sync(mask, !done && ref >= 0)) {
            if (done || ref < 0) continue;
            float k[kBW];
            int r[kBW];
            bool h[kBW];
            node_keys_d2<D>(bv.nodes, ref, x, k, r);
            if (vis) vis->nodes++;
#pragma unroll
            for (int c = 0; c < kBW; ++c) {
                h[c] = r[c] != kEmptyRef && k[c] <= best;
                if (cones && h[c]) {
                    float lo[3], hi[3];
                    node_child_box<D>(bv.nodes, ref, c, lo, hi);
                    if (cone_prunes<D>(ldn(cones + kBW * ref + c), lo, hi, x, k[c], tau)) h[c] = false;
                }
            }
            if (!take_children<kBW>(k, r, h, ref, stack, sd, sp, err)) WOST_POP(stack, sd, sp, ref, done, best);
        }
        if (!done && ref < 0) {
            int s0 = leaf_start(ref), cnt = leaf_count(ref);
            if (vis) vis->sprims += cnt;
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
                if (d2 <= best && (always || sil_rule(o0, o1, tau))) {
                    int id = __ldg(bv.ids + s);
                    if (d2 < best || id < best_id) { best = d2; best_slot = s; best_id = id; }
                }
            }
            WOST_POP(stack, sd, sp, ref, done, best);
        }
    }
    return best_slot;
}

// ---- ray cast against Neumann primitives --------------------------------------
// kExit: count only primitives the ray leaves the domain through.  The
// boundary is closed and oriented (2D: domain left of a -> b; 3D: triangles
// counter-clockwise seen from outside), so from inside the domain the first
// crossing is always such an exit; an entry hit can only come from a start
// point that rounding put a hair outside the boundary, and taking it would
// put the walker on the wrong side.  2D: exit iff cross(v, b - a) > 0;
// 3D: exit iff v . ((b - a) x (c - a)) > 0, i.e. the Moller-Trumbore
// determinant (b - a) . (v x (c - a)) is negative.  Exit hits count from
// t > -tneg and within about tneg of the primitive (segment parameter /
// barycentric slack tneg over the length / smallest height): a walker that
// stands on a Neumann primitive within rounding of its end vertex and heads
// out through the next primitive crosses it at t ~ 0, and rounding can put
// that crossing slightly behind the start or past the primitive's end; a
// start point inside the domain has no exit crossing behind it.
template <int D, bool kExit = false>
__device__ __forceinline__ bool ray_prim(const float4 *__restrict__ P, int s, const float *o, const float *v, float &t,
                                         float tneg = 0.f) {
    if (D == 2) {
        float4 p = ldn(P + s);
        float ex = p.z - p.x, ey = p.w - p.y;
        float ax = p.x - o[0], ay = p.y - o[1];
        float den = v[0] * ey - v[1] * ex;
        if (kExit ? !(den > 0.f) : den == 0.f) return false;
        float tt = (ax * ey - ay * ex) / den;
        float ss = (ax * v[1] - ay * v[0]) / den;
        const float eta = kExit ? tneg * rsqrtf(ex * ex + ey * ey) : 0.f;
        if (ss < -eta || ss > 1.f + eta || !(tt > (kExit ? -tneg : 0.f))) return false;
        t = tt;
        return true;
    } else {
        float a[3], b[3], c[3];
        load_tri(P, s, a, b, c);
        float e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        float pv[3] = {v[1] * e2[2] - v[2] * e2[1], v[2] * e2[0] - v[0] * e2[2], v[0] * e2[1] - v[1] * e2[0]};
        float det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
        if (kExit ? !(det < 0.f) : det == 0.f) return false;
        float eta = 0.f;
        if (kExit) {
            float n0 = e1[1] * e2[2] - e1[2] * e2[1], n1 = e1[2] * e2[0] - e1[0] * e2[2], n2 = e1[0] * e2[1] - e1[1] * e2[0];
            float e3[3] = {e2[0] - e1[0], e2[1] - e1[1], e2[2] - e1[2]};
            float l2 = fmaxf(fmaxf(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]),
                             e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
            eta = tneg * sqrtf(l2) * rsqrtf(n0 * n0 + n1 * n1 + n2 * n2);
        }
        float inv = 1.f / det;
        float tv[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
        float u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * inv;
        if (u < -eta || u > 1.f + eta) return false;
        float qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
        float w = (v[0] * qv[0] + v[1] * qv[1] + v[2] * qv[2]) * inv;
        if (w < -eta || u + w > 1.f + eta) return false;
        float tt = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
        if (!(tt > (kExit ? -tneg : 0.f))) return false;
        t = tt;
        return true;
    }
}

// FP64 re-test of a hit: the same intersection in double precision
template <int D, bool kExit = false>
__device__ __forceinline__ bool ray_prim64(const DevBVH &bv, int s, const float *of, const float *vf, double &t,
                                           double tneg = 0.0) {
    double o[3] = {of[0], of[1], D == 3 ? of[2] : 0.0}, v[3] = {vf[0], vf[1], D == 3 ? vf[2] : 0.0};
    if (D == 2) {
        const double *p = bv.prims64 + 4 * (size_t)s;
        double ex = p[2] - p[0], ey = p[3] - p[1], ax = p[0] - o[0], ay = p[1] - o[1];
        double den = v[0] * ey - v[1] * ex;
        if (kExit ? !(den > 0.0) : den == 0.0) return false;
        double tt = (ax * ey - ay * ex) / den, ss = (ax * v[1] - ay * v[0]) / den;
        const double eta = kExit ? tneg / sqrt(ex * ex + ey * ey) : 0.0;
        if (ss < -eta || ss > 1.0 + eta || !(tt > (kExit ? -tneg : 0.0))) return false;
        t = tt;
        return true;
    } else {
        const double *a = bv.prims64 + 9 * (size_t)s, *b = a + 3, *c = a + 6;
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double pv[3] = {v[1] * e2[2] - v[2] * e2[1], v[2] * e2[0] - v[0] * e2[2], v[0] * e2[1] - v[1] * e2[0]};
        double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
        if (kExit ? !(det < 0.0) : det == 0.0) return false;
        double eta = 0.0;
        if (kExit) {
            double n0 = e1[1] * e2[2] - e1[2] * e2[1], n1 = e1[2] * e2[0] - e1[0] * e2[2], n2 = e1[0] * e2[1] - e1[1] * e2[0];
            double e3[3] = {e2[0] - e1[0], e2[1] - e1[1], e2[2] - e1[2]};
            double l2 = fmax(fmax(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]),
                             e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2]);
            eta = tneg * sqrt(l2 / (n0 * n0 + n1 * n1 + n2 * n2));
        }
        double inv = 1.0 / det;
        double tv[3] = {o[0] - a[0], o[1] - a[1], o[2] - a[2]};
        double u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * inv;
        if (u < -eta || u > 1.0 + eta) return false;
        double qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
        double w = (v[0] * qv[0] + v[1] * qv[1] + v[2] * qv[2]) * inv;
        if (w < -eta || u + w > 1.0 + eta) return false;
        double tt = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
        if (!(tt > (kExit ? -tneg : 0.0))) return false;
        t = tt;
        return true;
    }
}

// first Neumann hit with 0 < t <= tmax, skipping leaf slot `skip`; returns
// slot or -1 (kExit: exit hits only, from t > -tneg, see ray_prim)
template <int D, bool kExit = false>
__device__ WOST_QUERY_FN int ray_neumann(const DevBVH &bv, const float *o, const float *v, float tmax, int skip, float &thit,
                           int *err, Visits *vis = nullptr, float tneg = 0.f) {
    constexpr int kBW = bvh_width(D);
    thit = tmax;
    if (bv.nprims == 0) return -1;
    const unsigned mask = __activemask();
    float inv[3];
#pragma unroll
    for (int k = 0; k < D; ++k) inv[k] = 1.f / v[k];   // +-inf for a zero component is fine in the slab test
    float best = tmax;
    int best_slot = -1, best_id = 0x7fffffff;
    int stack[kStack];
    float st[kStack];
    int sp = 0, ref = 0;
    bool done = false;
    // while-while: descend inner nodes together until every lane holds a
    // leaf (or is done), then test the leaves together
    while (__any_sync(mask, !done)) {
        while (__any_sync(mask, !done && ref >= 0)) {
            if (done || ref < 0) continue;
            float k[kBW];
            int r[kBW];
            bool h[kBW];
            node_keys_ray<D>(bv.nodes, ref, o, inv, best, k, r, kExit ? tneg : 0.f);
            if (vis) vis->nodes++;
#pragma unroll
            for (int c = 0; c < kBW; ++c) h[c] = r[c] != kEmptyRef && k[c] <= best;
            if (!take_children<kBW>(k, r, h, ref, stack, st, sp, err)) WOST_POP(stack, st, sp, ref, done, best);
        }
        if (!done && ref < 0) {
            int s0 = leaf_start(ref), cnt = leaf_count(ref);
            if (vis) vis->nprims += cnt;
            for (int s = s0; s < s0 + cnt; ++s) {
                float t;
                if (s != skip && ray_prim<D, kExit>(bv.prims, s, o, v, t, tneg) && t <= best) {
                    int id = __ldg(bv.ids + s);
                    if (t < best || id < best_id) { best = t; best_slot = s; best_id = id; }
                }
            }
            WOST_POP(stack, st, sp, ref, done, best);
        }
    }
    thit = best;
    return best_slot;
}

// ---- Neumann boundary sample of <N> (Sec. 3.2, Eq. wost_estm) ---------------
// Every Neumann primitive closer to x than r is a candidate with weight w its
// length (2D) or area (3D).  The candidate with the smallest key -log(u)/w,
// u in (0, 1] from the Philox counter (pid, wid, step, P_NKEY | id), is
// chosen: probability w / W (W = the summed weight) whatever order the
// traversal visits the candidates in (weighted sampling with keys,
// Efraimidis & Spirakis 2006); ties go to the smaller id.  Returns the leaf
// slot of the choice (-1 if there is no candidate) and W.
template <int D>
__device__ int neumann_pick(const DevBVH &bv, const float *x, float r, uint32_t pid, uint32_t wid, uint32_t step,
                            uint32_t k0, uint32_t k1, float &W, int *err, Visits *vis = nullptr) {
    constexpr int kBW = bvh_width(D);
    W = 0.f;
    if (bv.nprims == 0) return -1;
    const float r2 = r * r;
    const unsigned mask = __activemask();
    int best_slot = -1, best_id = 0x7fffffff;
    float best_key = __int_as_float(0x7f800000);
    int stack[kStack];
    float sd[kStack];
    int sp = 0, ref = 0;
    bool done = false;
    float lim = r2;   // the search radius never shrinks: WOST_POP compares keys with it
    while (__any_sync(mask, !done)) {
        while (__any_sync(mask, !done && ref >= 0)) {
            if (done || ref < 0) continue;
            float k[kBW];
            int rr[kBW];
            bool h[kBW];
            node_keys_d2<D>(bv.nodes, ref, x, k, rr);
            if (vis) vis->nodes++;
#pragma unroll
            for (int c = 0; c < kBW; ++c) h[c] = rr[c] != kEmptyRef && k[c] < r2;
            if (!take_children<kBW>(k, rr, h, ref, stack, sd, sp, err)) WOST_POP(stack, sd, sp, ref, done, lim);
        }
        if (!done && ref < 0) {
            int s0 = leaf_start(ref), cnt = leaf_count(ref);
            if (vis) vis->nprims += cnt;
            for (int s = s0; s < s0 + cnt; ++s) {
                float d2, w;
                if (D == 2) {
                    float4 p = ldn(bv.prims + s);
                    float qx, qy;
                    d2 = seg_d2<float>(p.x, p.y, p.z, p.w, x[0], x[1], qx, qy);
                    w = sqrtf((p.z - p.x) * (p.z - p.x) + (p.w - p.y) * (p.w - p.y));
                } else {
                    float a[3], b[3], c[3], q[3];
                    load_tri(bv.prims, s, a, b, c);
                    d2 = tri_d2<float>(a, b, c, x, q);
                    float e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
                    float n0 = e1[1] * e2[2] - e1[2] * e2[1], n1 = e1[2] * e2[0] - e1[0] * e2[2], n2 = e1[0] * e2[1] - e1[1] * e2[0];
                    w = 0.5f * sqrtf(n0 * n0 + n1 * n1 + n2 * n2);
                }
                if (!(d2 < r2) || !(w > 0.f)) continue;
                const int id = __ldg(bv.ids + s);
                U4 u = philox(pid, wid, step, P_NKEY | (uint32_t)id, k0, k1);
                const float uu = ((float)(u.x >> 8) + 1.f) * (1.0f / 16777216.0f);   // (0, 1]
                const float key = -logf(uu) / w;
                W += w;
                if (key < best_key || (key == best_key && id < best_id)) { best_key = key; best_slot = s; best_id = id; }
            }
            WOST_POP(stack, sd, sp, ref, done, lim);
        }
    }
    return best_slot;
}

// number of crossings of the ray o + t v (t > 0) with all primitives of a BVH
template <int D>
__device__ int ray_count(const DevBVH &bv, const float *o, const float *v, int *err) {
    constexpr int kBW = bvh_width(D);
    if (bv.nprims == 0) return 0;
    const unsigned mask = __activemask();
    float inv[3];
#pragma unroll
    for (int k = 0; k < D; ++k) inv[k] = 1.f / v[k];
    const float big = 3.0e38f;
    int cnt = 0, stack[kStack], sp = 0, ref = 0;
    float skey[kStack];
    bool done = false;
    while (__any_sync(mask, !done)) {
        if (done) continue;
        bool pop = false;
        if (ref >= 0) {
            float k[kBW];
            int r[kBW];
            bool h[kBW];
            node_keys_ray<D>(bv.nodes, ref, o, inv, big, k, r, 0.f);
#pragma unroll
            for (int c = 0; c < kBW; ++c) h[c] = r[c] != kEmptyRef && k[c] <= big;
            if (!take_children<kBW>(k, r, h, ref, stack, skey, sp, err)) pop = true;
        } else {
            int s0 = leaf_start(ref), c = leaf_count(ref);
            for (int s = s0; s < s0 + c; ++s) {
                float t;
                cnt += ray_prim<D>(bv.prims, s, o, v, t) ? 1 : 0;
            }
            pop = true;
        }
        if (pop) {
            if (sp == 0) done = true;
            else ref = stack[--sp];
        }
    }
    return cnt;
}

}  // namespace wost
