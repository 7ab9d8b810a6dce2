// Scene construction: boundary validation, inward normals, silhouette
// elements (Neumann vertices in 2D, Neumann edges in 3D), three binned-SAH
// BVHs and their upload in leaf order (FP32 for traversal, FP64 copies for
// the epsilon-shell and ray re-tests).  Sec. 5.3: the queries of a WoSt step
// run on a linear BVH in the paper; here the hierarchy is built once on the
// host (not timed) and traversed in the persistent walk kernel.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>

#include "geom.cuh"
#include "internal.h"

namespace wost {

namespace {

#ifndef WOST_BVH_LEAF
#define WOST_BVH_LEAF 16
#endif
constexpr int kLeaf = WOST_BVH_LEAF;   // primitives per leaf (<= 16)
constexpr int kBins = 16;
constexpr int kSahDepth = 40;   // beyond this depth, median splits bound the tree depth

struct Box {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(const Box &b) {
        for (int k = 0; k < 3; ++k) { lo[k] = std::min(lo[k], b.lo[k]); hi[k] = std::max(hi[k], b.hi[k]); }
    }
    void grow(const float *p, int d) {
        for (int k = 0; k < d; ++k) { lo[k] = std::min(lo[k], p[k]); hi[k] = std::max(hi[k], p[k]); }
    }
    float cost(int d) const {
        if (lo[0] > hi[0]) return 0.f;
        float e[3];
        for (int k = 0; k < 3; ++k) e[k] = std::max(hi[k] - lo[k], 0.f);
        return d == 2 ? e[0] + e[1] : e[0] * e[1] + e[1] * e[2] + e[2] * e[0];
    }
};

struct Item {
    Box b;
    float c[3];
    int idx;
    // silhouette elements: inward normals of the two adjacent Neumann
    // primitives; cone_free marks elements that are always silhouettes
    float n0[3] = {0, 0, 0}, n1[3] = {0, 0, 0};
    bool cone_free = false;
};

// Bounding cone (unit axis, cos of the half-angle) of the normals of items
// [b, e); cos < 0 (half-angle beyond 90 degrees or an always-silhouette
// element inside) disables pruning for that child.
static float4 normal_cone(const std::vector<Item> &items, int b, int e, int d) {
    double ax[3] = {0, 0, 0};
    for (int i = b; i < e; ++i) {
        if (items[i].cone_free) return make_float4(0.f, 0.f, 0.f, -2.f);
        for (int k = 0; k < d; ++k) ax[k] += items[i].n0[k] + items[i].n1[k];
    }
    double L = 0;
    for (int k = 0; k < d; ++k) L += ax[k] * ax[k];
    L = std::sqrt(L);
    if (L < 1e-12) return make_float4(0.f, 0.f, 0.f, -2.f);
    for (int k = 0; k < d; ++k) ax[k] /= L;
    double cmin = 1.0;
    for (int i = b; i < e; ++i)
        for (const float *n : {items[i].n0, items[i].n1}) {
            double c = 0;
            for (int k = 0; k < d; ++k) c += ax[k] * n[k];
            cmin = std::min(cmin, c);
        }
    // shrink slightly so that FP32 rounding of the normals stays inside
    cmin -= 1e-6;
    if (cmin <= 0) return make_float4(0.f, 0.f, 0.f, -2.f);
    return make_float4((float)ax[0], (float)ax[1], (float)ax[2], (float)cmin);
}

struct BNode {
    Box box[2];
    int ref[2];
    int range[2][2];   // item ranges of the two children
};

struct Builder {
    int d;
    std::vector<Item> items;
    std::vector<BNode> nodes;
    int maxdepth = 0;

    static int leaf_ref(int start, int count) { return ~((start << 4) | (count - 1)); }

    Box range_box(int b, int e) const {
        Box r;
        for (int i = b; i < e; ++i) r.grow(items[i].b);
        return r;
    }

    int split_median(int b, int e, int axis) {
        int m = (b + e) / 2;
        std::nth_element(items.begin() + b, items.begin() + m, items.begin() + e,
                         [&](const Item &x, const Item &y) {
                             return x.c[axis] < y.c[axis] || (x.c[axis] == y.c[axis] && x.idx < y.idx);
                         });
        return m;
    }

    int rec(int b, int e, int depth) {
        maxdepth = std::max(maxdepth, depth);
        int n = e - b;
        if (n <= kLeaf) return leaf_ref(b, n);
        Box cb;
        for (int i = b; i < e; ++i) cb.grow(items[i].c, d);
        int axis = 0;
        for (int k = 1; k < d; ++k)
            if (cb.hi[k] - cb.lo[k] > cb.hi[axis] - cb.lo[axis]) axis = k;
        float ext = cb.hi[axis] - cb.lo[axis];
        int mid;
        if (!(ext > 0.f)) {
            mid = (b + e) / 2;   // identical centroids: split by index
        } else if (depth > kSahDepth) {
            mid = split_median(b, e, axis);
        } else {
            Box bb[kBins];
            int bn[kBins] = {0};
            auto bin_of = [&](const Item &it) {
                int k = (int)((it.c[axis] - cb.lo[axis]) / ext * kBins);
                return std::min(std::max(k, 0), kBins - 1);
            };
            for (int i = b; i < e; ++i) { int k = bin_of(items[i]); bn[k]++; bb[k].grow(items[i].b); }
            float best = INFINITY;
            int bestk = -1;
            for (int s = 1; s < kBins; ++s) {
                Box L, R;
                int nl = 0, nr = 0;
                for (int k = 0; k < s; ++k) { L.grow(bb[k]); nl += bn[k]; }
                for (int k = s; k < kBins; ++k) { R.grow(bb[k]); nr += bn[k]; }
                if (!nl || !nr) continue;
                float c = L.cost(d) * nl + R.cost(d) * nr;
                if (c < best) { best = c; bestk = s; }
            }
            if (bestk < 0) {
                mid = split_median(b, e, axis);
            } else {
                auto it = std::partition(items.begin() + b, items.begin() + e,
                                         [&](const Item &x) { return bin_of(x) < bestk; });
                mid = (int)(it - items.begin());
                if (mid == b || mid == e) mid = split_median(b, e, axis);
            }
        }
        int node = (int)nodes.size();
        nodes.push_back(BNode{});
        int l = rec(b, mid, depth + 1);
        int r = rec(mid, e, depth + 1);
        nodes[node].ref[0] = l;
        nodes[node].ref[1] = r;
        nodes[node].box[0] = range_box(b, mid);
        nodes[node].box[1] = range_box(mid, e);
        nodes[node].range[0][0] = b; nodes[node].range[0][1] = mid;
        nodes[node].range[1][0] = mid; nodes[node].range[1][1] = e;
        return node;
    }

    // returns false if the tree is too deep for the device traversal stack
    bool build() {
        nodes.clear();
        int n = (int)items.size();
        if (n == 0) return true;
        if (n <= kLeaf) {
            BNode r;
            r.ref[0] = leaf_ref(0, n);
            r.ref[1] = leaf_ref(0, 1);
            r.box[0] = range_box(0, n);   // r.box[1] stays empty (inverted): never entered
            r.range[0][0] = 0; r.range[0][1] = n;
            r.range[1][0] = 0; r.range[1][1] = 0;
            nodes.push_back(r);
            maxdepth = 1;
            return true;
        }
        rec(0, n, 0);
        return maxdepth < 62;   // device traversal stack holds 64 entries
    }

    // ---- device layout ----
    // Width 2: the binary nodes, child boxes in the parent.  Width 4: each
    // node takes up to four descendants of a binary node (its children, with
    // the inner child of the larger box surface opened until there are
    // four); empty slots carry kEmptyRef and an inverted box.
    struct Child { Box box; int ref; int range[2]; };
    struct WNode { Child ch[4]; int n; };
    std::vector<WNode> wide;
    int wdepth = 0;

    int collapse(int bnode, int depth) {
        wdepth = std::max(wdepth, depth);
        Child ch[4];
        int n = 0;
        for (int c = 0; c < 2; ++c)
            ch[n++] = Child{nodes[bnode].box[c], nodes[bnode].ref[c], {nodes[bnode].range[c][0], nodes[bnode].range[c][1]}};
        while (n < 4) {
            int pick = -1;
            float area = -1.f;
            for (int i = 0; i < n; ++i)
                if (ch[i].ref >= 0 && ch[i].box.cost(d) > area) { pick = i; area = ch[i].box.cost(d); }
            if (pick < 0) break;
            const BNode &b = nodes[ch[pick].ref];
            Child c0{b.box[0], b.ref[0], {b.range[0][0], b.range[0][1]}};
            Child c1{b.box[1], b.ref[1], {b.range[1][0], b.range[1][1]}};
            ch[pick] = c0;
            ch[n++] = c1;
        }
        const int id = (int)wide.size();
        wide.push_back(WNode{});
        for (int i = 0; i < 4; ++i) {
            Child c;
            if (i < n) {
                c = ch[i];
                if (c.ref >= 0) c.ref = collapse(c.ref, depth + 1);
            } else {
                c = Child{Box{}, kEmptyRef, {0, 0}};
            }
            wide[id].ch[i] = c;
        }
        wide[id].n = n;
        return id;
    }

    // most stack entries a traversal below wide node id can hold: a visit
    // pushes all but one of its taken children
    int stack_need(int id) const {
        int need = 0;
        for (int c = 0; c < 4; ++c)
            if (wide[id].ch[c].ref >= 0) need = std::max(need, stack_need(wide[id].ch[c].ref));
        return need + std::max(wide[id].n - 1, 0);
    }

    // builds the wide tree (width 4); false if a traversal could overflow
    // the device stack
    bool widen() {
        wide.clear();
        wdepth = 0;
        if (bvh_width(d) == 2 || nodes.empty()) return true;
        collapse(0, 1);
        return stack_need(0) < kStack;
    }

    int device_nodes() const { return bvh_width(d) == 2 ? (int)nodes.size() : (int)wide.size(); }

    // one cone per child
    std::vector<float4> cones() const {
        std::vector<float4> out;
        auto cone = [&](int b, int e) {
            return e > b ? normal_cone(items, b, e, d) : make_float4(0.f, 0.f, 0.f, -2.f);
        };
        if (bvh_width(d) == 2) {
            for (const BNode &nd : nodes)
                for (int c = 0; c < 2; ++c) out.push_back(cone(nd.range[c][0], nd.range[c][1]));
        } else {
            for (const WNode &wn : wide)
                for (int c = 0; c < 4; ++c) out.push_back(cone(wn.ch[c].range[0], wn.ch[c].range[1]));
        }
        return out;
    }

    std::vector<float4> pack() const {
        std::vector<float4> out;
        auto bits = [](int r) { float f; std::memcpy(&f, &r, 4); return f; };
        if (bvh_width(d) == 4) {
            // one coordinate of the four children per float4: lo x, lo y, (lo z,) hi x, hi y, (hi z,) refs
            for (const WNode &wn : wide) {
                for (int side = 0; side < 2; ++side)
                    for (int a = 0; a < d; ++a) {
                        float v[4];
                        for (int c = 0; c < 4; ++c) v[c] = side == 0 ? wn.ch[c].box.lo[a] : wn.ch[c].box.hi[a];
                        out.push_back(make_float4(v[0], v[1], v[2], v[3]));
                    }
                out.push_back(make_float4(bits(wn.ch[0].ref), bits(wn.ch[1].ref), bits(wn.ch[2].ref), bits(wn.ch[3].ref)));
            }
            return out;
        }
        for (const BNode &nd : nodes) {
            const Box &a = nd.box[0], &b = nd.box[1];
            float r0 = bits(nd.ref[0]), r1 = bits(nd.ref[1]);
            if (d == 2) {
                out.push_back(make_float4(a.lo[0], a.lo[1], a.hi[0], a.hi[1]));
                out.push_back(make_float4(b.lo[0], b.lo[1], b.hi[0], b.hi[1]));
                out.push_back(make_float4(r0, r1, 0.f, 0.f));
            } else {
                out.push_back(make_float4(a.lo[0], a.lo[1], a.lo[2], a.hi[0]));
                out.push_back(make_float4(a.hi[1], a.hi[2], b.lo[0], b.lo[1]));
                out.push_back(make_float4(b.lo[2], b.hi[0], b.hi[1], b.hi[2]));
                out.push_back(make_float4(r0, r1, 0.f, 0.f));
            }
        }
        return out;
    }
};

template <class T>
wost_status upload(wost_scene *s, const std::vector<T> &v, const T **out) {
    *out = nullptr;
    if (v.empty()) return WOST_OK;
    void *p = nullptr;
    cudaError_t e = cudaMalloc(&p, v.size() * sizeof(T));
    if (e != cudaSuccess) {
        set_error("cudaMalloc failed while uploading the scene");
        return e == cudaErrorMemoryAllocation ? WOST_ERR_OOM : WOST_ERR_CUDA;
    }
    s->allocs.push_back(p);
    WOST_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    *out = reinterpret_cast<const T *>(p);
    return WOST_OK;
}

bool valid_fn(const wost_fn &f) {
    if (f.kind < 0 || f.kind > 10) return false;
    if (f.kind == 7 && (f.params[0] < 0 || f.params[0] > 8)) return false;
    return true;
}

DevFn to_dev(const wost_fn &f) {
    DevFn o{};
    o.kind = f.kind;
    o.n = f.nparams;
    for (int i = 0; i < 40; ++i) o.p[i] = (float)f.params[i];
    return o;
}

}  // namespace

}  // namespace wost

using namespace wost;

wost_scene::~wost_scene() {
    for (void *p : allocs) cudaFree(p);
    ws_points.release(); ws_status.release(); ws_sum.release(); ws_sum2.release(); ws_ctr.release(); ws_out.release();
    ws_wf.release();
    ws_order.release();
    if (pinned) cudaFreeHost(pinned);
}

extern "C" wost_status wost_create_scene(const wost_scene_desc *desc, wost_scene **out) {
    if (!desc || !out) { set_error("wost_create_scene: null argument"); return WOST_ERR_INVALID_ARG; }
    *out = nullptr;
    const int d = desc->dim;
    if (d != 2 && d != 3) { set_error("wost_create_scene: dim must be 2 or 3"); return WOST_ERR_INVALID_ARG; }
    if (desc->nverts <= 0 || desc->nprims <= 0 || !desc->verts || !desc->prims || !desc->bc) {
        set_error("wost_create_scene: empty or null geometry");
        return WOST_ERR_INVALID_ARG;
    }
    if (desc->nprims >= (1LL << 27) || desc->nverts >= (1LL << 31)) {
        set_error("wost_create_scene: too many primitives");
        return WOST_ERR_INVALID_ARG;
    }
    if (!valid_fn(desc->g) || !valid_fn(desc->f) || !valid_fn(desc->h)) {
        set_error("wost_create_scene: unknown data-function kind");
        return WOST_ERR_INVALID_ARG;
    }
    const int64_t nv = desc->nverts, np = desc->nprims;
    int ndir = 0;
    for (int64_t i = 0; i < np; ++i) {
        if (desc->bc[i] > 1) { set_error("wost_create_scene: bc must be 0 or 1"); return WOST_ERR_INVALID_ARG; }
        ndir += desc->bc[i] == 0;
        for (int k = 0; k < d; ++k) {
            int32_t v = desc->prims[i * d + k];
            if (v < 0 || v >= nv) { set_error("wost_create_scene: vertex index out of range"); return WOST_ERR_INVALID_ARG; }
        }
    }
    for (int64_t i = 0; i < nv * d; ++i)
        if (!std::isfinite(desc->verts[i])) { set_error("wost_create_scene: non-finite vertex"); return WOST_ERR_INVALID_ARG; }
    if (ndir == 0) { set_error("wost_create_scene: no Dirichlet primitive (ill-posed)"); return WOST_ERR_ILL_POSED; }
    int dev = -1;
    WOST_CUDA(cudaGetDevice(&dev));

    auto *s = new wost_scene();
    s->dim = d;
    s->device = dev;
    s->nverts = nv;
    s->nprims = np;
    s->scene_id = desc->scene_id;
    const double *V = desc->verts;
    const int32_t *P = desc->prims;
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < nv; ++i)
        for (int k = 0; k < d; ++k) { lo[k] = std::min(lo[k], V[i * d + k]); hi[k] = std::max(hi[k], V[i * d + k]); }
    double diag = 0;
    for (int k = 0; k < d; ++k) { diag += (hi[k] - lo[k]) * (hi[k] - lo[k]); s->lo[k] = lo[k]; s->hi[k] = hi[k]; }
    diag = std::sqrt(diag);

    // inward unit normals (2D: left perpendicular of b - a; 3D: -(e1 x e2))
    std::vector<double> nin((size_t)np * d);
    for (int64_t i = 0; i < np; ++i) {
        const double *a = V + (size_t)P[i * d] * d, *b = V + (size_t)P[i * d + 1] * d;
        double *n = &nin[(size_t)i * d];
        if (d == 2) {
            double ex = b[0] - a[0], ey = b[1] - a[1], L = std::sqrt(ex * ex + ey * ey);
            n[0] = -ey / L; n[1] = ex / L;
        } else {
            const double *c = V + (size_t)P[i * d + 2] * d;
            double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
            double cx = e1[1] * e2[2] - e1[2] * e2[1], cy = e1[2] * e2[0] - e1[0] * e2[2], cz = e1[0] * e2[1] - e1[1] * e2[0];
            double L = std::sqrt(cx * cx + cy * cy + cz * cz);
            n[0] = -cx / L; n[1] = -cy / L; n[2] = -cz / L;
        }
    }

    auto fv = [&](int64_t vi, int k) { return (float)V[vi * d + k]; };

    // ---- primitive BVHs (Dirichlet, Neumann) ----
    auto build_prims = [&](int bcv, DevBVH &bv, int &count, int &depth, std::vector<int> *slot_of) -> wost_status {
        Builder B;
        B.d = d;
        for (int64_t i = 0; i < np; ++i) {
            if (desc->bc[i] != bcv) continue;
            Item it;
            for (int k = 0; k < 3; ++k) it.c[k] = 0.f;
            for (int j = 0; j < d; ++j) {
                float p[3] = {fv(P[i * d + j], 0), fv(P[i * d + j], 1), d == 3 ? fv(P[i * d + j], 2) : 0.f};
                it.b.grow(p, d);
                for (int k = 0; k < d; ++k) it.c[k] += p[k] / d;
            }
            if (d == 2) { it.b.lo[2] = it.b.hi[2] = 0.f; }
            it.idx = (int)i;
            B.items.push_back(it);
        }
        count = (int)B.items.size();
        if (!B.build() || !B.widen()) { set_error("wost_create_scene: BVH too deep"); return WOST_ERR_INVALID_ARG; }
        depth = B.maxdepth;
        std::vector<float4> prims;
        std::vector<double> p64;
        std::vector<int> ids;
        if (slot_of) slot_of->assign(np, -1);
        for (size_t sidx = 0; sidx < B.items.size(); ++sidx) {
            int i = B.items[sidx].idx;
            ids.push_back(i);
            if (slot_of) (*slot_of)[i] = (int)sidx;
            const int32_t *q = P + (size_t)i * d;
            if (d == 2) {
                prims.push_back(make_float4(fv(q[0], 0), fv(q[0], 1), fv(q[1], 0), fv(q[1], 1)));
                for (int j = 0; j < 2; ++j) for (int k = 0; k < 2; ++k) p64.push_back(V[(size_t)q[j] * 2 + k]);
            } else {
                prims.push_back(make_float4(fv(q[0], 0), fv(q[0], 1), fv(q[0], 2), fv(q[1], 0)));
                prims.push_back(make_float4(fv(q[1], 1), fv(q[1], 2), fv(q[2], 0), fv(q[2], 1)));
                prims.push_back(make_float4(fv(q[2], 2), 0.f, 0.f, 0.f));
                for (int j = 0; j < 3; ++j) for (int k = 0; k < 3; ++k) p64.push_back(V[(size_t)q[j] * 3 + k]);
            }
        }
        wost_status st;
        if ((st = upload(s, B.pack(), &bv.nodes)) != WOST_OK) return st;
        bv.nnodes = B.device_nodes();
        if ((st = upload(s, prims, &bv.prims)) != WOST_OK) return st;
        if ((st = upload(s, ids, &bv.ids)) != WOST_OK) return st;
        if ((st = upload(s, p64, &bv.prims64)) != WOST_OK) return st;
        bv.nprims = count;
        return WOST_OK;
    };
    wost_status st;
    std::vector<int> neu_slot;
    if ((st = build_prims(0, s->dev.dir, s->ndir, s->depth_dir, nullptr)) != WOST_OK) { delete s; return st; }
    if ((st = build_prims(1, s->dev.neu, s->nneu, s->depth_neu, &neu_slot)) != WOST_OK) { delete s; return st; }

    // inward normals of Neumann primitives in leaf order
    {
        std::vector<int> ids(s->nneu);
        std::vector<float> nn((size_t)s->nneu * d);
        for (int64_t i = 0; i < np; ++i)
            if (neu_slot[i] >= 0)
                for (int k = 0; k < d; ++k) nn[(size_t)neu_slot[i] * d + k] = (float)nin[(size_t)i * d + k];
        if ((st = upload(s, nn, &s->dev.nin_neu)) != WOST_OK) { delete s; return st; }
    }

    // ---- silhouette elements ----
    {
        struct Elem { int64_t key; int a, b, f0, f1; };
        std::vector<Elem> el;
        if (d == 2) {
            std::vector<int> in_seg(nv, -1), out_seg(nv, -1);
            for (int64_t i = 0; i < np; ++i)
                if (desc->bc[i] == 1) { out_seg[P[2 * i]] = (int)i; in_seg[P[2 * i + 1]] = (int)i; }
            for (int64_t v = 0; v < nv; ++v)
                if (in_seg[v] >= 0 || out_seg[v] >= 0) el.push_back({v, (int)v, (int)v, in_seg[v], out_seg[v]});
        } else {
            struct E { int a, b, f; };
            std::vector<E> es;
            for (int64_t i = 0; i < np; ++i)
                if (desc->bc[i] == 1)
                    for (int k = 0; k < 3; ++k) {
                        int a = P[3 * i + k], b = P[3 * i + (k + 1) % 3];
                        es.push_back({std::min(a, b), std::max(a, b), (int)i});
                    }
            std::sort(es.begin(), es.end(), [](const E &x, const E &y) {
                return x.a != y.a ? x.a < y.a : (x.b != y.b ? x.b < y.b : x.f < y.f);
            });
            for (size_t i = 0; i < es.size();) {
                size_t j = i;
                while (j < es.size() && es[j].a == es[i].a && es[j].b == es[i].b) ++j;
                bool two = (j - i) == 2;
                el.push_back({(int64_t)es[i].a * nv + es[i].b, es[i].a, es[i].b, two ? es[i].f : -1, two ? es[i + 1].f : -1});
                i = j;
            }
        }
        Builder B;
        B.d = d;
        for (size_t e = 0; e < el.size(); ++e) {
            Item it;
            float pa[3] = {fv(el[e].a, 0), fv(el[e].a, 1), d == 3 ? fv(el[e].a, 2) : 0.f};
            float pb[3] = {fv(el[e].b, 0), fv(el[e].b, 1), d == 3 ? fv(el[e].b, 2) : 0.f};
            it.b.grow(pa, d);
            it.b.grow(pb, d);
            if (d == 2) it.b.lo[2] = it.b.hi[2] = 0.f;
            for (int k = 0; k < 3; ++k) it.c[k] = 0.5f * (pa[k] + pb[k]);
            it.idx = (int)e;
            it.cone_free = el[e].f0 < 0 || el[e].f1 < 0;
            for (int k = 0; k < d; ++k) {
                if (el[e].f0 >= 0) it.n0[k] = (float)nin[(size_t)el[e].f0 * d + k];
                if (el[e].f1 >= 0) it.n1[k] = (float)nin[(size_t)el[e].f1 * d + k];
            }
            B.items.push_back(it);
        }
        s->nsil = (int)el.size();
        if (!B.build() || !B.widen()) { set_error("wost_create_scene: BVH too deep"); delete s; return WOST_ERR_INVALID_ARG; }
        s->depth_sil = B.maxdepth;
        std::vector<float4> prims;
        std::vector<int> ids;
        std::vector<int64_t> keys;
        for (const Item &it : B.items) {
            const Elem &e = el[it.idx];
            ids.push_back(it.idx);
            keys.push_back(e.key);
            bool always = e.f0 < 0 || e.f1 < 0;
            float n0[3] = {0, 0, 0}, n1[3] = {0, 0, 0};
            for (int k = 0; k < d; ++k) {
                if (e.f0 >= 0) n0[k] = (float)nin[(size_t)e.f0 * d + k];
                if (e.f1 >= 0) n1[k] = (float)nin[(size_t)e.f1 * d + k];
            }
            if (d == 2) {
                prims.push_back(make_float4(fv(e.a, 0), fv(e.a, 1), n0[0], n0[1]));
                prims.push_back(make_float4(n1[0], n1[1], always ? 1.f : 0.f, 0.f));
            } else {
                prims.push_back(make_float4(fv(e.a, 0), fv(e.a, 1), fv(e.a, 2), fv(e.b, 0)));
                prims.push_back(make_float4(fv(e.b, 1), fv(e.b, 2), n0[0], n0[1]));
                prims.push_back(make_float4(n0[2], n1[0], n1[1], n1[2]));
                prims.push_back(make_float4(always ? 1.f : 0.f, 0.f, 0.f, 0.f));
            }
        }
        DevBVH &bv = s->dev.sil;
        if ((st = upload(s, B.cones(), &s->dev.sil_cones)) != WOST_OK) { delete s; return st; }
        if ((st = upload(s, B.pack(), &bv.nodes)) != WOST_OK ||
            (st = upload(s, prims, &bv.prims)) != WOST_OK || (st = upload(s, ids, &bv.ids)) != WOST_OK) {
            delete s;
            return st;
        }
        bv.nnodes = B.device_nodes();
        const int64_t *kp = nullptr;
        if ((st = upload(s, keys, &kp)) != WOST_OK) { delete s; return st; }
        s->sil_key = const_cast<int64_t *>(kp);
        bv.prims64 = nullptr;
        bv.nprims = s->nsil;
    }
    s->dev.dim = d;
    s->dev.scale = (float)diag;
    s->dev.tau = (float)(1e-6 * diag);
    s->dev.g = to_dev(desc->g);
    s->dev.f = to_dev(desc->f);
    s->dev.has_source = desc->f.kind != 0;
    s->dev.h = to_dev(desc->h);
    s->dev.has_flux = desc->h.kind != 0 && s->nneu > 0;
    *out = s;
    return WOST_OK;
}

extern "C" wost_status wost_destroy_scene(wost_scene *s) {
    delete s;
    return WOST_OK;
}

extern "C" wost_status wost_scene_device(const wost_scene *s, int32_t *device) {
    if (!s || !device) { set_error("wost_scene_device: null argument"); return WOST_ERR_INVALID_ARG; }
    *device = s->device;
    return WOST_OK;
}

extern "C" wost_status wost_diag_scene_rebind(wost_scene *s, int32_t device) {
    if (!s) { set_error("wost_diag_scene_rebind: null scene"); return WOST_ERR_INVALID_ARG; }
    s->device = device;
    return WOST_OK;
}

extern "C" wost_status wost_scene_bbox(const wost_scene *s, double lo[3], double hi[3]) {
    if (!s || !lo || !hi) { set_error("wost_scene_bbox: null argument"); return WOST_ERR_INVALID_ARG; }
    for (int k = 0; k < 3; ++k) {
        double e = k < s->dim ? s->hi[k] - s->lo[k] : 0;
        lo[k] = k < s->dim ? s->lo[k] - 0.05 * e : 0;
        hi[k] = k < s->dim ? s->hi[k] + 0.05 * e : 1;
    }
    return WOST_OK;
}
