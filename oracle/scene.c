/* Boundary geometry of the oracle -- test infrastructure.
 *
 * Brute-force queries over every primitive (no acceleration structure):
 *  - closest Dirichlet point (Sec. 3.2: epsilon-shell test and R_D),
 *  - closest Neumann silhouette (Sec. 3.2: the star radius is the smaller of
 *    the distance to the Dirichlet boundary and to the nearest silhouette),
 *  - first Neumann hit along a ray (Sec. 3.2: next point on the star boundary),
 *  - winding numbers (inside test).
 * Ties are broken by the smallest primitive index (strict comparisons while
 * scanning in index order).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

struct orc_scene {
    int dim, nverts, nprims;
    double *V;
    int32_t *P;
    uint8_t *bc;
    int g_kind, f_kind, h_kind;
    double g_par[64], f_par[256], h_par[64];
    double scale;      /* bounding-box diagonal */
    double *nin;       /* inward unit normal per primitive */
    /* silhouette elements: 2D = Neumann vertices, 3D = Neumann edges */
    int nsil;
    int32_t *sil_v;    /* 2 vertex indices (2D: the vertex twice) */
    int32_t *sil_f;    /* 2 adjacent Neumann primitives, -1 = none */
};

/* ---- small vector helpers ------------------------------------------------ */
static double dot(int d, const double *a, const double *b)
{
    double s = 0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}
static void sub(int d, const double *a, const double *b, double *o)
{
    for (int i = 0; i < d; ++i) o[i] = a[i] - b[i];
}
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm(int d, const double *a) { return sqrt(dot(d, a, a)); }
static const double *vert(const orc_scene *s, int i) { return s->V + (size_t)i * s->dim; }

/* ---- data functions ------------------------------------------------------ */
double orc_eval_fn(int kind, const double *p, int d, const double *x)
{
    switch (kind) {
    case 0: return 0.0;
    case 1: return p[0];
    case 2: return exp(p[0] * x[0]) * cos(p[0] * x[1]);
    case 3: return x[0] * x[0] - x[1] * x[1];
    case 4: return dot(d, x, x);
    case 5: {
        double r[3];
        sub(d, x, p, r);
        return 1.0 / norm(d, r);
    }
    case 6: {
        double r[3];
        sub(d, x, p, r);
        return log(norm(d, r));
    }
    case 7: {
        int n = (int)p[0];
        double sg = p[1], acc = 0;
        for (int i = 0; i < n; ++i) {
            const double *c = p + 3 + 4 * i;
            double r[3];
            sub(d, x, c, r);
            acc += p[2 + 4 * i] * exp(-dot(d, r, r) / (2 * sg * sg));
        }
        return acc;
    }
    case 8: return cosh(p[0] * x[0]) * cos(p[0] * x[1]);
    case 9: {
        /* quadratic polynomial c + b.x + sum_i a_ii x_i^2 + a_xy xy + a_xz xz + a_yz yz,
           p = [c, bx, by, bz, axx, ayy, azz, axy, axz, ayz]; z = 0 in 2D */
        double X = x[0], Y = x[1], Z = d == 3 ? x[2] : 0.0;
        return p[0] + p[1] * X + p[2] * Y + p[3] * Z + p[4] * X * X + p[5] * Y * Y + p[6] * Z * Z +
               p[7] * X * Y + p[8] * X * Z + p[9] * Y * Z;
    }
    case 10: return p[0] * atan2(x[1], x[0]) + p[1];   /* polar angle, harmonic in 2D */
    }
    return NAN;
}

/* ---- primitive distance / intersection ----------------------------------- */
static double seg_closest(const double *a, const double *b, const double *x, double *q, int d)
{
    double e[3], ax[3];
    sub(d, b, a, e);
    sub(d, x, a, ax);
    double ee = dot(d, e, e);
    double t = ee > 0 ? dot(d, ax, e) / ee : 0.0;
    if (t < 0) t = 0;
    if (t > 1) t = 1;
    double r[3];
    for (int i = 0; i < d; ++i) {
        q[i] = a[i] + t * e[i];
        r[i] = x[i] - q[i];
    }
    return norm(d, r);
}

/* closest point on triangle: the orthogonal projection when it lies inside,
   otherwise the best of the three edge segments */
static double tri_closest(const double *a, const double *b, const double *c, const double *x,
                          double *q)
{
    double e1[3], e2[3], nrm[3], ax[3];
    sub(3, b, a, e1);
    sub(3, c, a, e2);
    cross3(e1, e2, nrm);
    double nn = dot(3, nrm, nrm);
    sub(3, x, a, ax);
    if (nn > 0) {
        double h = dot(3, ax, nrm) / nn;
        double p[3];
        for (int i = 0; i < 3; ++i) p[i] = x[i] - h * nrm[i];
        /* barycentric coordinates of p via sub-triangle areas */
        double pa[3], pb[3], pc[3], c1[3], c2[3], c3[3];
        sub(3, a, p, pa);
        sub(3, b, p, pb);
        sub(3, c, p, pc);
        cross3(pb, pc, c1);
        cross3(pc, pa, c2);
        cross3(pa, pb, c3);
        double wa = dot(3, c1, nrm), wb = dot(3, c2, nrm), wc = dot(3, c3, nrm);
        if (wa >= 0 && wb >= 0 && wc >= 0) {
            memcpy(q, p, sizeof(double) * 3);
            double r[3];
            sub(3, x, p, r);
            return norm(3, r);
        }
    }
    double best = INFINITY, qq[3];
    const double *E[3][2] = {{a, b}, {b, c}, {c, a}};
    for (int k = 0; k < 3; ++k) {
        double dd = seg_closest(E[k][0], E[k][1], x, qq, 3);
        if (dd < best) {
            best = dd;
            memcpy(q, qq, sizeof(double) * 3);
        }
    }
    return best;
}

static double prim_closest(const orc_scene *s, int i, const double *x, double *q)
{
    const int32_t *p = s->P + (size_t)i * s->dim;
    if (s->dim == 2) return seg_closest(vert(s, p[0]), vert(s, p[1]), x, q, 2);
    return tri_closest(vert(s, p[0]), vert(s, p[1]), vert(s, p[2]), x, q);
}

/* ray x + t v against segment a-b (2D): t > tmin and the segment parameter in [0,1] */
static int ray_seg(const double *x, const double *v, const double *a, const double *b, double tmin, double *t)
{
    double e[2] = {b[0] - a[0], b[1] - a[1]};
    double ax[2] = {a[0] - x[0], a[1] - x[1]};
    double den = v[0] * e[1] - v[1] * e[0];
    if (den == 0) return 0;
    double tt = (ax[0] * e[1] - ax[1] * e[0]) / den;
    double ss = (ax[0] * v[1] - ax[1] * v[0]) / den;
    if (ss < 0 || ss > 1 || !(tt > tmin)) return 0;
    *t = tt;
    return 1;
}

/* ray against triangle (3D), Moeller & Trumbore (1997) */
static int ray_tri(const double *x, const double *v, const double *a, const double *b,
                   const double *c, double tmin, double *t)
{
    double e1[3], e2[3], pv[3], tv[3], qv[3];
    sub(3, b, a, e1);
    sub(3, c, a, e2);
    cross3(v, e2, pv);
    double det = dot(3, e1, pv);
    if (det == 0) return 0;
    double inv = 1.0 / det;
    sub(3, x, a, tv);
    double u = dot(3, tv, pv) * inv;
    if (u < 0 || u > 1) return 0;
    cross3(tv, e1, qv);
    double w = dot(3, v, qv) * inv;
    if (w < 0 || u + w > 1) return 0;
    double tt = dot(3, e2, qv) * inv;
    if (!(tt > tmin)) return 0;
    *t = tt;
    return 1;
}

void orc_inward_normal(const orc_scene *s, int i, double *n)
{
    memcpy(n, s->nin + (size_t)i * s->dim, sizeof(double) * s->dim);
}

/* ---- scene construction -------------------------------------------------- */
typedef struct { int32_t a, b, f; } edge_rec;
static int edge_cmp(const void *p, const void *q)
{
    const edge_rec *x = p, *y = q;
    if (x->a != y->a) return x->a < y->a ? -1 : 1;
    if (x->b != y->b) return x->b < y->b ? -1 : 1;
    return x->f < y->f ? -1 : (x->f > y->f);
}

orc_scene *orc_scene_create(int dim, int nverts, const double *V, int nprims, const int32_t *P,
                            const uint8_t *bc, int g_kind, const double *g_par, int ng,
                            int f_kind, const double *f_par, int nf, int h_kind, const double *h_par,
                            int nh)
{
    orc_scene *s = calloc(1, sizeof(orc_scene));
    s->dim = dim;
    s->nverts = nverts;
    s->nprims = nprims;
    s->V = malloc(sizeof(double) * nverts * dim);
    memcpy(s->V, V, sizeof(double) * nverts * dim);
    s->P = malloc(sizeof(int32_t) * nprims * dim);
    memcpy(s->P, P, sizeof(int32_t) * nprims * dim);
    s->bc = malloc(nprims);
    memcpy(s->bc, bc, nprims);
    s->g_kind = g_kind;
    s->f_kind = f_kind;
    s->h_kind = h_kind;
    if (ng > 64) ng = 64;
    if (nf > 256) nf = 256;
    if (nh > 64) nh = 64;
    for (int i = 0; i < ng; ++i) s->g_par[i] = g_par[i];
    for (int i = 0; i < nf; ++i) s->f_par[i] = f_par[i];
    for (int i = 0; i < nh; ++i) s->h_par[i] = h_par[i];

    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = 0; i < nverts; ++i)
        for (int k = 0; k < dim; ++k) {
            double c = V[(size_t)i * dim + k];
            if (c < lo[k]) lo[k] = c;
            if (c > hi[k]) hi[k] = c;
        }
    double dg[3];
    sub(dim, hi, lo, dg);
    s->scale = norm(dim, dg);

    /* inward normals: 2D segment a->b with the domain on its left has inward
       normal = left perpendicular of (b - a); 3D triangles wind
       counter-clockwise seen from outside, so inward = -(e1 x e2) */
    s->nin = malloc(sizeof(double) * nprims * dim);
    for (int i = 0; i < nprims; ++i) {
        const int32_t *p = P + (size_t)i * dim;
        double *n = s->nin + (size_t)i * dim;
        if (dim == 2) {
            const double *a = vert(s, p[0]), *b = vert(s, p[1]);
            double e[2] = {b[0] - a[0], b[1] - a[1]};
            double L = norm(2, e);
            n[0] = -e[1] / L;
            n[1] = e[0] / L;
        } else {
            double e1[3], e2[3], c[3];
            sub(3, vert(s, p[1]), vert(s, p[0]), e1);
            sub(3, vert(s, p[2]), vert(s, p[0]), e2);
            cross3(e1, e2, c);
            double L = norm(3, c);
            for (int k = 0; k < 3; ++k) n[k] = -c[k] / L;
        }
    }

    /* silhouette elements */
    if (dim == 2) {
        int32_t *in_seg = malloc(sizeof(int32_t) * nverts), *out_seg = malloc(sizeof(int32_t) * nverts);
        for (int i = 0; i < nverts; ++i) in_seg[i] = out_seg[i] = -1;
        for (int i = 0; i < nprims; ++i)
            if (bc[i] == 1) {
                out_seg[P[2 * i]] = i;      /* segment leaves its first vertex */
                in_seg[P[2 * i + 1]] = i;   /* and arrives at its second */
            }
        s->sil_v = malloc(sizeof(int32_t) * 2 * nverts);
        s->sil_f = malloc(sizeof(int32_t) * 2 * nverts);
        s->nsil = 0;
        for (int v = 0; v < nverts; ++v)
            if (in_seg[v] >= 0 || out_seg[v] >= 0) {
                s->sil_v[2 * s->nsil] = s->sil_v[2 * s->nsil + 1] = v;
                s->sil_f[2 * s->nsil] = in_seg[v];
                s->sil_f[2 * s->nsil + 1] = out_seg[v];
                s->nsil++;
            }
        free(in_seg);
        free(out_seg);
    } else {
        int nn = 0;
        for (int i = 0; i < nprims; ++i) nn += bc[i] == 1;
        edge_rec *E = malloc(sizeof(edge_rec) * 3 * (nn + 1));
        int ne = 0;
        for (int i = 0; i < nprims; ++i)
            if (bc[i] == 1)
                for (int k = 0; k < 3; ++k) {
                    int32_t a = P[3 * i + k], b = P[3 * i + (k + 1) % 3];
                    E[ne].a = a < b ? a : b;
                    E[ne].b = a < b ? b : a;
                    E[ne].f = i;
                    ne++;
                }
        qsort(E, ne, sizeof(edge_rec), edge_cmp);
        s->sil_v = malloc(sizeof(int32_t) * 2 * (ne + 1));
        s->sil_f = malloc(sizeof(int32_t) * 2 * (ne + 1));
        s->nsil = 0;
        for (int i = 0; i < ne;) {
            int j = i;
            while (j < ne && E[j].a == E[i].a && E[j].b == E[i].b) ++j;
            int cnt = j - i;
            s->sil_v[2 * s->nsil] = E[i].a;
            s->sil_v[2 * s->nsil + 1] = E[i].b;
            /* exactly two Neumann faces: interior edge, tested per query;
               otherwise (border of the Neumann set, non-manifold) always a silhouette */
            s->sil_f[2 * s->nsil] = cnt == 2 ? E[i].f : -1;
            s->sil_f[2 * s->nsil + 1] = cnt == 2 ? E[i + 1].f : -1;
            s->nsil++;
            i = j;
        }
        free(E);
    }
    return s;
}

void orc_scene_free(orc_scene *s)
{
    if (!s) return;
    free(s->V); free(s->P); free(s->bc); free(s->nin); free(s->sil_v); free(s->sil_f);
    free(s);
}

int orc_scene_nsil(const orc_scene *s) { return s->nsil; }
double orc_scene_scale(const orc_scene *s) { return s->scale; }

/* ---- queries -------------------------------------------------------------- */
int orc_closest_dirichlet(const orc_scene *s, const double *x, double *dist, double *xbar)
{
    int best = -1;
    double bd = INFINITY, q[3];
    for (int i = 0; i < s->nprims; ++i) {
        if (s->bc[i] != 0) continue;
        double dd = prim_closest(s, i, x, q);
        if (dd < bd) {
            bd = dd;
            best = i;
            if (xbar) memcpy(xbar, q, sizeof(double) * s->dim);
        }
    }
    *dist = bd;
    return best;
}

/* Silhouette classification.  o = signed distance of x to the supporting
   line/plane of an adjacent Neumann primitive, positive on the domain side.
   With tolerance tau: front (o > tau), back (o < -tau), on (|o| <= tau).
   The shared vertex/edge is a silhouette when one neighbour is seen from the
   back and the other from the front or edge-on (x on its plane). */
static int is_silhouette(const orc_scene *s, int e, const double *x)
{
    int f0 = s->sil_f[2 * e], f1 = s->sil_f[2 * e + 1];
    if (f0 < 0 || f1 < 0) return 1;
    const double *p = vert(s, s->sil_v[2 * e]);
    double r[3];
    sub(s->dim, x, p, r);
    double o0 = dot(s->dim, s->nin + (size_t)f0 * s->dim, r);
    double o1 = dot(s->dim, s->nin + (size_t)f1 * s->dim, r);
    double tau = 1e-6 * s->scale;
    int c0 = o0 > tau ? 1 : (o0 < -tau ? -1 : 0);
    int c1 = o1 > tau ? 1 : (o1 < -tau ? -1 : 0);
    return (c0 == -1 && c1 >= 0) || (c1 == -1 && c0 >= 0);
}

int orc_closest_silhouette(const orc_scene *s, const double *x, double *dist)
{
    int best = -1;
    double bd = INFINITY, q[3];
    for (int e = 0; e < s->nsil; ++e) {
        if (!is_silhouette(s, e, x)) continue;
        const double *a = vert(s, s->sil_v[2 * e]), *b = vert(s, s->sil_v[2 * e + 1]);
        double dd = seg_closest(a, b, x, q, s->dim);
        if (dd < bd) {
            bd = dd;
            best = e;
        }
    }
    *dist = bd;
    return best;
}

static int ray_neumann(const orc_scene *s, const double *x, const double *v, double tmax, int skip,
                       int exit_only, double *t)
{
    /* exit casts: rounding band of a position, 16 units of 2^-24 of the
       scene scale */
    const double band = 16.0 * ldexp(1.0, -24) * s->scale;
    const int d = s->dim;
    int best = -1;
    double bt = INFINITY;
    for (int i = 0; i < s->nprims; ++i) {
        if (s->bc[i] != 1 || i == skip) continue;
        const int32_t *p = s->P + (size_t)i * d;
        double tt;
        int hit;
        if (exit_only) {
            /* the ray leaves the domain through primitive i iff it points
               against the inward normal and crosses the primitive's line /
               plane at t > -band within distance band of the primitive (a
               walk standing within rounding of a vertex that heads out
               through the next primitive crosses it at t ~ 0) */
            double ng[3], am[3], q[3], qc[3];
            orc_inward_normal(s, i, ng);
            double vn = dot(d, v, ng);
            if (!(vn < 0)) continue;
            sub(d, vert(s, p[0]), x, am);
            tt = dot(d, am, ng) / vn;
            if (!(tt > -band)) continue;
            for (int k = 0; k < d; ++k) q[k] = x[k] + tt * v[k];
            hit = prim_closest(s, i, q, qc) <= band;
        } else {
            hit = d == 2 ? ray_seg(x, v, vert(s, p[0]), vert(s, p[1]), 0.0, &tt)
                         : ray_tri(x, v, vert(s, p[0]), vert(s, p[1]), vert(s, p[2]), 0.0, &tt);
        }
        if (hit && tt <= tmax && tt < bt) {
            bt = tt;
            best = i;
        }
    }
    *t = bt;
    return best;
}

int orc_ray_neumann(const orc_scene *s, const double *x, const double *v, double tmax, int skip,
                    double *t)
{
    return ray_neumann(s, x, v, tmax, skip, 0, t);
}

int orc_ray_neumann_exit(const orc_scene *s, const double *x, const double *v, double tmax, int skip,
                         double *t)
{
    return ray_neumann(s, x, v, tmax, skip, 1, t);
}

double orc_winding(const orc_scene *s, const double *x)
{
    double acc = 0;
    for (int i = 0; i < s->nprims; ++i) {
        const int32_t *p = s->P + (size_t)i * s->dim;
        if (s->dim == 2) {
            double a[2], b[2];
            sub(2, vert(s, p[0]), x, a);
            sub(2, vert(s, p[1]), x, b);
            acc += atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1]);
        } else {
            /* solid angle of a triangle, Van Oosterom & Strackee (1983) */
            double A[3], B[3], C[3], bc[3];
            sub(3, vert(s, p[0]), x, A);
            sub(3, vert(s, p[1]), x, B);
            sub(3, vert(s, p[2]), x, C);
            cross3(B, C, bc);
            double la = norm(3, A), lb = norm(3, B), lc = norm(3, C);
            double num = dot(3, A, bc);
            double den = la * lb * lc + dot(3, A, B) * lc + dot(3, A, C) * lb + dot(3, B, C) * la;
            acc += 2 * atan2(num, den);
        }
    }
    return acc / (s->dim == 2 ? 2 * M_PI : 4 * M_PI);
}

int orc_point_status(const orc_scene *s, const double *x, double eps, double *value)
{
    if (orc_winding(s, x) < 0.5) {
        *value = NAN;
        return 2;
    }
    double d, xb[3];
    orc_closest_dirichlet(s, x, &d, xb);
    if (d <= eps) {
        *value = orc_eval_fn(s->g_kind, s->g_par, s->dim, xb);
        return 1;
    }
    *value = 0;
    return 0;
}

/* ---- Neumann boundary sample of <N> (Sec. 3.2, Eq. wost_estm) ----------------
   Every Neumann primitive closer to x than r is a candidate, with weight its
   length (2D) or area (3D).  One candidate is chosen with probability
   weight / W, W the summed weight, by the smallest key -log(u_i) / w_i with
   u_i in (0, 1] drawn for the primitive itself (Philox counter (point, walk,
   step, 2^31 | primitive id)): the choice depends on the candidate set only,
   not on the order the candidates are visited in (Efraimidis & Spirakis
   2006, weighted sampling with keys).  The point z is uniform on the chosen
   primitive (counter purpose 96), so its density is 1 / W.  Returns the
   chosen primitive (-1 when there is no candidate), z and W. */
static double prim_size(const orc_scene *s, int i)
{
    const int32_t *p = s->P + (size_t)i * s->dim;
    double e1[3], e2[3], c[3];
    sub(s->dim, vert(s, p[1]), vert(s, p[0]), e1);
    if (s->dim == 2) return norm(2, e1);
    sub(3, vert(s, p[2]), vert(s, p[0]), e2);
    cross3(e1, e2, c);
    return 0.5 * norm(3, c);
}

int orc_neumann_sample(const orc_scene *s, const double *x, double r, const uint32_t key[2], uint32_t pid,
                       uint32_t wid, uint32_t step, double *z, double *W)
{
    int best = -1;
    double best_key = INFINITY, total = 0, q[3];
    for (int i = 0; i < s->nprims; ++i) {
        if (s->bc[i] != 1) continue;
        if (!(prim_closest(s, i, x, q) < r)) continue;
        double w = prim_size(s, i);
        uint32_t ctr[4] = {pid, wid, step, 0x80000000u | (uint32_t)i}, o[4];
        orc_philox4x32_10(ctr, key, o);
        double u = ((double)(o[0] >> 8) + 1.0) * ldexp(1.0, -24);     /* (0, 1] */
        double k = -log(u) / w;
        total += w;
        if (k < best_key) {
            best_key = k;
            best = i;
        }
    }
    *W = total;
    if (best < 0) return -1;
    uint32_t ctr[4] = {pid, wid, step, 96u}, o[4];
    orc_philox4x32_10(ctr, key, o);
    double u0 = orc_u01(o[0]), u1 = orc_u01(o[1]);
    const int32_t *p = s->P + (size_t)best * s->dim;
    if (s->dim == 2) {
        for (int k = 0; k < 2; ++k) z[k] = (1 - u0) * vert(s, p[0])[k] + u0 * vert(s, p[1])[k];
    } else {
        /* uniform on a triangle: barycentrics (1 - sqrt u0, sqrt u0 (1 - u1), sqrt u0 u1) */
        double su = sqrt(u0);
        for (int k = 0; k < 3; ++k)
            z[k] = (1 - su) * vert(s, p[0])[k] + su * (1 - u1) * vert(s, p[1])[k] + su * u1 * vert(s, p[2])[k];
    }
    return best;
}

/* accessors used by the walk */
int orc__scene_dim(const orc_scene *s) { return s->dim; }
int orc__scene_fkind(const orc_scene *s) { return s->f_kind; }
int orc__scene_hkind(const orc_scene *s) { return s->h_kind; }
double orc__eval_h(const orc_scene *s, const double *x) { return orc_eval_fn(s->h_kind, s->h_par, s->dim, x); }
double orc__eval_g(const orc_scene *s, const double *x) { return orc_eval_fn(s->g_kind, s->g_par, s->dim, x); }
double orc__eval_f(const orc_scene *s, const double *x) { return orc_eval_fn(s->f_kind, s->f_par, s->dim, x); }
