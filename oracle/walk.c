/* Walk on stars with guided direction sampling -- oracle (test infrastructure).
 *
 * One walk follows the single-sample estimator of Sec. 3.2 (Eq. wost_estm) in
 * the reparameterised form of Sec. 4.1:
 *   <u(x_k)> = <u(nu; x_k)> / (|S^{d-1}| alpha(x_k) p(nu | x_k)) - <N> + <S>
 * with
 *   - termination in the epsilon-shell of the Dirichlet boundary, value g at
 *     the closest Dirichlet point (Sec. 3.2);
 *   - star radius r = max(min(R_D, R_S), eps) (Sec. 3.2; the floor eps is a
 *     reading: the paper states no lower bound);
 *   - source term <S> = -(r^2 / 2d) f(y): y drawn with density proportional
 *     to the ball's Green function (radius r sqrt(U1 U2) in 2D, r Beta(2,2)
 *     in 3D), counted only when visible from x_k (y in St).  The sign follows
 *     Laplacian u = f with G >= 0 the Green function of -Laplacian (a reading,
 *     pinned by manufactured solutions); alpha = 1/2 cancels against the
 *     hemisphere density on Neumann points;
 *   - Neumann contribution <N> = G(x, z) h(z) / (alpha p(z)), entering with a
 *     minus sign as printed: with G >= 0 (the reading above) and h the
 *     derivative along the normal that points into the domain (the paper's
 *     normal convention, Sec. 4.1 footnote), Green's second identity on the
 *     star St gives alpha u(x) = int P u - int_{dSt_N} G h - int_St G f.
 *     z is drawn on the Neumann boundary inside B(x, r) with density 1 / W
 *     (orc_neumann_sample); it lies on dSt_N when it faces x: inside B there
 *     is no silhouette, so no Neumann point there is hidden from x.
 *     G(x, z) = ln(r / |z - x|) / 2 pi (2D), (1/|z - x| - 1/r) / 4 pi (3D);
 *   - direction: uniform (Sec. 4.1 Eq. for p_u) or, when guided, one-sample
 *     MIS between the vMF mixture decoded by the neural field and uniform
 *     with selection probability c(x) (Sec. 4.4 Eq. mis_pdf); on a Neumann
 *     point directions below the tangent plane are reflected (Sec. 4.3), the
 *     guided density there being V(nu) + V(nu^-);
 *   - the next point is the first Neumann hit within r, else x + r nu; the
 *     normal at a Neumann point faces the side the walk arrived from
 *     (Sec. 4.1 footnote);
 *   - Russian roulette once the walk is long (Sec. 6.1 enables it only beyond
 *     128 steps and states no survival rule; the reading here): from step
 *     rr_depth on, after the epsilon-shell test, the walk goes on with
 *     probability q = rr_survival (purpose-97 draw) and its throughput is
 *     divided by q, else it ends with recursive value 0 -- an unbiased
 *     estimator of the step's u(x_k).  For the suffix pass that step's weight
 *     and non-recursive terms carry the same 1/q;
 *   - a hard cap of `maxsteps` moves, after which the walk is closed with g at
 *     the current closest Dirichlet point (counted as truncated; with
 *     roulette on, a safety net only).
 * Random numbers: Philox4x32-10 with key (seed_lo, seed_hi + scene_id) and
 * counter (point, walk, step, purpose); purpose 0 MIS choice / lobe / 3D vMF,
 * 1 uniform direction, 2 source direction and radius, 3.. 2D vMF retries.
 */
#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

int orc__scene_dim(const orc_scene *s);
int orc__scene_fkind(const orc_scene *s);
int orc__scene_hkind(const orc_scene *s);
double orc__eval_h(const orc_scene *s, const double *x);
double orc__eval_g(const orc_scene *s, const double *x);
double orc__eval_f(const orc_scene *s, const double *x);

static double sphere_area(int d) { return d == 2 ? 2 * M_PI : 4 * M_PI; }

static void draw(const uint32_t key[2], uint32_t pid, uint32_t wid, uint32_t step,
                 uint32_t purpose, double u[4])
{
    uint32_t ctr[4] = {pid, wid, step, purpose}, o[4];
    orc_philox4x32_10(ctr, key, o);
    for (int i = 0; i < 4; ++i) u[i] = orc_u01(o[i]);
}

static void uniform_dir(int d, double u0, double u1, double *v)
{
    if (d == 2) {
        double th = 2 * M_PI * u0;
        v[0] = cos(th);
        v[1] = sin(th);
    } else {
        double z = 1 - 2 * u0, ph = 2 * M_PI * u1;
        double s = sqrt(fmax(0.0, 1 - z * z));
        v[0] = s * cos(ph);
        v[1] = s * sin(ph);
        v[2] = z;
    }
}

static double vdot(int d, const double *a, const double *b)
{
    double s = 0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

static void reflect(int d, const double *v, const double *n, double *o)
{
    double t = vdot(d, v, n);
    for (int i = 0; i < d; ++i) o[i] = v[i] - 2 * t * n[i];
}

/* Beta(2,2) by inversion of F(s) = 3 s^2 - 2 s^3 (trigonometric root) */
static double beta22_inv(double u)
{
    return 0.5 + cos((acos(1 - 2 * u) + 4 * M_PI) / 3);
}

/* One-sample MIS direction (Sec. 4.4): with probability c (purpose-0 draw
   u0) pick a lobe by the lambda-CDF (u1) and sample it (2D Best-Fisher with
   purposes 3.., 3D from u2, u3); returns 1 and the direction if the mixture
   was chosen, 0 (nu untouched) for the uniform branch. */
int orc_guided_draw(int d, int K, const double *mu, const double *kap, const double *lam, double c,
                    const uint32_t key[2], uint32_t pid, uint32_t wid, uint32_t step, double *nu)
{
    double u[4];
    draw(key, pid, wid, step, 0, u);
    if (!(u[0] < c)) return 0;
    int lobe = K - 1;
    double cdf = 0;
    for (int i = 0; i < K; ++i) {
        cdf += lam[i];
        if (u[1] < cdf) {
            lobe = i;
            break;
        }
    }
    const double *m = mu + lobe * d;
    if (d == 2) {
        double th = orc_vmf2_sample_angle(kap[lobe], key, pid, wid, step, NULL);
        nu[0] = m[0] * cos(th) - m[1] * sin(th);
        nu[1] = m[0] * sin(th) + m[1] * cos(th);
    } else {
        orc_vmf3_sample(kap[lobe], m, u[2], u[3], nu);
    }
    return 1;
}

typedef struct { double w, S; } step_info;

double orc_walk(const orc_scene *s, const orc_field *fld, const orc_params *p, uint32_t pid,
                uint32_t wid, const double *x0, int *steps, int *truncated, double *recs,
                int max_recs, int *nrec)
{
    return orc_walk_terms(s, fld, p, pid, wid, x0, steps, truncated, recs, max_recs, nrec, NULL);
}

double orc_walk_terms(const orc_scene *s, const orc_field *fld, const orc_params *p, uint32_t pid,
                      uint32_t wid, const double *x0, int *steps, int *truncated, double *recs,
                      int max_recs, int *nrec, double *terms)
{
    const int d = orc__scene_dim(s);
    const int K = fld ? fld->K : 0;
    const int has_src = orc__scene_fkind(s) != 0;
    const int has_flux = orc__scene_hkind(s) != 0;
    const uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32) + p->scene_id};
    const double area = sphere_area(d);
    double x[3] = {0, 0, 0}, n[3] = {0, 0, 0};
    memcpy(x, x0, sizeof(double) * d);
    double T = 1, acc = 0, term = 0;
    int on_neu = 0, prim = -1, k, trunc = 0, nr = 0;
    step_info *info = recs ? malloc(sizeof(step_info) * (p->maxsteps + 1)) : NULL;

    for (k = 0;; ++k) {
        double RD, xbar[3];
        orc_closest_dirichlet(s, x, &RD, xbar);
        if (RD <= p->eps || k == p->maxsteps) {
            term = orc__eval_g(s, xbar);
            acc += T * term;
            trunc = RD > p->eps;
            break;
        }
        /* Russian roulette */
        double rr = 1.0;
        if (p->rr_depth > 0 && k >= p->rr_depth) {
            double u[4];
            draw(key, pid, wid, (uint32_t)k, 97, u);
            if (!(u[0] < p->rr_survival)) {
                term = 0;
                break;
            }
            rr = 1.0 / p->rr_survival;
            T *= rr;
        }
        double RS;
        orc_closest_silhouette(s, x, &RS);
        double r = fmax(fmin(RD, RS), p->eps);

        /* source contribution */
        double S = 0;
        if (has_src) {
            double u[4], vs[3], t;
            draw(key, pid, wid, (uint32_t)k, 2, u);
            uniform_dir(d, u[0], u[1], vs);
            if (on_neu && vdot(d, vs, n) < 0) reflect(d, vs, n, vs);
            double rho = d == 2 ? r * sqrt(u[2] * u[3]) : r * beta22_inv(u[2]);
            if (orc_ray_neumann_exit(s, x, vs, rho, on_neu ? prim : -1, &t) < 0) {
                double y[3];
                for (int i = 0; i < d; ++i) y[i] = x[i] + rho * vs[i];
                S = -(r * r / (2.0 * d)) * orc__eval_f(s, y);
            }
            acc += T * S;
        }

        /* Neumann contribution -<N> */
        if (has_flux) {
            double z[3], W, Nt = 0;
            int j = orc_neumann_sample(s, x, r, key, pid, wid, (uint32_t)k, z, &W);
            if (j >= 0) {
                double dz[3], nz[3];
                for (int i = 0; i < d; ++i) dz[i] = z[i] - x[i];
                double dd = sqrt(vdot(d, dz, dz));
                orc_inward_normal(s, j, nz);
                if (dd > 0 && dd < r && vdot(d, dz, nz) < 0) {
                    double G = d == 2 ? log(r / dd) / (2 * M_PI) : (1 / dd - 1 / r) / (4 * M_PI);
                    Nt = G * orc__eval_h(s, z) * W / (on_neu ? 0.5 : 1.0);
                }
            }
            S -= Nt;
            acc -= T * Nt;
        }

        /* direction */
        double nu[3] = {0, 0, 0}, c = 0, mu[3 * 32], kap[32], lam[32];
        int from_guide = 0;
        if (p->guided) {
            double raw[256];
            orc_field_forward(fld, x, raw);
            orc_theta_map(fld, raw, mu, kap, lam, &c);
            if (p->c_mode == 1) c = p->c_fixed;
            from_guide = orc_guided_draw(d, K, mu, kap, lam, c, key, pid, wid, (uint32_t)k, nu);
        }
        if (!from_guide) {
            double u[4];
            draw(key, pid, wid, (uint32_t)k, 1, u);
            uniform_dir(d, u[0], u[1], nu);
        }
        double dn = on_neu ? vdot(d, nu, n) : 1;
        if (on_neu && dn < 0 && (p->reflect || !from_guide)) {
            reflect(d, nu, n, nu);
            dn = -dn;
        }
        if (on_neu && dn <= 0) {
            /* zero density (Eq. angular_req): the recursive term is 0 and
               the walk's last value is this step's source term */
            term = S * rr;
            break;
        }

        /* densities and the step weight 1 / (|S| alpha p~) */
        double alpha = on_neu ? 0.5 : 1.0;
        double pu = (on_neu ? 2.0 : 1.0) / area;
        double pg = 0, ptil = pu, w = 1;
        if (p->guided) {
            pg = orc_mixture_pdf(d, K, mu, kap, lam, nu);
            if (on_neu && p->reflect) {
                double nm[3];
                reflect(d, nu, n, nm);
                pg += orc_mixture_pdf(d, K, mu, kap, lam, nm);
            }
            ptil = c * pg + (1 - c) * pu;
            /* |S| alpha p_u == 1 exactly, so c = 0 reproduces plain WoSt */
            w = 1.0 / (c * area * alpha * pg + (1 - c));
        }
        if (recs && nr < max_recs) {
            double *R = recs + (size_t)nr * ORC_REC;
            memset(R, 0, sizeof(double) * ORC_REC);
            memcpy(R, x, sizeof(double) * d);
            memcpy(R + 3, nu, sizeof(double) * d);
            if (on_neu) memcpy(R + 6, n, sizeof(double) * d);
            R[9] = on_neu;
            R[10] = ptil;
            info[nr].w = w * rr;
            info[nr].S = S * rr;
            nr++;
        }
        T *= w;

        /* next point on the star boundary */
        double t;
        int hit = orc_ray_neumann_exit(s, x, nu, r, on_neu ? prim : -1, &t);
        if (hit >= 0) {
            /* the walk stands at the hit point moved 16 * 2^-24 * scale along
               the primitive's inward normal, strictly inside the domain */
            const double band = 16.0 * ldexp(1.0, -24) * orc_scene_scale(s);
            t = fmax(t, 0.0);
            orc_inward_normal(s, hit, n);
            for (int i = 0; i < d; ++i) x[i] += t * nu[i] + band * n[i];
            on_neu = 1;
            prim = hit;
        } else {
            for (int i = 0; i < d; ++i) x[i] += r * nu[i];
            on_neu = 0;
            prim = -1;
        }
    }
    if (info) {
        if (terms) {
            for (int i = 0; i < nr; ++i) {
                terms[2 * i] = info[i].w;
                terms[2 * i + 1] = info[i].S;
            }
            terms[2 * nr] = term;
        }
        /* suffix pass: v_n = terminal value, v_k = w_k v_{k+1} + S_k;
           target of record k is |v_{k+1}| (Sec. 4.1 Eq. guiding_dist) */
        double v = term;
        for (int i = nr - 1; i >= 0; --i) {
            recs[(size_t)i * ORC_REC + 11] = fabs(v);
            v = info[i].w * v + info[i].S;
        }
        free(info);
    }
    if (nrec) *nrec = nr;
    if (steps) *steps = k + 1;
    if (truncated) *truncated = trunc;
    return acc;
}

/* ---- threaded driver ------------------------------------------------------ */
typedef struct {
    const orc_scene *s;
    const orc_field *fld;
    const orc_params *p;
    const double *points;
    int npoints, walk_begin, nwalks, tid, nth;
    double *sum, *sum2, *recs;
    int *nrec;
    int64_t steps, trunc;
} job_t;

static void *worker(void *arg)
{
    job_t *j = arg;
    int d = orc__scene_dim(j->s);
    for (int i = j->tid; i < j->npoints; i += j->nth) {
        double s1 = 0, s2 = 0;
        for (int w = 0; w < j->nwalks; ++w) {
            int st, tr, nr = 0;
            int first = (w == 0) && j->recs;
            double v = orc_walk(j->s, j->fld, j->p, (uint32_t)i, (uint32_t)(j->walk_begin + w),
                                j->points + (size_t)i * d, &st, &tr,
                                first ? j->recs + (size_t)i * j->p->maxsteps * ORC_REC : NULL,
                                j->p->maxsteps, &nr);
            if (first && j->nrec) j->nrec[i] = nr;
            s1 += v;
            s2 += v * v;
            j->steps += st;
            j->trunc += tr;
        }
        j->sum[i] += s1;
        j->sum2[i] += s2;
    }
    return NULL;
}

void orc_solve(const orc_scene *s, const orc_field *fld, const orc_params *p,
               const double *points, int npoints, int walk_begin, int nwalks, double *sum,
               double *sum2, int64_t *steps, int64_t *truncated, double *recs, int *nrec)
{
    int nth = p->nthreads > 0 ? p->nthreads : 1;
    pthread_t *th = malloc(sizeof(pthread_t) * nth);
    job_t *jobs = calloc(nth, sizeof(job_t));
    for (int t = 0; t < nth; ++t) {
        jobs[t] = (job_t){s, fld, p, points, npoints, walk_begin, nwalks, t, nth,
                          sum, sum2, recs, nrec, 0, 0};
        pthread_create(&th[t], NULL, worker, &jobs[t]);
    }
    int64_t st = 0, tr = 0;
    for (int t = 0; t < nth; ++t) {
        pthread_join(th[t], NULL);
        st += jobs[t].steps;
        tr += jobs[t].trunc;
    }
    if (steps) *steps += st;
    if (truncated) *truncated += tr;
    free(th);
    free(jobs);
}
