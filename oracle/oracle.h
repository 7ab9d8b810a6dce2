/*
 * CPU FP64 oracle for guided walk on stars -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, deliberately unoptimised restatement of the method of
 * "Guiding-Based Importance Sampling for Walk on Stars" (arXiv 2410.18944),
 * used to check the CUDA implementation.  Only the test-suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it; the product path
 * never does.  It shares no code, header or constant table with the CUDA
 * library: every function below is written independently from the paper
 * (and, where the paper defers, from the published methods it cites).
 *
 * Geometry is brute force (every primitive is tested for every query), all
 * arithmetic is double precision, random numbers come from Philox4x32-10.
 *
 * Pins (see tests/test_oracle_*.py): closed-form harmonic solutions,
 * manufactured Poisson solutions, brute-force geometric identities,
 * quadrature of the vMF densities, sampler histograms/moments, Philox
 * known-answer vectors, finite differences of the training loss.  The
 * learned-field trajectory of online training is "parity unpinned"
 * (it depends on floating-point order); the loss gradient itself is pinned.
 */
#ifndef WOST_ORACLE_H
#define WOST_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- Philox4x32-10 (Salmon et al., SC'11) ------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* 24-bit uniform in [0,1): (u >> 8) * 2^-24 */
double orc_u01(uint32_t u);

/* ---- scene -------------------------------------------------------------- */
typedef struct orc_scene orc_scene;
orc_scene *orc_scene_create(int dim, int nverts, const double *V, int nprims, const int32_t *P,
                            const uint8_t *bc, int g_kind, const double *g_par, int ng,
                            int f_kind, const double *f_par, int nf, int h_kind, const double *h_par,
                            int nh);
void orc_scene_free(orc_scene *s);
int orc_scene_nsil(const orc_scene *s);
double orc_scene_scale(const orc_scene *s);

/* data functions (kind codes of the input descriptors) */
double orc_eval_fn(int kind, const double *par, int dim, const double *x);

/* closest Dirichlet primitive (Sec. 3.2 epsilon-shell / star radius):
   returns its index (smallest on ties) or -1, distance and closest point. */
int orc_closest_dirichlet(const orc_scene *s, const double *x, double *dist, double *xbar);
/* closest silhouette element of the Neumann boundary seen from x (Sec. 3.2):
   returns its index or -1 and the distance (+inf when none). */
int orc_closest_silhouette(const orc_scene *s, const double *x, double *dist);
/* first Neumann primitive hit by x + t v, 0 < t <= tmax, skipping `skip`. */
int orc_ray_neumann(const orc_scene *s, const double *x, const double *v, double tmax, int skip,
                    double *t);
/* the same, counting only primitives the ray leaves the domain through
   (v . inward normal < 0), whose line / plane it crosses at t > -band within
   distance band of the primitive, band = 16 * 2^-24 * scale (a walk
   standing within rounding of a vertex that heads out through the next
   primitive crosses it at t ~ 0; the walk moves by max(t, 0)).  The walks cast these:
   inside a closed boundary the first crossing is an exit, and the normal of
   the walker's new position is then the primitive's inward normal -- the
   side the walk is on (Sec. 4.1, normal convention at Eq. angular_req). */
int orc_ray_neumann_exit(const orc_scene *s, const double *x, const double *v, double tmax, int skip,
                         double *t);
/* sample of the Neumann boundary inside the ball B(x, r) for <N> (Sec. 3.2,
   Eq. wost_estm): returns the chosen Neumann primitive (-1 if none is closer
   than r), the point z (uniform on it; density 1 / W) and W, the summed
   length / area of the Neumann primitives closer than r */
int orc_neumann_sample(const orc_scene *s, const double *x, double r, const uint32_t key[2], uint32_t pid,
                       uint32_t wid, uint32_t step, double *z, double *W);
/* winding number (2D) / generalised winding number (3D) */
double orc_winding(const orc_scene *s, const double *x);
/* inward unit normal of a primitive */
void orc_inward_normal(const orc_scene *s, int prim, double *n);

/* ---- von Mises-Fisher (Sec. 3.3) ---------------------------------------- */
double orc_i0e(double x);
double orc_i1e(double x);
double orc_vmf_pdf(int dim, double kappa, const double *mu, const double *nu);
double orc_vmf_mean_cos(int dim, double kappa);     /* A_d(kappa) = E[mu . nu] */
/* 2D Best-Fisher rejection sampler; draws come from Philox purposes 3.. */
double orc_vmf2_sample_angle(double kappa, const uint32_t key[2], uint32_t pid, uint32_t wid,
                             uint32_t step, int *ntries);
void orc_vmf3_sample(double kappa, const double *mu, double xi, double xi2, double *nu);
void orc_onb(const double *n, double *b1, double *b2);

/* ---- neural field (Sec. 5.2) -------------------------------------------- */
typedef struct {
    int dim, K, L, log2T, F, H;     /* lobes, levels, table log2, features, hidden width */
    int base_res, max_res;
    double lo[3], hi[3];            /* padded scene box mapped to [0,1]^d */
    const double *grid;             /* L x 2^log2T x F */
    const double *W1;               /* H x (L F) */
    const double *W2;               /* H x H */
    const double *W3;               /* nout x H, nout = (dim + 2) K + 1 */
    const double *b3;               /* nout */
    int grid_type;                  /* 0 hash grid (grid: L x 2^log2T x F), 1 dense grid
                                       (every level dense, level l at entry offset
                                       sum_{j<l} (N_j + 1)^d; grid: entries x F) */
} orc_field;
/* lattice entries of all levels (L 2^log2T for the hash grid) */
int64_t orc_field_entries(const orc_field *f);
int orc_field_nout(const orc_field *f);
int orc_level_res(const orc_field *f, int level);
void orc_field_encode(const orc_field *f, const double *x, double *feat);
void orc_field_forward(const orc_field *f, const double *x, double *raw);
/* normalisation map of Tab. "reg_map": raw -> mu (K x d), kappa, lambda, c */
void orc_theta_map(const orc_field *f, const double *raw, double *mu, double *kappa,
                   double *lambda, double *c);
double orc_mixture_pdf(int dim, int K, const double *mu, const double *kappa,
                       const double *lambda, const double *nu);

/* ---- walk on stars (Sec. 3.2, 4.1-4.4) ---------------------------------- */
typedef struct {
    double eps;          /* epsilon-shell width */
    int maxsteps;        /* hard cap on steps */
    int guided;          /* 0 plain WoSt, 1 guided */
    int c_mode;          /* 0 learned c = sigmoid(c'), 1 fixed c = c_fixed */
    double c_fixed;
    int reflect;         /* 1 sample reflection at Neumann (Sec. 4.3), 0 ablation */
    uint64_t seed;
    uint32_t scene_id;
    int nthreads;
    int rr_depth;        /* Russian roulette from this step on (0 = off) */
    double rr_survival;  /* survival probability of a roulette step */
} orc_params;

/* training record exchange layout: 12 doubles
   x[3], nu[3], n[3], on_neumann, q (sampling pdf p~), target p_t */
#define ORC_REC 12

/* guided direction draw of one step (purpose-0 Philox draw, lobe pick,
   vMF sample); returns 1 if the mixture branch was taken */
int orc_guided_draw(int dim, int K, const double *mu, const double *kappa, const double *lambda, double c,
                    const uint32_t key[2], uint32_t pid, uint32_t wid, uint32_t step, double *nu);

/* status of a query point: 0 walk, 1 inside the epsilon-shell (value = g),
   2 outside the domain (value = NaN) */
int orc_point_status(const orc_scene *s, const double *x, double eps, double *value);

/* one walk; returns its estimate.  recs (nullable) receives up to max_recs
   training records with targets filled by the suffix pass. */
double orc_walk(const orc_scene *s, const orc_field *fld, const orc_params *p, uint32_t pid,
                uint32_t wid, const double *x0, int *steps, int *truncated, double *recs,
                int max_recs, int *nrec);

/* orc_walk, and with recs: terms (nullable, 2 * max_recs + 1 doubles) receives
   the suffix-pass inputs of each record k, its step weight w_k and source
   term S_k at [2k], [2k + 1], and the walk's last value v_n at [2 nrec]. */
double orc_walk_terms(const orc_scene *s, const orc_field *fld, const orc_params *p, uint32_t pid,
                      uint32_t wid, const double *x0, int *steps, int *truncated, double *recs,
                      int max_recs, int *nrec, double *terms);

/* walks [walk_begin, walk_begin + nwalks) of every point (threads over points).
   Adds to sum/sum2 (per point), counts walk-steps and truncated walks.
   recs (nullable): point i's records of its *first* walk in the range go to
   recs + i*maxsteps*ORC_REC, nrec[i] of them. */
void orc_solve(const orc_scene *s, const orc_field *fld, const orc_params *p,
               const double *points, int npoints, int walk_begin, int nwalks, double *sum,
               double *sum2, int64_t *steps, int64_t *truncated, double *recs, int *nrec);

/* ---- training (Sec. 4.2 Eq. one_sample_kld, Sec. 4.4 Eq. one_sample_sp) -- */
/* Mean surrogate loss over n records; its gradient is the paper's one-sample
   estimator.  frozen_pg (nullable): per-record p_g used inside the
   selection-probability term (so FD of the loss reproduces the estimator).
   Gradient pointers may be NULL (loss only). */
double orc_train_loss(const orc_field *f, const double *recs, int n, double e_sel, int c_mode,
                      double c_fixed, int reflect, const double *frozen_pg, double *out_pg,
                      double *g_grid, double *g_W1, double *g_W2, double *g_W3, double *g_b3);
/* one Adam step (Kingma & Ba 2015) on a flat array */
void orc_adam(double *p, const double *g, double *m, double *v, int64_t n, double lr,
              double b1, double b2, double eps, int t);

#ifdef __cplusplus
}
#endif
#endif
