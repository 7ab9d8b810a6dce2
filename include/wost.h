/*
 * libwost -- guided walk on stars on one GB300 (sm_103a).
 *
 * C ABI of the data-parallel hot path of "Guiding-Based Importance Sampling
 * for Walk on Stars" (arXiv 2410.18944): batched walk-on-stars (WoSt) walks
 * for the Poisson problem with mixed Dirichlet / Neumann boundary
 * (Sec. 3.1, Eq. linear_elliptic; estimator Sec. 3.2 Eq. wost_estm and its
 * reparameterisation Sec. 4.1), with optional guided direction sampling from
 * a von Mises-Fisher mixture decoded by a hash-grid + MLP neural field
 * (Sec. 3.3, 4.2, 5.2), sample reflection at Neumann points (Sec. 4.3),
 * one-sample MIS with a learnable selection probability (Sec. 4.4) and the
 * online training step of the field (Sec. 4.2 Eq. one_sample_kld, Sec. 4.4
 * Eq. one_sample_sp, Sec. 5.2 "Online Training Scheme").
 *
 * Conventions for every call:
 *  - returns a wost_status; WOST_OK == 0.  On failure wost_last_error()
 *    returns a message for the calling thread (thread-local, valid until the
 *    next call on that thread).
 *  - handles (wost_scene, wost_field) are opaque, owned by the library and
 *    released with the matching *_destroy call.
 *  - input arrays are owned by the caller and only read during the call;
 *    no call keeps a caller pointer after it returns.
 *  - "host-or-device" pointers are interpreted according to the
 *    `*_on_device` flags of wost_exec; device pointers must be on the current
 *    CUDA device.  Work is enqueued on wost_exec.stream (NULL = legacy
 *    default stream) and the call synchronises that stream before returning
 *    unless stated otherwise.
 *  - a scene, field or batch belongs to the CUDA device that was current
 *    when it was created; every call that uses it first checks that this
 *    device is current and otherwise returns WOST_ERR_INVALID_ARG without
 *    launching anything.
 *  - a scene and a field each hold work buffers that their calls reuse
 *    (per-point sums, walk slots, the launch order, training records):
 *    calls that use the same scene or the same field must not run
 *    concurrently (from two host threads, or on two streams before the
 *    first has returned).  Calls on different handles are independent.
 *  - geometry is stored in FP32, per-point accumulators in FP64.
 *  - there is no CPU fallback: without a usable CUDA device every call that
 *    needs one returns WOST_ERR_CUDA.
 */
#ifndef WOST_H
#define WOST_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    WOST_OK = 0,
    WOST_ERR_INVALID_ARG = 1,  /* null pointer, bad size, bad descriptor */
    WOST_ERR_ILL_POSED = 2,    /* e.g. no Dirichlet primitive */
    WOST_ERR_CUDA = 3,         /* CUDA runtime error (message has details) */
    WOST_ERR_TIMEOUT = 4,      /* a bounded device-side wait gave up */
    WOST_ERR_OOM = 5,          /* device allocation failed */
    WOST_ERR_UNSUPPORTED = 6   /* valid but not supported by this library (e.g. a field shape) */
} wost_status;

/* Analytic data functions g (Dirichlet), f (source), h (Neumann flux).
   kind codes:
     0 zero            1 const p0              2 exp(p0 x) cos(p0 y)
     3 x^2 - y^2       4 |x|^2                 5 1/|x - p[0:3]|
     6 log|x - p[0:2]| 7 sum_i A_i exp(-|x - c_i|^2 / (2 s^2)),
                         p = [n, s, A_1, c_1(3), A_2, c_2(3), ...], n <= 8
     8 cosh(p0 x) cos(p0 y)
     9 c + b.x + a_xx x^2 + a_yy y^2 + a_zz z^2 + a_xy x y + a_xz x z + a_yz y z,
                         p = [c, bx, by, bz, a_xx, a_yy, a_zz, a_xy, a_xz, a_yz] (z = 0 in 2D)
    10 p0 atan2(y, x) + p1 (polar angle) */
typedef struct {
    int32_t kind;
    int32_t nparams;
    double params[40];
} wost_fn;

/* Boundary description (Sec. 3.1).  2D: prims are segments (2 vertex
   indices), oriented counter-clockwise around the domain (domain on the left).
   3D: prims are triangles (3 indices) wound counter-clockwise seen from
   outside.  bc[i] = 0 Dirichlet, 1 Neumann.  The boundary must be closed. */
typedef struct {
    int32_t dim;               /* 2 or 3 */
    int64_t nverts;
    const double *verts;       /* host, nverts * dim */
    int64_t nprims;
    const int32_t *prims;      /* host, nprims * dim */
    const uint8_t *bc;         /* host, nprims */
    wost_fn g;                 /* Dirichlet data */
    wost_fn f;                 /* source, Laplacian u = f */
    wost_fn h;                 /* Neumann flux du/dn, n the normal pointing into the domain
                                  (kind 0: zero flux, the <N> term is skipped) */
    uint32_t scene_id;         /* folded into the random-number key */
} wost_scene_desc;

typedef struct wost_scene wost_scene;
typedef struct wost_field wost_field;

/* Neural field of the guiding distribution (Sec. 5.2): L levels of a hash
   grid (2^log2_table entries x F features, FP32 master + FP16 copy), MLP
   (L F) -> H -> H -> (d + 2) K + 1 with ReLU, BF16 operands, FP32
   accumulation.  Fixed in this library: F = 2, L * F = 32, H = 64; K = 1..16
   lobes (8 by default; the lobe-count ablation of Sec. 6.3 compares 4, 8
   and 16).  Fields of 9..16 lobes are served by 16-lobe variants of the
   kernels: their guided walks always run the warp-specialised kernel with
   the standard walker count (exec guided_kernel 2 or a wide walker_warps
   give WOST_ERR_UNSUPPORTED), their training step runs one 128-record tile
   per SM instead of two, and many-scene batches reject them
   (WOST_ERR_UNSUPPORTED).
   Positions are mapped to [0,1]^d by the box [lo, hi]. */
typedef struct {
    int32_t dim;
    int32_t K;                 /* lobes (1..16, default 8) */
    int32_t levels;            /* L (16) */
    int32_t log2_table;        /* log2 of entries per level */
    int32_t features;          /* F (2) */
    int32_t hidden;            /* H (64) */
    int32_t base_res, max_res; /* N_min, N_max of the level resolutions */
    double lo[3], hi[3];
    uint64_t seed;             /* initialisation */
    float lr_grid, lr_mlp;     /* Adam learning rates */
    float beta1, beta2, adam_eps;
    float e_sel;               /* selection-loss fraction e (0.2, Sec. 4.4) */
    int32_t grid_type;         /* 0 hash grid: every level has 2^log2_table entries, dense
                                  indexing where (N_l + 1)^d fits, else the spatial hash;
                                  exchange layout grid [L][2^log2_table][F].
                                  1 dense grid (the encoding of Sec. 5.2): every level dense
                                  with its own (N_l + 1)^d vertices (x fastest), the levels one
                                  after the other; exchange layout grid [entries][F] */
} wost_field_desc;

/* Execution options of a solve. */
typedef struct {
    uint64_t seed;             /* walk random-number seed */
    void *stream;              /* cudaStream_t, NULL = default stream */
    int32_t points_on_device;  /* points pointer is device memory */
    int32_t out_on_device;     /* out_mean / out_var are device memory */
    int32_t c_mode;            /* 0 learned c = sigmoid(c'), 1 fixed c_fixed */
    float c_fixed;
    int32_t reflect;           /* 1 = sample reflection at Neumann (default) */
    int32_t train;             /* guided: train the field after each batch */
    int32_t train_until_wpp;   /* stop training after this many walks/point */
    int64_t max_train_records; /* record buffer capacity (0 = default) */
    int32_t walk_begin;        /* index of the first walk (RNG counter) */
    int32_t ctas_per_sm;       /* launch shape override (0 = default) */
    int32_t guided_kernel;     /* single-scene guided walks: 0 automatic (the warp-specialised
                                  kernel for launches that record training data, the wavefront for
                                  the others), 1 warp-specialised persistent kernel (decode tiles
                                  served inside the walk kernel), 2 wavefront (step and tcgen05
                                  decode kernels alternating over walk slots in global memory);
                                  all draw the same random numbers */
    int32_t wavefront_slots;   /* walks in flight in a wavefront launch that trains nothing
                                  (0 = 2^20); a launch that trains holds one walk per point */
    int64_t train_samples;     /* records per training step (Sec. 5.2, online training in
                                  minibatches): 0 = one step on every record of the batch.
                                  Otherwise, with n > train_samples records, k = ceil(n /
                                  train_samples): after each batch of wost_solve the field takes
                                  k Adam steps, step j on records j, j + k, j + 2k, ... < n (every
                                  record once); one wost_train_step / wost_train_grad call takes
                                  the stratum o = (t * 2654435761) mod k, t the field's Adam step
                                  count before the step */
    int32_t rr_depth;          /* Russian roulette (Sec. 6.1: only for walks longer than 128 steps)
                                  from this step on: 0 = off (walks end at the maxsteps cap); a
                                  step k >= rr_depth goes on with probability rr_survival and
                                  divides the throughput by it, else the walk ends with value 0 */
    float rr_survival;         /* in (0, 1]; default 0.995 */
    int64_t wait_ns;           /* guided walks: limit in nanoseconds of every device-side wait of
                                  one warp on others (a decode tile filled, decoded or consumed);
                                  0 = 2 s.  A wait that runs out ends the launch and the call
                                  returns WOST_ERR_TIMEOUT; the device stays usable */
    int32_t batch_wpp;         /* wost_solve, guided with train: walks per point in one training
                                  batch (Sec. 5.2: a batch is one walk per point of a 1024^2 grid,
                                  about 2^20 walks; a smaller point set takes several walks per
                                  point to fill a batch of that size).  0 or 1 = one walk per
                                  point.  Batch b holds walks [w0 + b B, w0 + (b + 1) B) of every
                                  point (B = batch_wpp, the last batch clipped at train_until_wpp
                                  and nwalks); the field trains after each batch on all its
                                  records; the walks past train_until_wpp are not batched.  The
                                  random numbers of a walk do not depend on the grouping */
    int32_t walker_warps;      /* guided launches of the warp-specialised kernel: walker warps
                                  per CTA beside its 4 decode-server warps, 0 (automatic), 16 or
                                  28 (WOST_ERR_INVALID_ARG otherwise).  Automatic: wost_solve takes
                                  28 when the scene's traversal data (BVH nodes, cones,
                                  primitives) exceeds 64 MB or, in 3D, when a launch holds at
                                  least two walks per lane of the 28-warp kernel, else 16;
                                  wost_batch_create lets its autotuner choose.  Results do not
                                  depend on it */
} wost_exec;

typedef struct {
    int64_t walk_steps;        /* loop iterations of all walks, incl. terminal */
    int64_t walks;
    int64_t truncated;         /* walks closed by the maxsteps cap */
    int64_t records;           /* training records produced */
    int64_t records_dropped;   /* records beyond the buffer capacity */
    int32_t train_steps;
    float last_loss;
    double ms_walk;            /* device time in walk kernels (CUDA events on the exec stream) */
    double ms_train;           /* device time in training kernels (gradient + Adam + copies) */
    int64_t kernel_launches;   /* kernels this call launched */
    int64_t walk_launches;     /* of which walk kernels */
    int64_t node_visits;       /* BVH nodes visited by all walk-step queries */
    int64_t prim_visits;       /* primitives / silhouette elements tested */
    double alg_bytes;          /* algorithmic bytes of the walk kernels: visited BVH nodes and
                                  primitives, hash-grid corner reads, query points, FP64
                                  accumulator updates, training-record writes and suffix pass */
    int64_t dir_prim_visits;   /* of prim_visits: Dirichlet primitives (closest point) */
    int64_t sil_prim_visits;   /* silhouette elements (closest silhouette) */
    int64_t neu_prim_visits;   /* Neumann primitives (ray casts and the Neumann-flux sample) */
} wost_stats;

const char *wost_last_error(void);
/* fills *exec with the defaults (seed 1, reflect 1, train_until_wpp 256) */
void wost_exec_defaults(wost_exec *exec);
/* fills *desc with the defaults for dimension dim (K 8, L 16, F 2, H 64,
   log2_table 16 in 2D / 19 in 3D, N_min 16, N_max 2048 / 512, lr 1e-2 grid /
   1e-3 MLP, beta (0.9, 0.99), eps 1e-8, e 0.2); lo/hi = [-1, 1]^d */
void wost_field_desc_defaults(wost_field_desc *desc, int32_t dim);

/* Validates the boundary, builds three BVHs (Dirichlet closest point,
   Neumann silhouette elements, Neumann ray cast; Sec. 5.3) on the host and
   uploads them.  WOST_ERR_ILL_POSED if there is no Dirichlet primitive. */
wost_status wost_create_scene(const wost_scene_desc *desc, wost_scene **out);
wost_status wost_destroy_scene(wost_scene *scene);
/* the CUDA device the scene belongs to (current at wost_create_scene) */
wost_status wost_scene_device(const wost_scene *scene, int32_t *device);
/* padded bounding box (5% of the extent on each side) for the field box */
wost_status wost_scene_bbox(const wost_scene *scene, double lo[3], double hi[3]);

/* Estimates u at npoints points (host-or-device, npoints * dim doubles)
   with nwalks walks each (Sec. 3.2; guided: Sec. 4).  Points outside the
   domain get NaN, points inside the eps-shell get g at the closest Dirichlet
   point with variance 0.  out_mean[i] is the sample mean, out_var[i]
   (nullable) the variance of that mean.  guided != 0 requires a field; with
   exec->train the field is trained after every batch of exec->batch_wpp
   walks per point (one by default, Sec. 5.2) until train_until_wpp walks per
   point.  Batches run in order,
   so the estimate is deterministic up to floating-point atomics.  Guided
   launches of the warp-specialised kernel hand out their points longest
   walks first, by the walk lengths of the scene's previous such launch on
   as many points; a walk's random numbers depend only on its (point, walk)
   pair, so this order changes no estimate.  One walk
   per point gives variance 0 (no sample variance from one sample).  With
   npoints == 0 the call does nothing and returns WOST_OK; points and the
   outputs may then be NULL. */
wost_status wost_solve(wost_scene *scene, wost_field *field, const double *points,
                       int64_t npoints, int32_t nwalks, double eps, int32_t maxsteps,
                       int32_t guided, double *out_mean, double *out_var, wost_stats *stats,
                       const wost_exec *exec);

/* Neural field lifetime and parameters (exchange layout, float32):
   grid [L][2^log2_table][F], W1 [H][L F], W2 [H][H], W3 [nout][H], b3 [nout]
   with nout = (dim + 2) K + 1; output order mu'_i (K x d), kappa'_i (K),
   lambda'_i (K), c' (Tab. reg_map).  Parameter and gradient arrays of
   set_params / get_params / wost_train_grad may be host or device memory
   (unified addressing); set_params resets the Adam moments and step count. */
wost_status wost_create_field(const wost_field_desc *desc, wost_field **out);
wost_status wost_destroy_field(wost_field *field);
wost_status wost_field_set_params(wost_field *field, const float *grid, const float *W1,
                                  const float *W2, const float *W3, const float *b3);
wost_status wost_field_get_params(const wost_field *field, float *grid, float *W1, float *W2,
                                  float *W3, float *b3);
/* Lattice entries of the field's grid, all levels (L 2^log2_table for the
   hash grid, sum_l (N_l + 1)^d for the dense grid). */
wost_status wost_field_grid_entries(const wost_field *field, int64_t *entries);
/* Raw network outputs (nout floats per point, host-or-device per exec) for
   npoints points (npoints * dim doubles): hash-grid encoding + MLP on tensor
   cores, the decode used inside the guided walk. */
wost_status wost_field_decode(wost_field *field, const double *points, int64_t npoints,
                              float *out_raw, const wost_exec *exec);

/* One training step of the field (Sec. 4.2, 4.4) on the records of the most
   recent guided batch of wost_solve (or those given by wost_train_records):
   fused recomputation of the forward, loss gradients (Eq. one_sample_kld,
   Eq. one_sample_sp), MLP backward on tensor cores, hash-grid scatter-add,
   Adam.  *out_loss (nullable) receives the mean surrogate loss. */
wost_status wost_train_step(wost_scene *scene, wost_field *field, const wost_exec *exec,
                            float *out_loss);
/* Replaces the field's record buffer with n caller records (12 floats each:
   x[3], nu[3], n[3], on_neumann, q, target; host-or-device per exec). */
wost_status wost_train_records(wost_field *field, const float *records, int64_t n,
                               const wost_exec *exec);
/* Copies up to cap records of the buffer to host memory; *n = count. */
wost_status wost_get_records(const wost_field *field, float *records, int64_t cap, int64_t *n);
/* The mean surrogate loss of wost_train_grad alone (the same fused kernel:
   forward recomputed from the records on tensor cores, no backward pass,
   gradient buffers untouched).  out_loss: one float, host memory, or device
   memory with exec->out_on_device (then the call only enqueues on
   exec->stream and does not synchronise). */
wost_status wost_train_loss(wost_field *field, const wost_exec *exec, float *out_loss);
/* Loss and gradients without the Adam update: grads in the exchange layout
   (host or device; nullable each), from the same fused kernel as
   wost_train_step: the forward is recomputed from the records and the
   backward runs on tensor cores (the binding's torch.autograd.Function). */
wost_status wost_train_grad(wost_field *field, const wost_exec *exec, float *out_loss,
                            float *g_grid, float *g_W1, float *g_W2, float *g_W3, float *g_b3);

/* ---- query entry points (the walk's building blocks, for testing) ------- */
/* closest Dirichlet primitive: index (-1 if none) and FP32 distance */
wost_status wost_query_closest(wost_scene *scene, const double *points, int64_t n,
                               int32_t *out_prim, float *out_dist);
/* closest silhouette element of the Neumann boundary (Sec. 3.2): its vertex
   (2D) or its edge's vertex pair a < b encoded a * nverts + b (3D), -1 if
   none, and the distance (+inf if none) */
wost_status wost_query_silhouette(wost_scene *scene, const double *points, int64_t n,
                                  int64_t *out_elem, float *out_dist);
/* first Neumann primitive hit along x + t v, 0 < t <= tmax, skipping prim
   skip[i] (-1 none); -1 if no hit */
wost_status wost_query_ray(wost_scene *scene, const double *org, const double *dir,
                           const double *tmax, const int32_t *skip, int64_t n,
                           int32_t *out_prim, float *out_t);
/* The cast a walk step makes (Sec. 3.2: the next point is the first hit on
   the star's Neumann boundary within r, else x + r nu), for testing it on its
   own.  Only primitives the ray leaves the domain through count (direction
   against the inward normal): inside a closed boundary the first crossing is
   an exit.  Crossings count from t > -b and within about b of the primitive,
   b = 16 * 2^-24 * (bounding-box diagonal), so a start point rounded a hair
   outside the boundary next to a vertex still leaves through the neighbour.
   org / dir / tmax are rounded to FP32 as a walk holds them; a winner whose
   FP32 parameter lies within b of tmax is re-tested in FP64 against the FP32
   tmax.  skip[i]: primitive id the ray starts on (-1 none, nullable array).
   Outputs: the primitive id (-1 if none within tmax) and its FP32 parameter
   (+inf if none).  Host arrays. */
wost_status wost_query_ray_exit(wost_scene *scene, const double *org, const double *dir,
                                const double *tmax, const int32_t *skip, int64_t n,
                                int32_t *out_prim, float *out_t);
/* vMF mixture: pdf at directions given identical parameters (K = 1..16
   lobes: mu K x d, kappa K, lambda K per row) and one guided sample per row from Philox
   counters (point, walk, step) with the walk's key; all host arrays. */
wost_status wost_mixture_eval(int32_t dim, int32_t K, const float *mu, const float *kappa,
                              const float *lambda, const float *nu, int64_t n, float *out_pdf);
wost_status wost_mixture_sample(int32_t dim, int32_t K, const float *mu, const float *kappa,
                                const float *lambda, const uint32_t *counters, uint64_t seed,
                                uint32_t scene_id, int64_t n, float *out_nu, float *out_pdf);

/* ---- many scenes in one launch ---------------------------------------------- */
/* A batch solves many independent problems -- scenes of uneven size, point
   sets of uneven size, different walk counts, eps, step caps and seeds --
   with the walks of all of them in one persistent walk launch (per training
   round when guided fields train, Sec. 5.2), the whole solve captured once
   into a CUDA graph and replayed by wost_batch_run.  Each job walks exactly
   as wost_solve(job.scene, job.field, job.points, ...) with exec.seed =
   job.seed would: the same estimator (Sec. 3.2, Sec. 4) and the same
   random streams, so a batch differs from the separate solves only in the
   order of floating-point atomic sums (and, when fields train, in the
   training steps that follow from that order). */
typedef struct {
    wost_scene *scene;
    wost_field *field;         /* guided batches: this job's field (distinct per job when
                                  training); NULL in plain batches */
    const double *points;      /* device, npoints * dim doubles (caller-owned, read at every run) */
    int64_t npoints;
    int32_t nwalks;
    double eps;
    int32_t maxsteps;
    uint64_t seed;             /* walk seed (key = seed, scene_id as in wost_solve) */
    double *out_mean;          /* device, npoints doubles (caller-owned, written at every run) */
    double *out_var;           /* device, npoints doubles, nullable: variance of the mean */
} wost_job;

typedef struct wost_batch wost_batch;

/* Launch parameters of a plan and how they were chosen. */
typedef struct {
    int32_t ctas_per_sm;       /* plain walk launch: resident CTAs per SM */
    int32_t flush_polls;       /* guided walk launch: server polls before a partial decode
                                  tile is closed and zero-padded */
    int32_t candidates;        /* launch shapes timed by the autotuner (0: none, fixed by exec) */
    double best_ms, worst_ms;  /* calibration-launch times of the best / worst candidate */
    int32_t walk_launches;     /* walk launches in the graph (1, or 1 per training round + 1) */
    int32_t train_steps;       /* training steps in the graph */
    int64_t graph_nodes;
    int32_t walker_warps;      /* guided walk launch: walker warps per CTA */
} wost_batch_info;

/* Plans a batch of njobs jobs, all of the same dimension: validates them,
   allocates the batch's work buffers (and the fields' training-record
   buffers when exec->train), picks the launch parameters and captures the
   solve into a CUDA graph.  Launch parameters: exec->ctas_per_sm > 0 fixes
   the plain launch shape; 0 lets an autotuner time candidate shapes (plain:
   CTAs per SM; guided: the decode-tile flush threshold) on one calibration
   walk per point of every job and keep the fastest.  Calibration launches
   record nothing and do not touch the fields.  guided != 0 needs a field
   per job; exec->c_mode, c_fixed, reflect, train, train_until_wpp and
   max_train_records apply to every job.  Pointers of the jobs are kept by
   the plan and must stay valid until wost_batch_destroy.  The guided
   autotuner also times 16 against 28 walker warps per CTA unless
   exec->walker_warps fixes the count. */
wost_status wost_batch_create(int32_t njobs, const wost_job *jobs, int32_t guided, const wost_exec *exec,
                              wost_batch **out);
/* Replays the plan on stream (cudaStream_t, NULL = default stream) and
   waits for it.  stats (nullable) sums all jobs; ms_walk is the device time
   of the whole graph (walks and training).  Re-running a plan with training
   continues to train the fields. */
wost_status wost_batch_run(wost_batch *batch, void *stream, wost_stats *stats);
wost_status wost_batch_info_get(const wost_batch *batch, wost_batch_info *info);
wost_status wost_batch_destroy(wost_batch *batch);
/* create + run + destroy */
wost_status wost_solve_batch(int32_t njobs, const wost_job *jobs, int32_t guided, const wost_exec *exec,
                             wost_stats *stats);

/* ---- plain solve without device allocation ---------------------------------- */
/* The paper has no counterpart to this entry point; it exists for callers
   that cannot allocate device memory while solving -- for instance when
   another component owns the whole device memory pool, or in a loop that
   must not pay the device-wide synchronisation implied by cudaFree.
   wost_solve_plain_static runs the plain (unguided) walk of wost_solve, with
   the same random streams, but keeps all of its scratch memory (per-point
   FP64 sums, point status, work counter, statistics) in one fixed array
   compiled into the library (about 6.6 MB, present on every GPU that loads
   the library until the process exits).  It calls no cudaMalloc / cudaFree.
     points_dev    device, npoints * dim doubles (caller-owned)
     out_mean_dev  device, npoints doubles (caller-owned); out_var_dev
                   nullable, variance of the mean
     npoints       at most WOST_STATIC_MAX_POINTS, else WOST_ERR_INVALID_ARG
     stream        cudaStream_t (NULL = default); synchronised before return
     out_walk_steps (nullable, host) walk-steps of the solve
   The scene must belong to the current device (WOST_ERR_INVALID_ARG
   otherwise, before any launch).
   The first call on a device looks up the array's device address with
   cudaGetSymbolAddress.  Every call
   reuses the same array and clears what must start at zero; calls whose GPU
   work overlaps (e.g. issued on two streams) race on it. */
#define WOST_STATIC_MAX_POINTS 262144
wost_status wost_solve_plain_static(wost_scene *scene, const double *points_dev, int64_t npoints,
                                    int32_t nwalks, double eps, int32_t maxsteps, uint64_t seed,
                                    void *stream, double *out_mean_dev, double *out_var_dev,
                                    int64_t *out_walk_steps);

/* ---- diagnostics ---------------------------------------------------------- */
/* The failure path of the bounded device-side waits, without a fault: one
   warp waits (the walk kernels' bounded wait) on a shared-memory mbarrier
   that gets its arrival only if `arrive` != 0.  Without it the wait runs out
   after limit_ns (0 < limit_ns <= 1e10) and the call returns
   WOST_ERR_TIMEOUT; the device stays usable.  With it the call returns
   WOST_OK. */
wost_status wost_diag_wait(int64_t limit_ns, int32_t arrive);
/* Records `device` as the device the scene belongs to, without moving any of
   its data.  For tests of the device check on one-GPU machines: with a
   device other than the current one, every later call on the scene returns
   WOST_ERR_INVALID_ARG before any launch; rebinding to the true device
   restores it. */
wost_status wost_diag_scene_rebind(wost_scene *scene, int32_t device);
/* D[128 x N] = A[128 x K] B[N x K]^T (host float arrays, row-major) through
   the library's tensor-core path (BF16 operands, FP32 accumulation); a_mn /
   b_mn select K-major (0) or MN-major (1) shared-memory storage.  N in
   [16, 256], K in [16, 128], both multiples of 16. */
wost_status wost_diag_umma(int32_t a_mn, int32_t b_mn, int32_t N, int32_t K, const float *A, const float *B,
                           float *D);

#ifdef __cplusplus
}
#endif
#endif
