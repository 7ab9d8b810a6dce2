/* Neural field of the guiding distribution -- oracle (test infrastructure).
 *
 * Sec. 5.2: a multi-resolution feature grid G(x) (L levels, F features per
 * lattice vertex, bi/tri-linear interpolation, levels concatenated) feeds a
 * ReLU MLP with two hidden layers of width H and a linear output layer with
 * bias.  The output has (d + 2) K + 1 entries: mu'_i (d each), kappa'_i,
 * lambda'_i, c' (Sec. 4.2, Eq. nn_to_theta), mapped by Tab. "reg_map".
 *
 * Lattice storage follows the hash-grid encoding of Mueller et al. (2022):
 * level l has resolution N_l = floor(N_min b^l) with b chosen so that
 * N_{L-1} = N_max; a level whose (N_l + 1)^d vertices fit the table of size
 * T = 2^log2T is indexed densely (x fastest), finer levels by the spatial
 * hash (i * 1) xor (j * 2654435761) xor (k * 805459861) mod T.
 * Positions are mapped to [0,1]^d by the box [lo, hi].
 *
 * Dense grid (grid_type 1; the encoding the paper uses, Sec. 5.2): the same
 * levels, every one stored densely with its own (N_l + 1)^d vertices, level l
 * starting at entry sum_{j<l} (N_j + 1)^d.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

int orc_field_nout(const orc_field *f) { return (f->dim + 2) * f->K + 1; }

int orc_level_res(const orc_field *f, int l)
{
    if (f->L == 1) return f->base_res;
    double b = exp((log((double)f->max_res) - log((double)f->base_res)) / (f->L - 1));
    return (int)floor(f->base_res * pow(b, l) + 1e-6);
}

static int64_t level_vertices(const orc_field *f, int l)
{
    int64_t side = orc_level_res(f, l) + 1, n = 1;
    for (int k = 0; k < f->dim; ++k) n *= side;
    return n;
}

/* first entry of level l in the grid array */
static int64_t level_offset(const orc_field *f, int l)
{
    if (f->grid_type == 0) return (int64_t)l << f->log2T;
    int64_t off = 0;
    for (int j = 0; j < l; ++j) off += level_vertices(f, j);
    return off;
}

int64_t orc_field_entries(const orc_field *f) { return level_offset(f, f->L); }

/* corner c (bit k of c selects +1 along axis k) of the cell around x:
   grid-array entry (level offset included) and interpolation weight */
static void level_corners(const orc_field *f, int l, const double *x, int64_t *idx, double *w)
{
    int d = f->dim, N = orc_level_res(f, l);
    int64_t T = (int64_t)1 << f->log2T, off = level_offset(f, l);
    int64_t cell[3];
    double fr[3];
    for (int k = 0; k < d; ++k) {
        double u = (x[k] - f->lo[k]) / (f->hi[k] - f->lo[k]);
        double p = u * N;
        double c = floor(p);
        if (c < 0) c = 0;
        if (c > N - 1) c = N - 1;
        cell[k] = (int64_t)c;
        fr[k] = p - c;
    }
    int64_t side = N + 1, nvert = 1;
    for (int k = 0; k < d; ++k) nvert *= side;
    for (int c = 0; c < (1 << d); ++c) {
        int64_t v[3];
        double wt = 1;
        for (int k = 0; k < d; ++k) {
            int bit = (c >> k) & 1;
            v[k] = cell[k] + bit;
            wt *= bit ? fr[k] : 1 - fr[k];
        }
        int64_t id;
        if (f->grid_type == 1 || nvert <= T) {
            id = v[0] + side * (v[1] + (d == 3 ? side * v[2] : 0));
        } else {
            uint32_t h = (uint32_t)v[0] * 1u;
            h ^= (uint32_t)v[1] * 2654435761u;
            if (d == 3) h ^= (uint32_t)v[2] * 805459861u;
            id = (int64_t)(h & (uint32_t)(T - 1));
        }
        idx[c] = off + id;
        w[c] = wt;
    }
}

void orc_field_encode(const orc_field *f, const double *x, double *feat)
{
    for (int l = 0; l < f->L; ++l) {
        int64_t idx[8];
        double w[8];
        level_corners(f, l, x, idx, w);
        for (int j = 0; j < f->F; ++j) {
            double s = 0;
            for (int c = 0; c < (1 << f->dim); ++c)
                s += w[c] * f->grid[(size_t)idx[c] * f->F + j];
            feat[l * f->F + j] = s;
        }
    }
}

/* dense layer y = W x (W is rows x cols, row-major) */
static void matvec(const double *W, const double *x, double *y, int rows, int cols)
{
    for (int r = 0; r < rows; ++r) {
        double s = 0;
        for (int c = 0; c < cols; ++c) s += W[(size_t)r * cols + c] * x[c];
        y[r] = s;
    }
}

/* forward with the intermediate activations kept (for the backward pass) */
void orc__field_forward_full(const orc_field *f, const double *x, double *feat, double *z1,
                             double *z2, double *raw)
{
    int nin = f->L * f->F, H = f->H, no = orc_field_nout(f);
    double h1[256], h2[256];
    orc_field_encode(f, x, feat);
    matvec(f->W1, feat, z1, H, nin);
    for (int i = 0; i < H; ++i) h1[i] = z1[i] > 0 ? z1[i] : 0;
    matvec(f->W2, h1, z2, H, H);
    for (int i = 0; i < H; ++i) h2[i] = z2[i] > 0 ? z2[i] : 0;
    matvec(f->W3, h2, raw, no, H);
    for (int i = 0; i < no; ++i) raw[i] += f->b3[i];
}

void orc_field_forward(const orc_field *f, const double *x, double *raw)
{
    double feat[256], z1[256], z2[256];
    orc__field_forward_full(f, x, feat, z1, z2, raw);
}

/* Tab. reg_map: mu = mu'/|mu'|, kappa = exp(kappa') (kappa' clamped to
   [-8, 8]), lambda = softmax(lambda'), c = sigmoid(c') */
void orc_theta_map(const orc_field *f, const double *raw, double *mu, double *kappa,
                   double *lambda, double *c)
{
    int d = f->dim, K = f->K;
    for (int i = 0; i < K; ++i) {
        double n2 = 0;
        for (int k = 0; k < d; ++k) n2 += raw[i * d + k] * raw[i * d + k];
        double nn = sqrt(n2);
        for (int k = 0; k < d; ++k) mu[i * d + k] = nn > 0 ? raw[i * d + k] / nn : (k == 0);
        double kp = raw[K * d + i];
        if (kp < -8) kp = -8;
        if (kp > 8) kp = 8;
        kappa[i] = exp(kp);
    }
    double mx = -INFINITY, s = 0;
    for (int i = 0; i < K; ++i) mx = fmax(mx, raw[K * d + K + i]);
    for (int i = 0; i < K; ++i) {
        lambda[i] = exp(raw[K * d + K + i] - mx);
        s += lambda[i];
    }
    for (int i = 0; i < K; ++i) lambda[i] /= s;
    if (c) *c = 1 / (1 + exp(-raw[K * (d + 2)]));
}

/* grid gradient scatter for the backward pass */
void orc__field_grid_backward(const orc_field *f, const double *x, const double *dfeat,
                              double *g_grid)
{
    for (int l = 0; l < f->L; ++l) {
        int64_t idx[8];
        double w[8];
        level_corners(f, l, x, idx, w);
        for (int c = 0; c < (1 << f->dim); ++c)
            for (int j = 0; j < f->F; ++j)
                g_grid[(size_t)idx[c] * f->F + j] += w[c] * dfeat[l * f->F + j];
    }
}
