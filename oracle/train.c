/* Online training loss of the guiding field -- oracle (test infrastructure).
 *
 * Per training record (x, nu, Neumann normal n, q = p~ at sampling time,
 * target p_t = |<u(x_{k+1})>|):
 *   l = -(p_t / q) [ log p_g(nu | Theta(x)) + e log p~_c(nu) ]
 * where p_g is the (reflected, Sec. 4.3) mixture density and
 * p~_c = c p_g0 + (1 - c) p_u with p_g0 held fixed.  Its gradient is exactly
 * the paper's one-sample estimators:
 *   d l / d Theta = -p_t grad V / (p~ V)            (Sec. 4.2, Eq. one_sample_kld)
 *   d l / d c     = -e p_t (p_g - p_u) / p~^2        (Sec. 4.4, Eq. one_sample_sp)
 * (Theta receives only the KL(p_t || V) term, c only the selection term, as
 * printed; q = p~ when the field has not moved since sampling.)  The loss is
 * the mean over records; gradients are back-propagated through the MLP and
 * scattered onto the lattice (Sec. 4.2, "back-propagated all the way to the
 * grid and MLP parameters").  Adam follows Kingma & Ba (2015).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"

void orc__field_forward_full(const orc_field *f, const double *x, double *feat, double *z1,
                             double *z2, double *raw);
void orc__field_grid_backward(const orc_field *f, const double *x, const double *dfeat,
                              double *g_grid);

static double vdot(int d, const double *a, const double *b)
{
    double s = 0;
    for (int i = 0; i < d; ++i) s += a[i] * b[i];
    return s;
}

double orc_train_loss(const orc_field *f, const double *recs, int n, double e_sel, int c_mode,
                      double c_fixed, int reflect, const double *frozen_pg, double *out_pg,
                      double *g_grid, double *g_W1, double *g_W2, double *g_W3, double *g_b3)
{
    const int d = f->dim, K = f->K, H = f->H, nin = f->L * f->F, no = orc_field_nout(f);
    const double area = d == 2 ? 2 * M_PI : 4 * M_PI;
    const int want_grad = g_W1 != NULL;
    double loss = 0;
    for (int r = 0; r < n; ++r) {
        const double *R = recs + (size_t)r * ORC_REC;
        const double *x = R, *nu = R + 3, *nrm = R + 6;
        int on_neu = R[9] != 0;
        double q = R[10], pt = R[11];
        double feat[256], z1[256], z2[256], raw[256];
        orc__field_forward_full(f, x, feat, z1, z2, raw);
        double mu[3 * 32], kap[32], lam[32], c;
        orc_theta_map(f, raw, mu, kap, lam, &c);
        if (c_mode == 1) c = c_fixed;

        /* directions at which the guided density is evaluated */
        double dirs[2][3];
        int nd = 1;
        memcpy(dirs[0], nu, sizeof(double) * 3);
        if (on_neu && reflect) {
            double t = vdot(d, nu, nrm);
            for (int i = 0; i < d; ++i) dirs[1][i] = nu[i] - 2 * t * nrm[i];
            nd = 2;
        }
        double v[2][32], sl[32], pg = 0;
        for (int i = 0; i < K; ++i) {
            sl[i] = 0;
            for (int j = 0; j < nd; ++j) {
                v[j][i] = orc_vmf_pdf(d, kap[i], mu + i * d, dirs[j]);
                sl[i] += v[j][i];
            }
            pg += lam[i] * sl[i];
        }
        if (out_pg) out_pg[r] = pg;
        double pu = (on_neu ? 2.0 : 1.0) / area;
        double pg0 = frozen_pg ? frozen_pg[r] : pg;
        double ptil = c * pg0 + (1 - c) * pu;
        double wt = pt / q;
        if (pt == 0) continue;
        double lpg = log(fmax(pg, 1e-300));
        loss += -wt * (lpg + (c_mode == 0 ? e_sel * log(ptil) : 0.0));
        if (!want_grad) continue;

        /* gradient w.r.t. the raw network outputs */
        double draw[256];
        memset(draw, 0, sizeof(draw));
        double dpg = -wt / fmax(pg, 1e-300) / n;
        for (int i = 0; i < K; ++i) {
            const double *m = mu + i * d;
            /* lambda' (softmax) */
            draw[K * d + K + i] = dpg * lam[i] * (sl[i] - pg);
            /* kappa' (exp, zero outside the clamp) and mu' (normalisation) */
            double kp = raw[K * d + i];
            double A = orc_vmf_mean_cos(d, kap[i]);
            double dk = 0, dm[3] = {0, 0, 0};
            for (int j = 0; j < nd; ++j) {
                double cm = vdot(d, m, dirs[j]);
                dk += v[j][i] * (cm - A);
                for (int k = 0; k < d; ++k) dm[k] += v[j][i] * (dirs[j][k] - cm * m[k]);
            }
            if (kp > -8 && kp < 8) draw[K * d + i] = dpg * lam[i] * kap[i] * dk;
            double nn = 0;
            for (int k = 0; k < d; ++k) nn += raw[i * d + k] * raw[i * d + k];
            nn = sqrt(nn);
            if (nn > 0)
                for (int k = 0; k < d; ++k) draw[i * d + k] = dpg * lam[i] * kap[i] * dm[k] / nn;
        }
        if (c_mode == 0) {
            double dc = -e_sel * wt * (pg0 - pu) / ptil / n;
            draw[K * (d + 2)] = dc * c * (1 - c);
        }

        /* MLP backward */
        double h1[256], h2[256], dh2[256], dz2[256], dh1[256], dz1[256], dfeat[256];
        for (int i = 0; i < H; ++i) {
            h1[i] = z1[i] > 0 ? z1[i] : 0;
            h2[i] = z2[i] > 0 ? z2[i] : 0;
        }
        for (int o = 0; o < no; ++o) {
            g_b3[o] += draw[o];
            for (int i = 0; i < H; ++i) g_W3[(size_t)o * H + i] += draw[o] * h2[i];
        }
        for (int i = 0; i < H; ++i) {
            double s = 0;
            for (int o = 0; o < no; ++o) s += f->W3[(size_t)o * H + i] * draw[o];
            dh2[i] = s;
            dz2[i] = z2[i] > 0 ? s : 0;
        }
        for (int o = 0; o < H; ++o)
            for (int i = 0; i < H; ++i) g_W2[(size_t)o * H + i] += dz2[o] * h1[i];
        for (int i = 0; i < H; ++i) {
            double s = 0;
            for (int o = 0; o < H; ++o) s += f->W2[(size_t)o * H + i] * dz2[o];
            dh1[i] = s;
            dz1[i] = z1[i] > 0 ? s : 0;
        }
        for (int o = 0; o < H; ++o)
            for (int i = 0; i < nin; ++i) g_W1[(size_t)o * nin + i] += dz1[o] * feat[i];
        for (int i = 0; i < nin; ++i) {
            double s = 0;
            for (int o = 0; o < H; ++o) s += f->W1[(size_t)o * nin + i] * dz1[o];
            dfeat[i] = s;
        }
        orc__field_grid_backward(f, x, dfeat, g_grid);
        (void)dh2;
        (void)dh1;
    }
    return loss / n;
}

void orc_adam(double *p, const double *g, double *m, double *v, int64_t n, double lr,
              double b1, double b2, double eps, int t)
{
    double c1 = 1 - pow(b1, t), c2 = 1 - pow(b2, t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1 - b1) * g[i];
        v[i] = b2 * v[i] + (1 - b2) * g[i] * g[i];
        double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * mh / (sqrt(vh) + eps);
    }
}
