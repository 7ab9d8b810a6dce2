/* von Mises-Fisher distributions -- oracle (test infrastructure).
 *
 * Sec. 3.3: v(nu | mu, kappa) = kappa^{d/2-1} / ((2 pi)^{d/2} I_{d/2-1}(kappa))
 * exp(kappa mu.nu) on S^{d-1}, d = 2, 3.  Written in exponentially scaled
 * form so that large kappa does not overflow:
 *   d = 2: exp(kappa (mu.nu - 1)) / (2 pi I0e(kappa)),  I0e = e^{-k} I0
 *   d = 3: kappa exp(kappa (mu.nu - 1)) / (2 pi (1 - e^{-2 kappa}))
 * Sampling (Sec. 3.3): 2D Best & Fisher (1979) rejection sampler, 3D the
 * inverse-CDF form for cos(theta) of the stable sampler the paper cites
 * (Tokuyoshi 2025), w = 1 + log1p(xi expm1(-2 kappa)) / kappa, with an
 * orthonormal frame from Duff et al. (2017).
 */
#include <math.h>

#include "oracle.h"

/* Modified Bessel functions, exponentially scaled, from their defining
   series (x < 20) and the classical large-argument asymptotic expansion
   (x >= 20, truncated at its smallest term). */
static double bessel_series(double x, int order)
{
    double q = x * x / 4, term = order == 0 ? 1.0 : x / 2, sum = term;
    for (int k = 1; k < 500; ++k) {
        term *= q / ((double)k * (double)(k + order));
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return sum;
}

static double bessel_asym_scaled(double x, int order)
{
    /* I_n(x) e^{-x} sqrt(2 pi x) ~ sum_k (-1)^k a_k / x^k,
       a_k = prod_{j=1..k} (4 n^2 - (2j-1)^2) / (k! 8^k) */
    double mu4 = 4.0 * order * order, term = 1.0, sum = 1.0, prev = INFINITY;
    for (int k = 1; k < 200; ++k) {
        double f = (mu4 - (double)(2 * k - 1) * (2 * k - 1)) / (k * 8.0 * x);
        double nt = -term * f;
        if (fabs(nt) >= fabs(prev)) break;
        prev = nt;
        term = nt;
        sum += term;
        if (fabs(term) < 1e-18 * fabs(sum)) break;
    }
    return sum / sqrt(2 * M_PI * x);
}

double orc_i0e(double x)
{
    x = fabs(x);
    return x < 20 ? bessel_series(x, 0) * exp(-x) : bessel_asym_scaled(x, 0);
}

double orc_i1e(double x)
{
    double s = x < 0 ? -1 : 1;
    x = fabs(x);
    return s * (x < 20 ? bessel_series(x, 1) * exp(-x) : bessel_asym_scaled(x, 1));
}

double orc_vmf_pdf(int dim, double kappa, const double *mu, const double *nu)
{
    double c = 0;
    for (int i = 0; i < dim; ++i) c += mu[i] * nu[i];
    if (dim == 2) return exp(kappa * (c - 1)) / (2 * M_PI * orc_i0e(kappa));
    if (kappa == 0) return 1 / (4 * M_PI);
    return kappa * exp(kappa * (c - 1)) / (2 * M_PI * (-expm1(-2 * kappa)));
}

double orc_vmf_mean_cos(int dim, double kappa)
{
    if (dim == 2) return orc_i1e(kappa) / orc_i0e(kappa);
    /* coth(k) - 1/k, with its series near 0 */
    if (kappa < 1e-3) return kappa / 3 - kappa * kappa * kappa / 45;
    return 1 / tanh(kappa) - 1 / kappa;
}

double orc_mixture_pdf(int dim, int K, const double *mu, const double *kappa,
                       const double *lambda, const double *nu)
{
    double s = 0;
    for (int i = 0; i < K; ++i) s += lambda[i] * orc_vmf_pdf(dim, kappa[i], mu + i * dim, nu);
    return s;
}

/* Best & Fisher (1979): envelope parameter rho of the wrapped-Cauchy
   proposal, here in a cancellation-free form of (tau - sqrt(2 tau)) / (2 k). */
double orc_vmf2_sample_angle(double kappa, const uint32_t key[2], uint32_t pid, uint32_t wid,
                             uint32_t step, int *ntries)
{
    double s = sqrt(1 + 4 * kappa * kappa);
    double tau = 1 + s;
    double rho = 2 * kappa * tau / ((s + 1) * (tau + sqrt(2 * tau)));
    double r = (1 + rho * rho) / (2 * rho);
    double f = 0, u3 = 0;
    int j;
    for (j = 0; j < 64; ++j) {
        uint32_t ctr[4] = {pid, wid, step, 3u + (uint32_t)j}, o[4];
        orc_philox4x32_10(ctr, key, o);
        double u1 = orc_u01(o[0]), u2 = orc_u01(o[1]);
        u3 = orc_u01(o[2]);
        double z = cos(M_PI * u1);
        f = (1 + r * z) / (r + z);
        double c = kappa * (r - f);
        if (c * (2 - c) - u2 > 0) break;
        if (log(c / u2) + 1 - c >= 0) break;
    }
    if (ntries) *ntries = j + 1;
    if (f > 1) f = 1;
    if (f < -1) f = -1;
    double th = acos(f);
    return u3 < 0.5 ? -th : th;
}

/* Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin (2017):
   branchless orthonormal basis around a unit vector n. */
void orc_onb(const double *n, double *b1, double *b2)
{
    double sg = n[2] >= 0 ? 1.0 : -1.0;
    double a = -1.0 / (sg + n[2]);
    double b = n[0] * n[1] * a;
    b1[0] = 1 + sg * n[0] * n[0] * a;
    b1[1] = sg * b;
    b1[2] = -sg * n[0];
    b2[0] = b;
    b2[1] = sg + n[1] * n[1] * a;
    b2[2] = -n[1];
}

void orc_vmf3_sample(double kappa, const double *mu, double xi, double xi2, double *nu)
{
    double w;
    if (kappa == 0) w = 1 - 2 * xi;
    else w = 1 + log1p(xi * expm1(-2 * kappa)) / kappa;
    if (w > 1) w = 1;
    if (w < -1) w = -1;
    double st = sqrt(1 - w * w), ph = 2 * M_PI * xi2;
    double b1[3], b2[3];
    orc_onb(mu, b1, b2);
    for (int i = 0; i < 3; ++i) nu[i] = w * mu[i] + st * (cos(ph) * b1[i] + sin(ph) * b2[i]);
}
