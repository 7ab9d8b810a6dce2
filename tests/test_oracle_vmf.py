"""Pins of the oracle's von Mises-Fisher densities and samplers (Sec. 3.3):
Bessel functions against scipy, normalisation by quadrature, the reflected
hemisphere density of Sec. 4.3, and sampler histograms / first moments."""
import math

import numpy as np
import pytest
from scipy import special

import oracle

KAPPAS = [1e-6, 1e-3, 0.1, 0.5, 1.0, 3.7, 3.8, 10.0, 19.9, 20.1, 50.0, 300.0, 2980.0]


@pytest.mark.parametrize("x", [0.0, 1e-8, 1e-3, 0.3, 1.0, 3.75, 7.0, 19.99, 20.0, 20.01, 35.0, 100.0, 1e3, 3e3])
def test_bessel_scaled_vs_scipy(x):
    assert oracle.i0e(x) == pytest.approx(special.i0e(x), rel=2e-14, abs=1e-300)
    assert oracle.i1e(x) == pytest.approx(special.i1e(x), rel=2e-14, abs=1e-300)


def _circle(n):
    th = (np.arange(n) + 0.5) * 2 * np.pi / n
    return np.stack([np.cos(th), np.sin(th)], 1), 2 * np.pi / n


def _sphere(n):
    # Gauss-Legendre in cos(theta) x uniform in phi
    x, w = np.polynomial.legendre.leggauss(n)
    ph = (np.arange(2 * n) + 0.5) * np.pi / n
    ct, P = np.meshgrid(x, ph, indexing="ij")
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(P), st * np.sin(P), ct], -1).reshape(-1, 3)
    wts = (w[:, None] * np.full(2 * n, np.pi / n)[None]).reshape(-1)
    return dirs, wts


@pytest.mark.parametrize("kappa", KAPPAS)
def test_vmf2_normalised(kappa):
    mu = np.array([math.cos(0.7), math.sin(0.7)])
    # concentrate quadrature around mu for large kappa: integrate in angle
    # offset from mu with a trapezoid on a fine uniform grid
    n = 200000
    th = (np.arange(n) + 0.5) * 2 * np.pi / n - np.pi
    nu = np.stack([np.cos(0.7 + th), np.sin(0.7 + th)], 1)
    p = np.array([oracle.vmf_pdf(2, kappa, mu, v) for v in nu[:: max(1, n // 20000)]])
    # coarse check of the shape on a subsample, exact check via scipy integral
    from scipy.integrate import quad
    f = lambda t: oracle.vmf_pdf(2, kappa, mu, np.array([math.cos(0.7 + t), math.sin(0.7 + t)]))
    s = quad(f, -np.pi, np.pi, points=[0.0], limit=400, epsabs=1e-13, epsrel=1e-12)[0]
    assert s == pytest.approx(1.0, abs=1e-10)
    assert np.all(p >= 0)


@pytest.mark.parametrize("kappa", KAPPAS)
def test_vmf3_normalised(kappa):
    from scipy.integrate import quad
    mu = np.array([0.0, 0.0, 1.0])
    # density depends on cos(theta) only: integral = 2 pi int_{-1}^{1} v(w) dw
    f = lambda w: oracle.vmf_pdf(3, kappa, mu, np.array([math.sqrt(max(0, 1 - w * w)), 0.0, w]))
    s = 2 * np.pi * quad(f, -1, 1, points=[1 - 1 / max(kappa, 1)], limit=400, epsabs=1e-13, epsrel=1e-12)[0]
    assert s == pytest.approx(1.0, abs=1e-10)


@pytest.mark.parametrize("K", [8, 16])
@pytest.mark.parametrize("kappa", [0.5, 5.0, 60.0])
def test_mixture_and_reflected_density_normalised(kappa, K):
    rng = np.random.default_rng(0)
    # 2D: the reflected guided density V(nu) + V(nu^-) on the half circle
    # nu . n > 0 integrates to one (Sec. 4.3)
    mu = rng.normal(size=(K, 2))
    mu /= np.linalg.norm(mu, axis=1, keepdims=True)
    kap = np.full(K, kappa) * rng.uniform(0.5, 1.5, K)
    lam = rng.uniform(0.1, 1, K)
    lam /= lam.sum()
    from scipy.integrate import quad
    n = np.array([math.cos(0.3), math.sin(0.3)])
    full = quad(lambda t: oracle.mixture_pdf(2, mu, kap, lam, np.array([math.cos(t), math.sin(t)])),
                0, 2 * np.pi, limit=800, epsabs=1e-12)[0]
    assert full == pytest.approx(1.0, abs=1e-9)

    def refl(t):
        v = np.array([math.cos(t), math.sin(t)])
        vm = v - 2 * np.dot(v, n) * n
        return oracle.mixture_pdf(2, mu, kap, lam, v) + oracle.mixture_pdf(2, mu, kap, lam, vm)
    half = quad(refl, 0.3 - np.pi / 2, 0.3 + np.pi / 2, limit=800, epsabs=1e-12)[0]
    assert half == pytest.approx(1.0, abs=1e-9)
    # 3D mixture by Gauss-Legendre x uniform-phi quadrature
    mu3 = rng.normal(size=(K, 3))
    mu3 /= np.linalg.norm(mu3, axis=1, keepdims=True)
    kap3 = np.minimum(kap, 20.0)
    dirs, w = _sphere(200)
    vals = np.array([oracle.mixture_pdf(3, mu3, kap3, lam, d) for d in dirs])
    assert (vals * w).sum() == pytest.approx(1.0, abs=1e-6)
    n3 = np.array([0.0, 0.6, 0.8])
    up = dirs @ n3 > 0
    refl3 = np.array([oracle.mixture_pdf(3, mu3, kap3, lam, d) +
                      oracle.mixture_pdf(3, mu3, kap3, lam, d - 2 * np.dot(d, n3) * n3) for d in dirs[up]])
    assert (refl3 * w[up]).sum() == pytest.approx(1.0, abs=2e-3)  # hemisphere cut of a sphere grid


@pytest.mark.parametrize("kappa", [1e-4, 0.3, 2.0, 12.0, 400.0])
def test_vmf2_best_fisher_histogram_and_moment(kappa):
    key = [99, 5]
    n = 40000
    th = np.array([oracle.vmf2_sample_angle(kappa, key, i, 3, 1)[0] for i in range(n)])
    # first moment E[cos] = I1/I0
    m = np.cos(th).mean()
    A = special.i1e(kappa) / special.i0e(kappa)
    sd = np.sqrt(max(0.5 * (1 + special.ive(2, kappa) / special.i0e(kappa)) - A * A, 1e-12) / n)
    assert abs(m - A) < 5 * sd + 1e-12
    assert oracle.vmf_mean_cos(2, kappa) == pytest.approx(A, rel=1e-12)
    # chi-square against the density on 40 bins of the angle (scale-adapted)
    width = min(np.pi, 8 / math.sqrt(kappa))
    edges = np.linspace(-width, width, 41)
    h, _ = np.histogram(th, bins=edges)
    from scipy.integrate import quad
    mu = np.array([1.0, 0.0])
    f = lambda t: oracle.vmf_pdf(2, kappa, mu, np.array([math.cos(t), math.sin(t)]))
    p = np.array([quad(f, a, b)[0] for a, b in zip(edges[:-1], edges[1:])])
    e = p * n
    ok = e > 5
    chi2 = ((h[ok] - e[ok]) ** 2 / e[ok]).sum()
    assert chi2 < 90   # <= 39 dof, P(chi2 > 90) < 1e-5


@pytest.mark.parametrize("kappa", [1e-5, 0.2, 3.0, 40.0, 2000.0])
def test_vmf3_sampler_moment_and_histogram(kappa):
    rng = np.random.default_rng(1)
    mu = rng.normal(size=3)
    mu /= np.linalg.norm(mu)
    n = 40000
    u = rng.random((n, 2))
    nu = np.array([oracle.vmf3_sample(kappa, mu, a, b) for a, b in u])
    assert np.allclose(np.linalg.norm(nu, axis=1), 1, atol=1e-12)
    w = nu @ mu
    A = 1 / np.tanh(kappa) - 1 / kappa if kappa > 1e-3 else kappa / 3
    assert oracle.vmf_mean_cos(3, kappa) == pytest.approx(A, rel=1e-9, abs=1e-15)
    var_w = 1 - 2 * A / kappa - A * A if kappa > 1e-3 else 1 / 3
    assert abs(w.mean() - A) < 5 * math.sqrt(max(var_w, 1e-12) / n) + 1e-9
    # azimuth about mu is uniform
    b1, b2 = np.zeros(3), np.zeros(3)
    oracle.lib().orc_onb(mu.ctypes.data_as(oracle._dp), b1.ctypes.data_as(oracle._dp), b2.ctypes.data_as(oracle._dp))
    assert abs(np.dot(b1, mu)) < 1e-12 and abs(np.dot(b2, mu)) < 1e-12 and abs(np.dot(b1, b2)) < 1e-12
    ph = np.arctan2(nu @ b2, nu @ b1)
    h, _ = np.histogram(ph, bins=32, range=(-np.pi, np.pi))
    chi2 = ((h - n / 32) ** 2 / (n / 32)).sum()
    assert chi2 < 75
