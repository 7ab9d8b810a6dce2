"""Pins of the oracle's walk on stars (Sec. 3.2, 4.1, 4.3, 4.4) against
closed-form solutions of the Laplace/Poisson problem (Eq. linear_elliptic)
and against invariants of the estimator."""
import numpy as np
import pytest

import oracle
import wost_inputs as wi


def _check_closed_form(sc, pts, nwalks, eps=1e-4, guided=False, field=None, c_mode=0, c_fixed=0.5,
                       seed=3, zmax=4.5, maxsteps=1024):
    S = oracle.Scene(sc)
    prm = oracle.make_params(eps=eps, maxsteps=maxsteps, guided=int(guided), c_mode=c_mode,
                             c_fixed=c_fixed, seed=seed)
    r = oracle.solve(S, prm, pts, 0, nwalks, field=field)
    m, v = oracle.mean_var(r["sum"], r["sum2"], nwalks)
    ex = wi.eval_fn(sc.exact, pts)
    z = (m - ex) / np.sqrt(v + 1e-300)
    # epsilon-shell bias is O(eps |grad u|); it is far below the tolerance here
    assert np.all(np.abs(z) < zmax), (z, m, ex)
    assert r["truncated"] == 0
    return r


def _interior(sc, n, seed, margin=0.15):
    rng = np.random.default_rng(seed)
    lo, hi = sc.bbox
    out = []
    S = oracle.Scene(sc)
    while len(out) < n:
        p = rng.uniform(lo, hi)
        if S.winding(p[None])[0] > 0.5 and S.closest_dirichlet(p[None])[1][0] > margin:
            out.append(p)
    return np.array(out)


def test_laplace_2d_ngon_exp_cos():
    sc = wi.ngon(64)
    _check_closed_form(sc, _interior(sc, 12, 0), 6000)


def test_laplace_2d_neumann_half_disk():
    sc = wi.half_disk(64, 16)
    pts = _interior(sc, 12, 1, margin=0.1)
    _check_closed_form(sc, pts, 4000)


def test_laplace_2d_two_neumann_walls():
    sc = wi.rectangle_channel()
    _check_closed_form(sc, _interior(sc, 10, 2, margin=0.1), 4000)


def test_poisson_2d_manufactured_with_neumann():
    # u = |x|^2: Laplacian 4, du/dy = 0 on the flat Neumann edge
    sc = wi.half_disk(64, 16, g=wi.Fn(wi.FN_SQNORM))
    sc.f = wi.Fn(wi.FN_CONST, [4.0])
    _check_closed_form(sc, _interior(sc, 10, 3, margin=0.1), 4000)


def test_poisson_source_sign_and_scale():
    # flipping the source sign must break the match (pins the sign of <S>)
    sc = wi.half_disk(64, 16, g=wi.Fn(wi.FN_SQNORM))
    sc.f = wi.Fn(wi.FN_CONST, [-4.0])
    S = oracle.Scene(sc)
    pts = np.array([[0.0, 0.3], [0.2, 0.5]])
    r = oracle.solve(S, oracle.make_params(eps=1e-4, maxsteps=1024, seed=5), pts, 0, 4000)
    m, v = oracle.mean_var(r["sum"], r["sum2"], 4000)
    ex = wi.eval_fn(sc.exact, pts)
    assert np.all(np.abs(m - ex) / np.sqrt(v) > 10)


def test_laplace_3d_sphere_inverse_distance():
    sc = wi.sphere_dirichlet(2)
    _check_closed_form(sc, _interior(sc, 6, 4, margin=0.2), 2000)


def test_laplace_3d_slab_two_neumann_planes():
    sc = wi.slab_box(3)
    _check_closed_form(sc, _interior(sc, 6, 5, margin=0.1), 2000)


def test_poisson_3d_manufactured():
    sc = wi.sphere_dirichlet(2, g=wi.Fn(wi.FN_SQNORM))
    sc.f = wi.Fn(wi.FN_CONST, [6.0])
    _check_closed_form(sc, _interior(sc, 6, 6, margin=0.2), 2000)


def _rand_field(sc, seed, **kw):
    lo, hi = sc.padded_bbox()
    return oracle.Field(oracle.FieldParams(**wi.random_field_params(sc.dim, seed, lo, hi, **kw)))


def test_guided_with_c_zero_equals_plain_draw_for_draw():
    sc = wi.star_polyline(256, seed=4)
    S = oracle.Scene(sc)
    fld = _rand_field(sc, 1)
    pts = _interior(sc, 8, 7, margin=0.05)
    for pid, p in enumerate(pts):
        for wid in range(20):
            a = oracle.walk(S, oracle.make_params(seed=9), pid, wid, p)
            b = oracle.walk(S, oracle.make_params(seed=9, guided=1, c_mode=1, c_fixed=0.0), pid, wid, p, field=fld)
            assert a["value"] == b["value"] and a["steps"] == b["steps"]


@pytest.mark.parametrize("dim", [2, 3])
def test_guided_mis_is_unbiased(dim):
    # any field gives an unbiased estimator under one-sample MIS (Sec. 4.4)
    sc = wi.half_disk(48, 12) if dim == 2 else wi.slab_box(2)
    fld = _rand_field(sc, 2, L=4, log2T=12, base_res=4, max_res=16, w_scale=2.0)
    n = 3000 if dim == 2 else 1500
    _check_closed_form(sc, _interior(sc, 6, 8, margin=0.1), n, guided=True, field=fld, c_mode=0)
    # guiding only (c = 1): still unbiased, the mixture has full support; a
    # mild field keeps the weights 1/(|S| alpha p_g) light-tailed enough for
    # a z-test (a sharp field is unbiased too but its variance estimate is not
    # reliable at this sample count)
    mild = _rand_field(sc, 3, L=4, log2T=12, base_res=4, max_res=16, w_scale=0.3, grid_scale=0.1)
    _check_closed_form(sc, _interior(sc, 4, 9, margin=0.1), n, guided=True, field=mild, c_mode=1,
                       c_fixed=1.0)


def test_records_and_suffix_pass():
    # all-Dirichlet harmonic problem, plain weights (=1): every record's
    # target equals |terminal value| = |walk estimate|
    sc = wi.ngon(32)
    S = oracle.Scene(sc)
    fld = _rand_field(sc, 3)
    prm = oracle.make_params(seed=4, guided=1, c_mode=1, c_fixed=0.0)
    for wid in range(10):
        w = oracle.walk(S, prm, 0, wid, np.array([0.1, 0.2]), field=fld, records=True)
        R = w["records"]
        assert len(R) == w["steps"] - 1
        assert np.allclose(R[:, 11], abs(w["value"]), rtol=1e-14)
        assert np.allclose(R[:, 10], 1 / (2 * np.pi))
    # guided on a Neumann problem: directions are unit, leave Neumann points
    # into the domain, and q = p~ > 0
    sc = wi.half_disk(48, 12)
    S = oracle.Scene(sc)
    fld = _rand_field(sc, 4)
    prm = oracle.make_params(seed=5, guided=1)
    allr = []
    for wid in range(40):
        allr.append(oracle.walk(S, prm, 0, wid, np.array([0.1, 0.05]), field=fld, records=True)["records"])
    R = np.concatenate(allr)
    assert np.allclose(np.linalg.norm(R[:, 3:5], axis=1), 1)
    on = R[:, 9] == 1
    assert on.any()
    assert np.all((R[on, 3:5] * R[on, 6:8]).sum(1) > 0)
    assert np.all(R[:, 10] > 0)


def test_truncation_and_point_status():
    sc = wi.rectangle_channel()
    S = oracle.Scene(sc)
    prm = oracle.make_params(eps=1e-4, maxsteps=3, seed=1)
    r = oracle.solve(S, prm, np.array([[0.0, 0.5]]), 0, 200)
    assert r["truncated"] > 150 and r["steps"] <= 200 * 4
    st, val = S.point_status(np.array([[0.0, 0.5], [3.0, 0.5], [1.0 - 5e-5, 0.5]]), 1e-4)
    assert list(st) == [0, 2, 1]
    assert np.isnan(val[1]) and val[2] == pytest.approx(np.cosh(np.pi) * np.cos(np.pi * 0.5), abs=1e-9)
