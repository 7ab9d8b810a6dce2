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


@pytest.mark.parametrize("dim,K", [(2, 8), (3, 8), (2, 16)])
def test_guided_mis_is_unbiased(dim, K):
    # any field gives an unbiased estimator under one-sample MIS (Sec. 4.4),
    # whatever its lobe count
    sc = wi.half_disk(48, 12) if dim == 2 else wi.slab_box(2)
    fld = _rand_field(sc, 2, L=4, log2T=12, base_res=4, max_res=16, w_scale=2.0, K=K)
    n = 3000 if dim == 2 else 1500
    _check_closed_form(sc, _interior(sc, 6, 8, margin=0.1), n, guided=True, field=fld, c_mode=0)
    # guiding only (c = 1): still unbiased, the mixture has full support; a
    # mild field keeps the weights 1/(|S| alpha p_g) light-tailed enough for
    # a z-test (a sharp field is unbiased too but its variance estimate is not
    # reliable at this sample count)
    mild = _rand_field(sc, 3, L=4, log2T=12, base_res=4, max_res=16, w_scale=0.3, grid_scale=0.1, K=K)
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


# ---------------------------------------------------------------------------
# nonzero Neumann flux: the -<N> term (Sec. 3.2, Eq. wost_estm)
# ---------------------------------------------------------------------------
def test_laplace_2d_neumann_flux_manufactured():
    # u = x^2 - y^2 + x y + y on the half disk, h = 1 + x on the flat edge
    sc = wi.half_disk_flux(64, 16)
    _check_closed_form(sc, _interior(sc, 10, 31, margin=0.1), 4000)


def test_poisson_2d_neumann_flux_manufactured():
    # u = x^2 + y^2 + y, f = 4, h = 1: source and flux terms together
    sc = wi.half_disk_flux(64, 16, poisson=True)
    _check_closed_form(sc, _interior(sc, 10, 32, margin=0.1), 4000)


def test_laplace_3d_neumann_flux_manufactured():
    # u = x^2 - y^2 + z + x z in the slab, h = (1 + x)(1 - 2z) on z = 0, 1
    sc = wi.slab_box_flux(3)
    _check_closed_form(sc, _interior(sc, 6, 33, margin=0.1), 2000)


def test_neumann_flux_sign():
    # the flux term with the opposite sign must break the match, and so
    # must dropping it (pins the sign and the presence of <N>)
    pts = np.array([[0.0, 0.15], [0.3, 0.25], [-0.4, 0.2]])
    for h in (wi.Fn(wi.FN_POLY2, [-1, -1, 0, 0, 0, 0, 0, 0, 0, 0]), wi.Fn()):
        sc = wi.half_disk_flux(64, 16)
        sc.h = h
        S = oracle.Scene(sc)
        r = oracle.solve(S, oracle.make_params(eps=1e-4, maxsteps=1024, seed=5), pts, 0, 4000)
        m, v = oracle.mean_var(r["sum"], r["sum2"], 4000)
        ex = wi.eval_fn(sc.exact, pts)
        assert np.all(np.abs(m - ex) / np.sqrt(v) > 8), (m, ex)


def test_neumann_sample_density_and_order_independence():
    # the <N> sample: the chosen primitive is a Neumann primitive closer than
    # r, W is the summed length of those, and the choice frequencies follow
    # length / W (chi-square over the candidates)
    sc = wi.half_disk_flux(64, 16)
    S = oracle.Scene(sc)
    x, r = np.array([0.05, 0.2]), 0.45
    V, P = sc.verts, sc.prims
    neu = np.nonzero(sc.bc == 1)[0]
    a, b = V[P[neu, 0]], V[P[neu, 1]]
    e = b - a
    t = np.clip(((x - a) * e).sum(1) / (e * e).sum(1), 0, 1)
    dist = np.linalg.norm(x - (a + t[:, None] * e), axis=1)
    cand = neu[dist < r]
    L = np.linalg.norm(e, axis=1)[dist < r]
    counts = {int(c): 0 for c in cand}
    n = 20000
    for w in range(n):
        i, z, W = S.neumann_sample(x, r, [7, 9], 3, w, 0)
        assert W == pytest.approx(L.sum(), rel=1e-12)
        counts[i] += 1
        sa, sb = V[P[i, 0]], V[P[i, 1]]
        # z on the chosen segment
        assert abs((z[0] - sa[0]) * (sb[1] - sa[1]) - (z[1] - sa[1]) * (sb[0] - sa[0])) < 1e-12
    obs = np.array([counts[int(c)] for c in cand])
    expct = n * L / L.sum()
    chi2 = ((obs - expct) ** 2 / expct).sum()
    assert chi2 < len(cand) + 6 * np.sqrt(2 * len(cand)), (chi2, len(cand))
    # nothing closer than r: no sample
    i, z, W = S.neumann_sample(np.array([0.0, 0.8]), 0.05, [7, 9], 3, 0, 0)
    assert i == -1 and W == 0


# ---------------------------------------------------------------------------
# Russian roulette beyond 128 steps (Sec. 6.1)
# ---------------------------------------------------------------------------
def test_russian_roulette_is_unbiased_where_the_cap_is_not():
    # thin annulus sector (width 0.1): about 200 steps per walk from the
    # middle; the hard cap at 128 steps closes long walks with g at the
    # closest Dirichlet point: biased
    sc = wi.annulus_sector()
    S = oracle.Scene(sc)
    pts = np.array([[0.95 * np.cos(a), 0.95 * np.sin(a)] for a in (0.6, 1.5, 2.3)])
    ex = wi.eval_fn(sc.exact, pts)
    nc = 6000
    r = oracle.solve(S, oracle.make_params(eps=1e-3, maxsteps=128, seed=21), pts, 0, nc)
    m, v = oracle.mean_var(r["sum"], r["sum2"], nc)
    assert r["truncated"] > 0.3 * nc * len(pts)
    assert np.abs((m - ex) / np.sqrt(v)).max() > 6, (m, ex)
    # roulette (survival 0.995, here from step 64 on so that most walks play
    # it) on the width-0.15 sector: unbiased against the closed form and
    # against uncapped walks, nothing truncated, shorter walks
    sc = wi.annulus_sector(r_in=0.85)
    S = oracle.Scene(sc)
    pts = pts * (0.925 / 0.95)
    ex = wi.eval_fn(sc.exact, pts)
    n = 2000
    r = oracle.solve(S, oracle.make_params(eps=1e-3, maxsteps=100000, seed=22, rr_depth=64, rr_survival=0.995),
                     pts, 0, n)
    m, v = oracle.mean_var(r["sum"], r["sum2"], n)
    assert r["truncated"] == 0
    assert np.all(np.abs((m - ex) / np.sqrt(v)) < 4.0), (m, ex)
    r2 = oracle.solve(S, oracle.make_params(eps=1e-3, maxsteps=100000, seed=122), pts, 0, n)
    m2, v2 = oracle.mean_var(r2["sum"], r2["sum2"], n)
    assert np.all(np.abs((m - m2) / np.sqrt(v + v2)) < 4.0)
    assert r["steps"] < 0.9 * r2["steps"]
    # a walk shorter than rr_depth steps is unchanged by roulette
    same = 0
    for wid in range(40):
        a = oracle.walk(S, oracle.make_params(eps=1e-3, maxsteps=100000, seed=23), 0, wid, pts[0])
        b = oracle.walk(S, oracle.make_params(eps=1e-3, maxsteps=100000, seed=23, rr_depth=64), 0, wid, pts[0])
        if a["steps"] <= 64:
            assert a["value"] == b["value"] and a["steps"] == b["steps"]
            same += 1
    assert same > 5


def test_russian_roulette_suffix_pass_carries_the_survival_weight():
    # records of a guided walk that plays roulette: v_k = w_k v_{k+1} + S_k
    # with the 1/q of a roulette step folded into w_k and S_k, so the first
    # record's target and the walk's value still satisfy the suffix relation
    sc = wi.annulus_sector(narc=256)
    sc.f = wi.Fn(wi.FN_CONST, [0.5])
    S = oracle.Scene(sc)
    lo, hi = sc.padded_bbox()
    fld = oracle.Field(oracle.FieldParams(**wi.random_field_params(2, 3, lo, hi, L=4, log2T=12, base_res=4,
                                                                    max_res=16, w_scale=0.5)))
    prm = oracle.make_params(eps=1e-3, maxsteps=100000, seed=23, guided=1, rr_depth=16, rr_survival=0.995)
    checked = 0
    for wid in range(40):
        o = oracle.walk(S, prm, 0, wid, np.array([0.0, 0.95]), field=fld, records=True)
        R, w, Sk = o["records"], o["w"], o["S"]
        if len(R) <= 16:
            continue
        v = o["last"]
        for k in range(len(R) - 1, -1, -1):
            assert R[k, 11] == pytest.approx(abs(v), rel=1e-12, abs=1e-300)
            v = w[k] * v + Sk[k]
        assert v == pytest.approx(o["value"], rel=1e-9, abs=1e-12)
        checked += 1
    assert checked > 5
