"""The error of each result of the CUDA path against the FP64 oracle, stated
as numbers (printed as "PRECISION {...}" lines, run with -s): FP32 geometry
with FP64 re-tests, the FP16 hash grid + BF16 MLP decode (outputs, mixture
parameters after the normalisation map of Tab. reg_map, and the mixture
density they give), the FP32 mixture density and sampler given identical
parameters, the BF16 fused training backward, and the FP64-accumulated
estimates on the same random streams.  The bounds asserted here are the ones
the parity tests use; the printed figures are what is measured."""
import json

import numpy as np
import pytest

import oracle
import wost_inputs as wi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2410_18944_gb300 import api as a, build
    build.build()
    return a


def _report(name, **vals):
    print("PRECISION " + json.dumps({"result": name, **{k: float(v) for k, v in vals.items()}}))


def _interior(sc, n, seed, margin=0.05):
    O = oracle.Scene(sc)
    rng = np.random.default_rng(seed)
    lo, hi = sc.bbox
    out = []
    while len(out) < n:
        p = rng.uniform(lo, hi).astype(np.float32).astype(np.float64)
        if O.winding(p[None])[0] > 0.5 and O.closest_dirichlet(p[None])[1][0] > margin:
            out.append(p)
    return np.array(out)


def _scene(dim):
    if dim == 2:
        return wi.star_polyline(512, seed=7, neumann_frac=0.6)
    return wi.displaced_icosphere(subdiv=2, seed=4, neumann_frac=0.5, with_source=False)


@pytest.mark.parametrize("dim", [2, 3])
def test_precision_of_the_boundary_queries(api, dim):
    sc = _scene(dim)
    S, O = api.Scene(sc), oracle.Scene(sc)
    pts = _interior(sc, 1000 if dim == 2 else 400, 5 + dim, margin=1e-3)
    gi, gd = S.query_closest(pts)
    oi, od, _ = O.closest_dirichlet(pts)
    err = np.abs(gd.astype(np.float64) - od)
    rel = err / od
    scale = O.scale
    _report(f"closest Dirichlet distance {dim}D (FP32 traversal, FP64 re-test)", max_rel=rel.max(),
            median_rel=np.median(rel), max_abs_over_scale=err.max() / scale, same_index=np.mean(gi == oi))
    # the FP32 output of an FP64-exact distance, plus the FP32 rounding of
    # the query point's coordinates (absolute, relative to the scene)
    assert np.all(err <= (1e-6 if dim == 2 else 2e-6) * scale + (2e-7 if dim == 2 else 4e-7) * od)
    gk, gs = S.query_silhouette(pts)
    ok_, os_ = O.closest_silhouette(pts)
    both = (gk >= 0) & (ok_ >= 0) & np.isfinite(gs) & (os_ > 0)
    rs = np.abs(gs[both].astype(np.float64) - os_[both]) / os_[both]
    _report(f"closest silhouette distance {dim}D", p999_rel=np.quantile(rs, 0.999), median_rel=np.median(rs),
            found_by_both=np.mean(both))
    # exit-only ray casts of the walk step from the points, radius 2
    rng = np.random.default_rng(11 + dim)
    v = rng.normal(size=(len(pts), dim))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    v = v.astype(np.float32).astype(np.float64)
    gp, gt = S.query_ray(pts, v, 2.0, exit_only=True)
    op, ot = O.ray_neumann(pts, v, 2.0, exit_only=True)
    same = (gp == op) & (gp >= 0)
    rt = np.abs(gt[same].astype(np.float64) - ot[same]) / ot[same]
    _report(f"exit-only ray parameter {dim}D", max_rel=rt.max(), median_rel=np.median(rt),
            same_primitive=np.mean(gp == op))
    assert np.median(rt) < 1e-5


def _theta_all(OF, raw):
    mus, kaps, lams, cs = [], [], [], []
    for r in raw:
        mu, kap, lam, c = OF.theta(r)
        mus.append(mu)
        kaps.append(kap)
        lams.append(lam)
        cs.append(c)
    return np.array(mus), np.array(kaps), np.array(lams), np.array(cs)


@pytest.mark.parametrize("dim", [2, 3])
def test_precision_of_the_field_decode(api, dim):
    # the FP16 grid / BF16 MLP decode against the FP64 forward of the same
    # (rounded) parameters, then the mixture parameters and density they give
    lo, hi = [-1.5] * dim, [1.5] * dim
    F = api.Field(dim, lo, hi)
    fp = wi.random_field_params(dim, 3, lo, hi, log2T=F.desc.log2_table)
    fp["grid"] = wi.round_to_fp16(fp["grid"])
    for k in ("W1", "W2", "W3"):
        fp[k] = wi.round_to_bf16(fp[k])
    fp["b3"] = fp["b3"].astype(np.float32).astype(np.float64)
    F.set_params(fp["grid"], fp["W1"], fp["W2"], fp["W3"], fp["b3"])
    OF = oracle.Field(oracle.FieldParams(**fp))
    rng = np.random.default_rng(30 + dim)
    pts = rng.uniform(-1.4, 1.4, (500, dim))
    g = F.decode(pts).astype(np.float64)
    o = OF.forward(pts)
    rel_l2 = np.linalg.norm(g - o) / np.linalg.norm(o)
    _report(f"field decode raw outputs {dim}D (FP16 grid, BF16 MLP, FP32 accumulation)", rel_l2=rel_l2,
            max_abs_over_scale=np.abs(g - o).max() / np.abs(o).max())
    assert rel_l2 < 2e-2
    gm, gk, gl, gc = _theta_all(OF, g)
    om, ok_, ol, oc = _theta_all(OF, o)
    ang = np.degrees(np.arccos(np.clip((gm * om).sum(-1), -1, 1)))
    krel = np.abs(gk - ok_) / ok_
    _report(f"mixture parameters from the decode {dim}D", mu_angle_deg_median=np.median(ang),
            mu_angle_deg_max=ang.max(), kappa_rel_median=np.median(krel), kappa_rel_max=krel.max(),
            lambda_abs_max=np.abs(gl - ol).max(), c_abs_max=np.abs(gc - oc).max())
    # density at random directions, FP64 evaluation of both parameter sets
    prel = []
    for i in range(0, len(pts), 5):
        nu = rng.normal(size=dim)
        nu /= np.linalg.norm(nu)
        a = oracle.mixture_pdf(dim, gm[i], gk[i], gl[i], nu)
        b = oracle.mixture_pdf(dim, om[i], ok_[i], ol[i], nu)
        prel.append(abs(a - b) / b)
    prel = np.array(prel)
    _report(f"mixture density from the decode {dim}D", rel_median=np.median(prel), rel_p99=np.quantile(prel, 0.99))


@pytest.mark.parametrize("dim", [2, 3])
def test_precision_of_the_mixture_given_identical_parameters(api, dim):
    rng = np.random.default_rng(60 + dim)
    n, K = 3000, 8
    mu = rng.normal(size=(n, K, dim))
    mu /= np.linalg.norm(mu, axis=2, keepdims=True)
    kap = np.exp(rng.uniform(-8, np.log(200.0), (n, K)))
    lam = rng.uniform(0.05, 1, (n, K))
    lam /= lam.sum(1, keepdims=True)
    mu, kap, lam = mu.astype(np.float32), kap.astype(np.float32), lam.astype(np.float32)
    nu = mu[:, 0] + 0.05 * rng.normal(size=(n, dim))
    nu = (nu / np.linalg.norm(nu, axis=1, keepdims=True)).astype(np.float32)
    g = api.mixture_eval(dim, mu, kap, lam, nu)
    u = lambda a: np.asarray(a, float) / np.linalg.norm(np.asarray(a, float), axis=-1, keepdims=True)  # noqa: E731
    o = np.array([oracle.mixture_pdf(dim, u(mu[i]), kap[i].astype(float), lam[i].astype(float), u(nu[i]))
                  for i in range(n)])
    rel = np.abs(g - o) / o
    _report(f"mixture density given identical parameters {dim}D (FP32)", max_rel=rel.max(),
            median_rel=np.median(rel))
    assert rel.max() < 1e-5
    ctr = np.stack([np.arange(n), np.full(n, 3), np.full(n, 5)], 1).astype(np.uint32)
    seed = 0x1234567890
    gnu, _ = api.mixture_sample(dim, mu, kap, lam, ctr, seed)
    same = 0
    for i in range(n):
        _, onu = oracle.guided_draw(dim, u(mu[i]), kap[i].astype(float), lam[i].astype(float), 1.0,
                                    [seed & 0xFFFFFFFF, seed >> 32], int(ctr[i, 0]), int(ctr[i, 1]), int(ctr[i, 2]))
        same += np.linalg.norm(gnu[i] - onu) < 1e-4 * max(1.0, np.sqrt(kap[i].max()) / 10)
    _report(f"mixture samples given identical parameters {dim}D", same_draw=same / n,
            decision_flips=1 - same / n)
    assert same / n >= 0.995


@pytest.mark.parametrize("dim", [2, 3])
def test_precision_of_the_training_gradient(api, dim):
    sc = wi.half_disk(48, 12) if dim == 2 else wi.slab_box(2)
    lo, hi = sc.padded_bbox()
    for kind, w_scale, positive in (("active", 0.5, True), ("general", 0.5, False)):
        F = api.Field(dim, lo, hi)
        fp = wi.random_field_params(dim, 8, lo, hi, log2T=F.desc.log2_table, w_scale=w_scale)
        if positive:
            fp["grid"] = np.abs(fp["grid"]) + 0.05
            fp["W1"], fp["W2"] = np.abs(fp["W1"]), np.abs(fp["W2"])
        fp["grid"] = wi.round_to_fp16(fp["grid"])
        for k in ("W1", "W2", "W3"):
            fp[k] = wi.round_to_bf16(fp[k])
        fp["b3"] = fp["b3"].astype(np.float32).astype(np.float64)
        F.set_params(fp["grid"], fp["W1"], fp["W2"], fp["W3"], fp["b3"])
        OF = oracle.Field(oracle.FieldParams(**fp))
        pts = _interior(sc, 64, 8)
        r = oracle.solve(oracle.Scene(sc), oracle.make_params(eps=1e-3, maxsteps=256, seed=3, guided=1), pts, 0,
                         1, field=OF, records=True)
        recs = r["records"].astype(np.float32)
        F.set_records(recs)
        gl, gg = F.train_grad()
        ol, og, _ = OF.train_loss(recs.astype(np.float64))
        vals = {"loss_rel": abs(gl - ol) / abs(ol)}
        for name, ov in zip(["grid", "W1", "W2", "W3", "b3"], og):
            gv = gg[name].astype(np.float64).ravel()
            ov = ov.ravel()
            vals[f"{name}_cos"] = gv @ ov / (np.linalg.norm(gv) * np.linalg.norm(ov) + 1e-300)
            vals[f"{name}_rel_l2"] = np.linalg.norm(gv - ov) / (np.linalg.norm(ov) + 1e-300)
        _report(f"training gradient {dim}D, {kind} ReLUs (BF16 backward, hi/lo gradient tiles)", **vals)
        assert vals["loss_rel"] < 2e-2


@pytest.mark.parametrize("dim", [2, 3])
def test_precision_of_the_estimates_on_the_same_streams(api, dim):
    # FP64 per-point sums on both sides, the same Philox streams: the walks
    # coincide until an FP32 decision differs
    sc = wi.star_polyline(512, seed=2) if dim == 2 else wi.slab_box(3)
    S, O = api.Scene(sc), oracle.Scene(sc)
    pts = _interior(sc, 48, 3, margin=0.02)
    n = 2048
    m, v, st = api.solve(S, pts, n, eps=1e-3, maxsteps=256, seed=5)
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=256, seed=5), pts, 0, n)
    om, ov = oracle.mean_var(r["sum"], r["sum2"], n)
    z = np.abs(m - om) / np.sqrt(v + ov)
    _report(f"plain estimates {dim}D, {n} walks/point", median_abs_z=np.median(z), max_abs_z=z.max(),
            max_abs_diff_over_se=(np.abs(m - om) / np.sqrt(ov)).max(),
            walk_steps_rel=abs(st["walk_steps"] - r["steps"]) / r["steps"])
    assert np.all(z < 4.0)
