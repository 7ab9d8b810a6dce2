"""Many scenes in one launch (wost_batch_* / wost_solve_batch) through the C
ABI.  A job of a batch uses the same random streams as the same problem
solved alone, so the batch must reproduce the separate wost_solve calls up
to the order of FP64 atomic sums -- for plain walks and for guided walks with
frozen fields (including decode tiles that mix several jobs' fields).  With
online training the batch is checked against closed forms, and the training
step's Adam step count, kept on the device for graph replays, against the
FP64 Adam of the oracle."""
import ctypes as C

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


def _interior(sc, n, seed, margin=0.05):
    O = oracle.Scene(sc)
    rng = np.random.default_rng(seed)
    lo, hi = sc.bbox
    out = []
    while len(out) < n:
        p = rng.uniform(lo, hi, (4 * n, sc.dim))
        keep = (O.winding(p) > 0.5) & (O.closest_dirichlet(p)[1] > margin)
        out.extend(p[keep])
    return np.array(out[:n])


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


def _field(api, dim, seed, sc, w_scale=1.0):
    lo, hi = sc.padded_bbox()
    F = api.Field(dim, lo, hi)
    fp = wi.random_field_params(dim, seed, lo, hi, log2T=F.desc.log2_table, w_scale=w_scale)
    F.set_params(fp["grid"], fp["W1"], fp["W2"], fp["W3"], fp["b3"])
    return F


def _small_star_jobs(njobs, seed, pts=(40, 1500), wpp=(2, 12)):
    return wi.config_batch(njobs=njobs, seed=seed, seg_range=(64, 2048), points_range=pts, wpp_range=wpp)


def _compare_to_separate(api, jobs, specs, means, vars_, st, guided=False, **kw):
    steps = 0
    walks = 0
    for j, (job, spec) in enumerate(zip(jobs, specs)):
        if len(job.points) == 0:
            assert means[j].numel() == 0
            continue
        m, v, s = api.solve(spec["scene"], spec["points"], job.nwalks, eps=spec.get("eps", 1e-3),
                            maxsteps=spec.get("maxsteps", 128), seed=job.seed, guided=guided,
                            field=spec.get("field"), **kw)
        mb, vb = means[j].cpu().numpy(), vars_[j].cpu().numpy()
        m, v = m.cpu().numpy(), v.cpu().numpy()
        # the same walks: equal up to the order of the FP64 atomic sums
        assert np.allclose(mb, m, rtol=1e-9, atol=1e-12, equal_nan=True), (j, np.nanmax(np.abs(mb - m)))
        assert np.allclose(vb, v, rtol=1e-6, atol=1e-12, equal_nan=True), j
        steps += s["walk_steps"]
        walks += s["walks"]
    assert st["walk_steps"] == steps
    assert st["walks"] == walks


def test_plain_batch_equals_separate_solves(api):
    jobs = _small_star_jobs(7, seed=41)
    # empty jobs in the middle and at the end
    jobs.insert(3, wi.BatchJob(wi.star_polyline(128, seed=9), np.zeros((0, 2)), 4, seed=5))
    jobs.append(wi.BatchJob(wi.star_polyline(96, seed=10), np.zeros((0, 2)), 3, seed=6))
    specs = [dict(scene=api.Scene(j.scene), points=_dev(j.points.reshape(-1, 2)), nwalks=j.nwalks, seed=j.seed,
                  eps=1e-3, maxsteps=128) for j in jobs]
    means, vars_, st = api.solve_batch(specs)
    assert st["walk_launches"] == 1
    _compare_to_separate(api, jobs, specs, means, vars_, st)


def test_plain_batch_3d_equals_separate_solves(api):
    scenes = [wi.sphere_dirichlet(2), wi.slab_box(2), wi.sphere_dirichlet(3, g=wi.Fn(wi.FN_SQNORM))]
    scenes[2].f = wi.Fn(wi.FN_CONST, [6.0])
    jobs = []
    for i, sc in enumerate(scenes):
        sc.scene_id = 7 + i
        jobs.append(wi.BatchJob(sc, _interior(sc, [300, 37, 1200][i], 50 + i), [5, 17, 3][i], seed=90 + i))
    specs = [dict(scene=api.Scene(j.scene), points=_dev(j.points), nwalks=j.nwalks, seed=j.seed) for j in jobs]
    means, vars_, st = api.solve_batch(specs)
    _compare_to_separate(api, jobs, specs, means, vars_, st)


@pytest.mark.parametrize("dim", [2, 3])
def test_guided_frozen_batch_equals_separate_solves(api, dim):
    # few walks per job: every CTA holds walks of several jobs at once, so
    # decode tiles mix fields and take one MMA pass per job
    if dim == 2:
        jobs = _small_star_jobs(6, seed=43, pts=(30, 600), wpp=(2, 6))
    else:
        jobs = []
        for i, sc in enumerate([wi.slab_box(2), wi.sphere_dirichlet(2), wi.slab_box(3)]):
            sc.scene_id = 20 + i
            jobs.append(wi.BatchJob(sc, _interior(sc, [200, 90, 400][i], 60 + i), [3, 5, 2][i], seed=70 + i))
    specs = []
    for i, j in enumerate(jobs):
        specs.append(dict(scene=api.Scene(j.scene), points=_dev(j.points), nwalks=j.nwalks, seed=j.seed,
                          field=_field(api, dim, 300 + i, j.scene, w_scale=1.2)))
    means, vars_, st = api.solve_batch(specs, guided=True, train=0)
    assert st["walk_launches"] == 1
    _compare_to_separate(api, jobs, specs, means, vars_, st, guided=True)
    # the wide launch (28 walker warps per CTA) draws the same walks
    means, vars_, st = api.solve_batch(specs, guided=True, train=0, walker_warps=28)
    _compare_to_separate(api, jobs, specs, means, vars_, st, guided=True)


def test_guided_plan_tunes_the_walker_count(api):
    # the autotuner times 16 and 28 walker warps (three flush thresholds
    # each) unless exec fixes the count; either way the plan's results equal
    # those of the same plan at the other count
    jobs = _small_star_jobs(4, seed=53, pts=(40, 400), wpp=(2, 4))
    specs = [dict(scene=api.Scene(j.scene), points=_dev(j.points), nwalks=j.nwalks, seed=j.seed,
                  field=_field(api, 2, 500 + i, j.scene, w_scale=1.2)) for i, j in enumerate(jobs)]
    b = api.Batch(specs, guided=True, train=0)
    info = b.info()
    assert info["candidates"] == 6 and info["walker_warps"] in (16, 28)
    b.run()
    m_auto = [m.cpu().numpy().copy() for m in b.mean]
    b.close()
    other = 16 + 28 - info["walker_warps"]
    b2 = api.Batch(specs, guided=True, train=0, walker_warps=other)
    info2 = b2.info()
    assert info2["candidates"] == 3 and info2["walker_warps"] == other
    b2.run()
    for a, m in zip(m_auto, b2.mean):
        assert np.allclose(a, m.cpu().numpy(), rtol=1e-9, atol=1e-12)
    b2.close()
    with pytest.raises(Exception):
        api.Batch(specs, guided=True, train=0, walker_warps=20)


def test_guided_training_batch_is_unbiased(api):
    # half disks with a zero-flux flat edge: x^2 - y^2 is exact
    shapes = [(48, 12, 400, 24), (32, 8, 150, 40), (64, 16, 900, 12), (24, 6, 60, 30)]
    jobs, specs = [], []
    for i, (narc, nflat, n, wpp) in enumerate(shapes):
        sc = wi.half_disk(narc, nflat)
        sc.scene_id = 30 + i
        pts = _interior(sc, n, 80 + i)
        jobs.append(wi.BatchJob(sc, pts, wpp, seed=40 + i))
        S = api.Scene(sc)
        lo, hi = S.bbox()
        specs.append(dict(scene=S, points=_dev(pts), nwalks=wpp, seed=40 + i, maxsteps=512,
                          field=api.Field(2, lo, hi, seed=11 + i)))
    p0 = [s["field"].get_params() for s in specs]
    until = 16
    b = api.Batch(specs, guided=True, train=1, train_until_wpp=until)
    info = b.info()
    assert info["walk_launches"] == until + 1
    assert info["train_steps"] == sum(min(j.nwalks, until) for j in jobs)
    st = b.run()
    assert st["records"] > 0 and st["records_dropped"] == 0
    assert st["train_steps"] == info["train_steps"]
    zs = []
    for j, job in enumerate(jobs):
        m, v = b.mean[j].cpu().numpy(), b.var[j].cpu().numpy()
        ex = wi.eval_fn(job.scene.exact, job.points)
        zs.append((m - ex) / np.sqrt(v))
    z = np.concatenate(zs)
    assert np.mean(np.abs(z) < 4.5) > 0.98, np.sort(np.abs(z))[-10:]
    p1 = [s["field"].get_params() for s in specs]
    for a, c in zip(p0, p1):
        assert np.all(np.isfinite(c["W1"])) and np.all(np.isfinite(c["grid"]))
        assert not np.array_equal(a["W3"], c["W3"])     # each field trained
    # a replay keeps training the same fields
    b.run()
    p2 = [s["field"].get_params() for s in specs]
    assert all(not np.array_equal(a["W3"], c["W3"]) for a, c in zip(p1, p2))
    b.close()


def test_plan_replay_info_and_fixed_shape(api):
    jobs = _small_star_jobs(5, seed=47)
    specs = [dict(scene=api.Scene(j.scene), points=_dev(j.points), nwalks=j.nwalks, seed=j.seed) for j in jobs]
    b = api.Batch(specs)
    info = b.info()
    assert info["candidates"] >= 1 and 1 <= info["ctas_per_sm"] <= info["candidates"]
    assert info["best_ms"] <= info["worst_ms"] and info["graph_nodes"] >= 4 and info["walk_launches"] == 1
    s1 = b.run()
    m1 = [m.cpu().numpy().copy() for m in b.mean]
    s2 = b.run()
    for a, m in zip(m1, b.mean):
        assert np.allclose(a, m.cpu().numpy(), rtol=1e-9, atol=1e-12)
    assert s1["walk_steps"] == s2["walk_steps"]
    b.close()
    b2 = api.Batch(specs, ctas_per_sm=2)
    assert b2.info()["candidates"] == 0 and b2.info()["ctas_per_sm"] == 2
    b2.run()
    for a, m in zip(m1, b2.mean):
        assert np.allclose(a, m.cpu().numpy(), rtol=1e-9, atol=1e-12)
    b2.close()


def test_batch_rejects_invalid_jobs(api):
    from paper_2410_18944_gb300 import _lib
    s2 = api.Scene(wi.ngon(16))
    s3 = api.Scene(wi.sphere_dirichlet(1))
    p2 = _dev(np.zeros((4, 2)))
    p3 = _dev(np.full((4, 3), 0.1))
    with pytest.raises(_lib.WostError, match="same dimension"):
        api.Batch([dict(scene=s2, points=p2, nwalks=2), dict(scene=s3, points=p3, nwalks=2)])
    with pytest.raises(_lib.WostError, match="field per job"):
        api.Batch([dict(scene=s2, points=p2, nwalks=2)], guided=True)
    F = api.Field(2)
    with pytest.raises(_lib.WostError, match="distinct fields"):
        api.Batch([dict(scene=s2, points=p2, nwalks=2, field=F), dict(scene=s2, points=p2, nwalks=2, field=F)],
                  guided=True, train=1)
    with pytest.raises(_lib.WostError, match="nwalks"):
        api.Batch([dict(scene=s2, points=p2, nwalks=0)])


def test_adam_step_count_advances_on_device(api):
    # two training steps on fixed records against the FP64 Adam of the
    # oracle with t = 1, 2 (the step count lives on the device so that graph
    # replays advance it)
    sc = wi.half_disk(48, 12)
    F = _field(api, 2, 17, sc, w_scale=0.5)
    O = oracle.Scene(sc)
    lo, hi = sc.padded_bbox()
    fp = wi.random_field_params(2, 17, lo, hi, log2T=F.desc.log2_table, w_scale=0.5)
    OF = oracle.Field(oracle.FieldParams(**fp))
    pts = _interior(sc, 64, 12)
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=256, seed=3, guided=1), pts, 0, 1, field=OF,
                     records=True)
    F.set_records(r["records"].astype(np.float32))
    d = F.desc
    p = F.get_params()
    W3 = p["W3"].astype(np.float64).ravel().copy()
    m, v = np.zeros_like(W3), np.zeros_like(W3)
    big = None
    for t in (1, 2):
        _, g = F.train_grad()
        gw = g["W3"].astype(np.float64).ravel().copy()
        if big is None:
            big = np.abs(gw) > 1e-3 * np.abs(gw).max()
        oracle.adam(W3, gw, m, v, d.lr_mlp, d.beta1, d.beta2, d.adam_eps, t)
        F.train_step()
    got = F.get_params()["W3"].astype(np.float64).ravel()
    assert big.sum() > 100
    assert np.allclose(got[big], W3[big], rtol=0, atol=2e-6), np.abs(got[big] - W3[big]).max()
