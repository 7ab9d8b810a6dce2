"""Edge cases of the CUDA path through the C ABI, against the FP64 oracle:
empty inputs, point counts that leave ragged warps, tiles and CTAs, a single
walk per point, a zero step cap, and decode batches whose last 128-row tile
is partial (every row of a tensor-core tile is independent, so a point
decodes to the same outputs alone or in any batch)."""
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
        p = rng.uniform(lo, hi).astype(np.float32).astype(np.float64)
        if O.winding(p[None])[0] > 0.5 and O.closest_dirichlet(p[None])[1][0] > margin:
            out.append(p)
    return np.array(out).reshape(n, sc.dim)


def _constant_field(api, dim, sc, seed, K=8):
    """Identical mixture parameters on both sides: a zero last layer and an
    FP16-representable bias, so the tensor-core decode returns the bias."""
    lo, hi = sc.padded_bbox()
    fp = wi.random_field_params(dim, seed, lo, hi, log2T=16 if dim == 2 else 19, K=K)
    rng = np.random.default_rng(seed)
    fp["W3"] = np.zeros_like(fp["W3"])
    fp["b3"] = wi.round_to_fp16(np.concatenate([rng.normal(size=K * dim), rng.uniform(-2.0, 1.0, K),
                                                rng.uniform(-1.0, 1.0, K), [-0.5]]))
    fp["grid"] = wi.round_to_fp16(fp["grid"])
    fp["W1"], fp["W2"] = wi.round_to_bf16(fp["W1"]), wi.round_to_bf16(fp["W2"])
    F = api.Field(dim, lo, hi, lr_grid=0.0, lr_mlp=0.0, K=K)
    F.set_params(fp["grid"], fp["W1"], fp["W2"], fp["W3"], fp["b3"])
    return F, oracle.Field(oracle.FieldParams(**fp))


@pytest.mark.parametrize("dim", [2, 3])
def test_empty_inputs(api, dim):
    sc = wi.half_disk(16, 4) if dim == 2 else wi.slab_box(1)
    S = api.Scene(sc)
    F = api.Field(dim, *sc.padded_bbox())
    none = np.zeros((0, dim))
    for guided in (False, True):
        m, v, st = api.solve(S, none, 8, guided=guided, field=F if guided else None, train=1 if guided else 0)
        assert m.shape == (0,) and v.shape == (0,)
        assert st["walks"] == 0 and st["walk_steps"] == 0 and st["train_steps"] == 0
    # device tensors of no rows
    md, vd, _ = api.solve(S, torch.zeros((0, dim), dtype=torch.float64, device="cuda"), 8)
    assert md.numel() == 0 and vd.numel() == 0
    assert F.decode(none).shape == (0, F.nout)
    idx, d = S.query_closest(none)
    assert idx.shape == (0,) and d.shape == (0,)


@pytest.mark.parametrize("n", [1, 31, 33, 129, 257])
def test_ragged_point_counts_plain_and_guided_vs_oracle(api, n):
    # point counts off the warp (32), tile (128) and CTA sizes: every point
    # draws its own streams, so the GPU and the oracle agree walk for walk
    sc = wi.star_polyline(256, seed=3, neumann_frac=0.4)
    S, O = api.Scene(sc), oracle.Scene(sc)
    pts = _interior(sc, n, 100 + n)
    nw, eps, maxsteps = 256, 1e-3, 256
    m, v, st = api.solve(S, pts, nw, eps=eps, maxsteps=maxsteps, seed=21)
    r = oracle.solve(O, oracle.make_params(eps=eps, maxsteps=maxsteps, seed=21), pts, 0, nw)
    om, ov = oracle.mean_var(r["sum"], r["sum2"], nw)
    z = (m - om) / np.sqrt(v + ov + 1e-300)
    assert st["walks"] == n * nw
    assert np.all(np.abs(z) < 4.0) and np.median(np.abs(z)) < 0.3, z
    F, OF = _constant_field(api, 2, sc, 30 + n)
    for kernel in (1, 2):   # warp-specialised, wavefront
        mg, vg, stg = api.solve(S, pts, 64, eps=eps, maxsteps=maxsteps, seed=22, guided=True, field=F,
                                guided_kernel=kernel)
        rg = oracle.solve(O, oracle.make_params(eps=eps, maxsteps=maxsteps, seed=22, guided=1), pts, 0, 64,
                          field=OF)
        gm, gv = oracle.mean_var(rg["sum"], rg["sum2"], 64)
        zg = (mg - gm) / np.sqrt(vg + gv + 1e-300)
        assert stg["walks"] == n * 64
        assert np.all(np.abs(zg) < 4.0) and np.median(np.abs(zg)) < 0.3, (kernel, zg)


def test_single_walk_per_point_matches_the_oracle_walk(api):
    # one walk per point: the estimate is that walk's value (variance 0 by
    # convention: no sample variance from one sample), equal to the oracle's
    # walk on the same stream wherever the two walks take the same steps
    sc = wi.half_disk(48, 12)
    S, O = api.Scene(sc), oracle.Scene(sc)
    pts = _interior(sc, 200, 7)
    prm = oracle.make_params(eps=1e-3, maxsteps=256, seed=9)
    m, v, st = api.solve(S, pts, 1, eps=1e-3, maxsteps=256, seed=9)
    assert np.all(v == 0.0) and st["walks"] == len(pts)
    same = 0
    for i in range(len(pts)):
        o = oracle.walk(O, prm, i, 0, pts[i])
        same += abs(m[i] - o["value"]) <= 1e-5 * max(1.0, abs(o["value"]))
    assert same >= 0.97 * len(pts), same


@pytest.mark.parametrize("dim", [2, 3])
def test_zero_step_cap_returns_g_at_the_closest_point(api, dim):
    # maxsteps 0: every walk is truncated before its first move and closed
    # with g at the closest Dirichlet point, the oracle's cap rule
    sc = wi.half_disk(48, 12) if dim == 2 else wi.sphere_dirichlet(2)
    S, O = api.Scene(sc), oracle.Scene(sc)
    pts = _interior(sc, 100, 8 + dim)
    m, v, st = api.solve(S, pts, 4, eps=1e-3, maxsteps=0, seed=3)
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=0, seed=3), pts, 0, 4)
    om, _ = oracle.mean_var(r["sum"], r["sum2"], 4)
    assert st["truncated"] == 4 * len(pts) and r["truncated"] == 4 * len(pts)
    # four equal samples: variance zero up to the rounding of the FP64 sums
    assert np.all(v <= 1e-12 * (m * m + 1e-30)), v.max()
    assert np.allclose(m, om, rtol=1e-5, atol=1e-6), np.abs(m - om).max()


@pytest.mark.parametrize("dim", [2, 3])
def test_decode_of_partial_tiles_is_row_independent(api, dim):
    sc = wi.half_disk(16, 4) if dim == 2 else wi.slab_box(1)
    lo, hi = sc.padded_bbox()
    F = api.Field(dim, lo, hi)
    fp = wi.random_field_params(dim, 12, lo, hi, log2T=F.desc.log2_table, w_scale=0.5)
    fp["grid"] = wi.round_to_fp16(np.abs(fp["grid"]) + 0.05)
    fp["W1"], fp["W2"] = np.abs(fp["W1"]), np.abs(fp["W2"])
    for k in ("W1", "W2", "W3"):
        fp[k] = wi.round_to_bf16(fp[k])
    fp["b3"] = fp["b3"].astype(np.float32).astype(np.float64)
    F.set_params(fp["grid"], fp["W1"], fp["W2"], fp["W3"], fp["b3"])
    OF = oracle.Field(oracle.FieldParams(**fp))
    pts = np.random.default_rng(40 + dim).uniform(lo, hi, (300, dim))
    full = F.decode(pts)
    for n in (1, 127, 129, 257):
        part = F.decode(pts[:n])
        assert np.array_equal(part, full[:n]), n
    o = OF.forward(pts)
    assert np.linalg.norm(full - o) / np.linalg.norm(o) < 2e-2


@pytest.mark.parametrize("dim", [2, 3])
def test_launch_order_changes_no_estimate(api, dim):
    # guided launches hand out their points longest walks first, by the walk
    # lengths of the scene's previous launch on as many points; with a
    # frozen field each launch holds one walk per point, so the per-point
    # sums add the same values in the same order whatever the order of the
    # points: a fresh scene, the same scene again (its first launch already
    # ordered) and a second scene must give identical estimates, and every
    # point must get all of its walks
    sc = wi.star_polyline(512, seed=4, neumann_frac=0.4) if dim == 2 else wi.slab_box(2)
    S1, S2 = api.Scene(sc), api.Scene(sc)
    F, _ = _constant_field(api, dim, sc, 70 + dim)
    pts = _interior(sc, 300, 80 + dim)
    kw = dict(eps=1e-3, maxsteps=256, seed=33, guided=True, field=F, guided_kernel=1)
    m1, v1, st1 = api.solve(S1, pts, 8, **kw)
    m2, v2, st2 = api.solve(S1, pts, 8, **kw)
    m3, v3, st3 = api.solve(S2, pts, 8, **kw)
    assert st1["walks"] == st2["walks"] == st3["walks"] == 8 * len(pts)
    assert st1["walk_steps"] == st2["walk_steps"] == st3["walk_steps"]
    assert np.array_equal(m1, m2) and np.array_equal(m1, m3)
    assert np.array_equal(v1, v2) and np.array_equal(v1, v3)
