"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle:
tensor-core operand layouts, boundary queries (bit-exact indices up to
floating-point near-ties), vMF mixture densities and samples, field decode,
plain and guided walks, and the training gradient."""
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


def _bf16(a):
    return wi.round_to_bf16(a)


# ---------------------------------------------------------------------------
# tensor-core operand layouts (the same descriptors the MLP kernels use)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("a_mn,b_mn", [(0, 0), (1, 1), (0, 1), (1, 0)])
@pytest.mark.parametrize("N,K", [(64, 32), (48, 64), (32, 128), (64, 128)])
def test_umma_layouts(api, a_mn, b_mn, N, K):
    rng = np.random.default_rng(N * 1000 + K + 7 * a_mn + 3 * b_mn)
    A = _bf16(rng.normal(size=(128, K)))
    B = _bf16(rng.normal(size=(N, K)))
    D = api.diag_umma(a_mn, b_mn, A, B)
    ref = A @ B.T
    assert np.allclose(D, ref, rtol=1e-5, atol=1e-4), np.abs(D - ref).max()


# ---------------------------------------------------------------------------
# queries
# ---------------------------------------------------------------------------
def _seg_dist(p, a, b):
    e = b - a
    t = np.clip(((p - a) * e).sum(-1) / (e * e).sum(-1), 0, 1)
    return np.linalg.norm(p - (a + t[..., None] * e), axis=-1)


def _tri_dist(p, tri):
    """FP64 point-triangle distance: projection if inside, else nearest edge."""
    a, b, c = tri
    n = np.cross(b - a, c - a)
    q = p - np.dot(p - a, n) / np.dot(n, n) * n
    w = [np.dot(np.cross(b - q, c - q), n), np.dot(np.cross(c - q, a - q), n), np.dot(np.cross(a - q, b - q), n)]
    if min(w) >= 0:
        return np.linalg.norm(p - q)
    return min(_seg_dist(p, u, v) for u, v in ((a, b), (b, c), (c, a)))


def test_closest_point_2d_parity(api):
    sc = wi.star_polyline(512, seed=5)
    S, O = api.Scene(sc), oracle.Scene(sc)
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1.3, 1.3, (4000, 2))
    gi, gd = S.query_closest(pts)
    oi, od, _ = O.closest_dirichlet(pts)
    scale = O.scale
    assert np.all(np.abs(gd - od) <= 1e-6 * scale + 2e-7 * od)
    mism = np.nonzero(gi != oi)[0]
    # a different index is accepted only for an FP32 near-tie
    for i in mism:
        a, b = sc.verts[sc.prims[gi[i], 0]], sc.verts[sc.prims[gi[i], 1]]
        assert sc.bc[gi[i]] == 0
        assert _seg_dist(pts[i], a, b) - od[i] <= 8 * 2 ** -24 * (od[i] + scale)
    assert len(mism) <= 0.002 * len(pts)


def test_closest_point_3d_parity(api):
    sc = wi.displaced_icosphere(subdiv=2, seed=3, with_source=False)
    S, O = api.Scene(sc), oracle.Scene(sc)
    rng = np.random.default_rng(1)
    pts = rng.uniform(-1.1, 1.1, (600, 3))
    gi, gd = S.query_closest(pts)
    oi, od, _ = O.closest_dirichlet(pts)
    scale = O.scale
    assert np.all(np.abs(gd - od) <= 2e-6 * scale + 4e-7 * od)
    mism = np.nonzero(gi != oi)[0]
    # closest points on shared edges / vertices tie exactly between the
    # adjacent triangles: a different index is accepted only for such a tie
    for i in mism:
        assert sc.bc[gi[i]] == 0
        assert _tri_dist(pts[i], sc.verts[sc.prims[gi[i]]]) - od[i] <= 8 * 2 ** -24 * (od[i] + scale)
    assert len(mism) <= 0.1 * len(pts)


# ---------------------------------------------------------------------------
# vMF mixtures
# ---------------------------------------------------------------------------
def _unit(a):
    """FP32 unit vectors renormalised in FP64 (the density lives on the
    sphere; an off-sphere input is ill-conditioned by kappa (|v| - 1))."""
    a = np.asarray(a, float)
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _rand_mixture(rng, n, dim, K=8, kmax=200.0):
    mu = rng.normal(size=(n, K, dim))
    mu /= np.linalg.norm(mu, axis=2, keepdims=True)
    kap = np.exp(rng.uniform(-8, np.log(kmax), (n, K)))
    lam = rng.uniform(0.05, 1, (n, K))
    lam /= lam.sum(1, keepdims=True)
    return mu.astype(np.float32), kap.astype(np.float32), lam.astype(np.float32)


@pytest.mark.parametrize("K", [8, 16])
@pytest.mark.parametrize("dim", [2, 3])
def test_mixture_pdf_parity(api, dim, K):
    rng = np.random.default_rng(10 + dim + 100 * (K // 16))
    n = 4000
    mu, kap, lam = _rand_mixture(rng, n, dim, K=K)
    nu = rng.normal(size=(n, dim))
    nu /= np.linalg.norm(nu, axis=1, keepdims=True)
    # half the directions close to a lobe mean (the density's bulk)
    nu[: n // 2] = mu[: n // 2, 0] + 0.05 * rng.normal(size=(n // 2, dim))
    nu /= np.linalg.norm(nu, axis=1, keepdims=True)
    nu = nu.astype(np.float32)
    g = api.mixture_eval(dim, mu, kap, lam, nu)
    # the density lives on the sphere: evaluate the oracle at the FP32
    # direction renormalised in FP64 (an off-sphere input is ill-conditioned
    # by kappa * (|nu| - 1))
    nu64 = _unit(nu)
    mu64 = _unit(mu)
    o = np.array([oracle.mixture_pdf(dim, mu64[i], kap[i].astype(float), lam[i].astype(float), nu64[i])
                  for i in range(n)])
    big = o > 1e-3 * o.max()
    rel = np.abs(g - o) / o
    assert np.all(rel[big] < 1e-5), rel[big].max()


@pytest.mark.parametrize("K", [8, 16])
@pytest.mark.parametrize("dim", [2, 3])
def test_mixture_sample_parity(api, dim, K):
    rng = np.random.default_rng(20 + dim + 100 * (K // 16))
    n = 4000
    mu, kap, lam = _rand_mixture(rng, n, dim, K=K, kmax=500.0)
    ctr = np.stack([np.arange(n), np.full(n, 3), np.full(n, 5)], 1).astype(np.uint32)
    seed = 0x1234567890
    gnu, gpdf = api.mixture_sample(dim, mu, kap, lam, ctr, seed)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    mu64 = _unit(mu)
    close = 0
    for i in range(n):
        hit, onu = oracle.guided_draw(dim, mu64[i], kap[i].astype(float), lam[i].astype(float), 1.0,
                                      key, int(ctr[i, 0]), int(ctr[i, 1]), int(ctr[i, 2]))
        assert hit == 1
        close += np.linalg.norm(gnu[i] - onu) < 1e-4 * max(1.0, np.sqrt(kap[i].max()) / 10)
        po = oracle.mixture_pdf(dim, mu64[i], kap[i].astype(float), lam[i].astype(float), _unit(gnu[i]))
        if po > 1e-3:
            assert abs(gpdf[i] - po) / po < 1e-5
    # the same counters give the same direction except near lobe-CDF or
    # rejection-test decision boundaries
    assert close / n >= 0.995, close / n


# ---------------------------------------------------------------------------
# field decode (hash grid + tcgen05 MLP) vs the FP64 field on identical
# low-precision parameters
# ---------------------------------------------------------------------------
def _field_pair(api, dim, seed, sc=None, positive=False, **kw):
    lo = [-1.5] * dim if sc is None else sc.padded_bbox()[0]
    hi = [1.5] * dim if sc is None else sc.padded_bbox()[1]
    F = api.Field(dim, lo, hi)
    fp = wi.random_field_params(dim, seed, lo, hi, log2T=F.desc.log2_table, **kw)
    if positive:
        fp["grid"] = np.abs(fp["grid"]) + 0.05
        fp["W1"], fp["W2"] = np.abs(fp["W1"]), np.abs(fp["W2"])
    fp["grid"] = wi.round_to_fp16(fp["grid"])
    for k in ("W1", "W2", "W3"):
        fp[k] = _bf16(fp[k])
    fp["b3"] = fp["b3"].astype(np.float32).astype(np.float64)
    F.set_params(fp["grid"], fp["W1"], fp["W2"], fp["W3"], fp["b3"])
    return F, oracle.Field(oracle.FieldParams(**fp)), fp


@pytest.mark.parametrize("dim", [2, 3])
def test_decode_parity(api, dim):
    F, OF, fp = _field_pair(api, dim, 3)
    rng = np.random.default_rng(30 + dim)
    pts = rng.uniform(-1.4, 1.4, (1000, dim))
    g = F.decode(pts)
    o = OF.forward(pts)
    err = np.abs(g - o)
    scale = np.abs(o).max()
    rel_l2 = np.linalg.norm(g - o) / np.linalg.norm(o)
    print(f"decode dim={dim}: rel-L2 {rel_l2:.2e}, max abs {err.max():.2e} (output scale {scale:.2f})")
    assert rel_l2 < 2e-2
    assert err.max() < 0.05 * scale


# ---------------------------------------------------------------------------
# walks
# ---------------------------------------------------------------------------
def _interior(sc, n, seed, margin=0.1):
    O = oracle.Scene(sc)
    rng = np.random.default_rng(seed)
    lo, hi = sc.bbox
    out = []
    while len(out) < n:
        p = rng.uniform(lo, hi)
        if O.winding(p[None])[0] > 0.5 and O.closest_dirichlet(p[None])[1][0] > margin:
            out.append(p)
    return np.array(out)


@pytest.mark.parametrize("name", ["ngon", "half_disk", "channel", "poisson2d", "sphere3d", "slab3d", "poisson3d"])
def test_plain_walk_closed_form(api, name):
    if name == "ngon":
        sc = wi.ngon(64)
    elif name == "half_disk":
        sc = wi.half_disk(64, 16)
    elif name == "channel":
        sc = wi.rectangle_channel()
    elif name == "poisson2d":
        sc = wi.half_disk(64, 16, g=wi.Fn(wi.FN_SQNORM))
        sc.f = wi.Fn(wi.FN_CONST, [4.0])
    elif name == "sphere3d":
        sc = wi.sphere_dirichlet(3)
    elif name == "slab3d":
        sc = wi.slab_box(3)
    else:
        sc = wi.sphere_dirichlet(3, g=wi.Fn(wi.FN_SQNORM))
        sc.f = wi.Fn(wi.FN_CONST, [6.0])
    pts = _interior(sc, 32, 1)
    S = api.Scene(sc)
    n = 20000
    m, v, st = api.solve(S, pts, n, eps=1e-4, maxsteps=4096, seed=11)
    ex = wi.eval_fn(sc.exact, pts)
    z = (m - ex) / np.sqrt(v)
    assert st["walks"] == n * len(pts)
    assert st["truncated"] == 0
    assert np.all(np.abs(z) < 4.0), z


def test_plain_walk_vs_oracle_star(api):
    sc = wi.star_polyline(512, seed=2)
    pts = _interior(sc, 48, 3, margin=0.02)
    S, O = api.Scene(sc), oracle.Scene(sc)
    n = 4096
    m, v, st = api.solve(S, pts, n, eps=1e-3, maxsteps=256, seed=5)
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=256, seed=5), pts, 0, n)
    om, ov = oracle.mean_var(r["sum"], r["sum2"], n)
    z = (m - om) / np.sqrt(v + ov)
    assert np.all(np.abs(z) < 4.0), z
    # same Philox streams: the walks coincide step for step until an FP32
    # decision differs, so the two estimates are far closer than independent ones
    assert np.median(np.abs(z)) < 0.3, np.median(np.abs(z))
    assert abs(st["walk_steps"] - r["steps"]) / r["steps"] < 0.02


def test_point_status(api):
    sc = wi.rectangle_channel()
    S = api.Scene(sc)
    pts = np.array([[0.0, 0.5], [3.0, 0.5], [1.0 - 5e-5, 0.5], [0.2, 0.7]])
    m, v, st = api.solve(S, pts, 64, eps=1e-4, maxsteps=512)
    assert np.isnan(m[1]) and v[2] == 0
    assert m[2] == pytest.approx(np.cosh(np.pi) * np.cos(np.pi * 0.5), abs=1e-5)
    assert st["walks"] == 64 * 2


def test_device_points_and_outputs(api):
    sc = wi.half_disk(48, 12)
    S = api.Scene(sc)
    pts = _interior(sc, 64, 4)
    m_h, v_h, _ = api.solve(S, pts, 256, eps=1e-3, seed=2)
    pd = torch.tensor(pts, dtype=torch.float64, device="cuda")
    m_d, v_d, _ = api.solve(S, pd, 256, eps=1e-3, seed=2)
    assert np.allclose(m_d.cpu().numpy(), m_h, rtol=1e-9, atol=1e-12)


# ---------------------------------------------------------------------------
# guided walks with a frozen field
# ---------------------------------------------------------------------------
def test_guided_c_zero_equals_plain(api):
    sc = wi.star_polyline(256, seed=4)
    S = api.Scene(sc)
    F, _, _ = _field_pair(api, 2, 5, sc)
    pts = _interior(sc, 64, 5, margin=0.02)
    mp, _, sp = api.solve(S, pts, 64, eps=1e-3, seed=9)
    mg, _, sg = api.solve(S, pts, 64, eps=1e-3, seed=9, guided=True, field=F, c_mode=1, c_fixed=0.0)
    assert np.allclose(mg, mp, rtol=1e-6, atol=1e-7)
    assert sg["walk_steps"] == sp["walk_steps"]


@pytest.mark.parametrize("dim,reflect", [(2, 1), (3, 1), (2, 0), (3, 0)])
def test_guided_frozen_field_vs_closed_form_and_oracle(api, dim, reflect):
    # reflect = 0: guided samples below the tangent plane at a Neumann point
    # are not reflected and end the walk's recursion (zero density), the
    # ablation of Sec. 4.3; still unbiased
    sc = wi.half_disk(48, 12) if dim == 2 else wi.slab_box(2)
    S, O = api.Scene(sc), oracle.Scene(sc)
    F, OF, _ = _field_pair(api, dim, 6, sc, w_scale=1.5)
    pts = _interior(sc, 24, 6)
    n = 8192 if dim == 2 else 4096
    m, v, st = api.solve(S, pts, n, eps=1e-3, maxsteps=1024, seed=7, guided=True, field=F, reflect=reflect)
    ex = wi.eval_fn(sc.exact, pts)
    z = (m - ex) / np.sqrt(v)
    assert np.all(np.abs(z) < 4.0), z
    no = 1024
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=1024, seed=7, guided=1, reflect=reflect), pts, 0, no,
                     field=OF)
    om, ov = oracle.mean_var(r["sum"], r["sum2"], no)
    zo = (m - om) / np.sqrt(v + ov)
    assert np.all(np.abs(zo) < 4.0), zo


# ---------------------------------------------------------------------------
# training gradient (fused tcgen05 backward) vs FP64 analytic gradient
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("dim,kind", [(2, "active"), (3, "active"), (2, "mild"), (3, "mild"), (2, "sharp"),
                                      (3, "sharp")])
def test_train_gradient_parity(api, dim, kind):
    # "active": non-negative grid, W1, W2 keep every ReLU active on both
    # sides, so the GPU and the FP64 forward share their masks and the
    # comparison isolates the fused backward (BF16 activations, hi/lo BF16
    # gradient tiles, FP32 accumulation).  "mild"/"sharp": general fields; a
    # BF16-rounded feature moves pre-activations by ~1e-3, flipping about 0.4
    # ReLU masks per record against the FP64 forward, each flip moving dX by
    # ~1/8 -- a few percent of rel-L2 on the grid and W1 gradients.
    sc = wi.half_disk(48, 12) if dim == 2 else wi.slab_box(2)
    F, OF, fp = _field_pair(api, dim, 8, sc, w_scale=1.5 if kind == "sharp" else 0.5,
                            positive=(kind == "active"))
    O = oracle.Scene(sc)
    pts = _interior(sc, 64, 8, margin=0.05)
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=256, seed=3, guided=1), pts, 0, 1, field=OF,
                     records=True)
    recs = r["records"]
    assert len(recs) > 300 and (recs[:, 9] == 1).any()
    recs32 = recs.astype(np.float32)
    F.set_records(recs32)
    gl, gg = F.train_grad()
    ol, og, _ = OF.train_loss(recs32.astype(np.float64))
    assert gl == pytest.approx(ol, rel=2e-2)
    for name, o in zip(["grid", "W1", "W2", "W3", "b3"], og):
        gv = gg[name].astype(np.float64).ravel()
        ov = o.ravel()
        cos = gv @ ov / (np.linalg.norm(gv) * np.linalg.norm(ov) + 1e-300)
        rel = np.linalg.norm(gv - ov) / (np.linalg.norm(ov) + 1e-300)
        print(f"grad {name} dim={dim}: cosine {cos:.6f} rel-L2 {rel:.3e}")
        if kind == "active":
            assert cos > 0.99995 and rel < 1e-2, (name, cos, rel)
        else:
            assert cos > 0.998 and rel < 6e-2, (name, cos, rel)
    # the training scatter of the coarse levels goes to several copies of
    # their gradient inside the unused entries of the level's table and sums
    # them back: those entries (past (N_l + 1)^d of a densely indexed level)
    # must come out exactly zero, as in the oracle
    d = F.desc
    T = 1 << d.log2_table
    g = gg["grid"].reshape(d.levels, T, d.features)
    dense_levels = 0
    for l, n in enumerate(wi.level_resolutions(d.levels, d.base_res, d.max_res)):
        V = (n + 1) ** dim
        if V <= T:
            dense_levels += 1
            assert not np.any(g[l, V:]), (l, V, np.count_nonzero(g[l, V:]))
    assert dense_levels >= 4


@pytest.mark.parametrize("dim", [2, 3])
def test_train_step_on_a_strided_subset(api, dim):
    # a training step of about m records takes the stratum o, o + k, ... of
    # the buffer (k = ceil(n / m), o = t * 2654435761 mod k with t the Adam
    # step count): the same loss and gradients as the explicit slice
    sc = wi.half_disk(48, 12) if dim == 2 else wi.slab_box(2)
    F, OF, fp = _field_pair(api, dim, 8, sc, w_scale=0.5, positive=True)
    O = oracle.Scene(sc)
    pts = _interior(sc, 96, 9, margin=0.05)
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=256, seed=4, guided=1), pts, 0, 1, field=OF,
                     records=True)
    recs = r["records"].astype(np.float32)
    n = len(recs)
    m = n // 5 + 3
    k = -(-n // m)
    assert k >= 2
    G = api.Field(dim, *sc.padded_bbox())

    def check(off):
        l_sub, g_sub = F.train_grad(samples=m)
        p = F.get_params()
        G.set_params(p["grid"], p["W1"], p["W2"], p["W3"], p["b3"])
        G.set_records(recs[off::k])
        l_ref, g_ref = G.train_grad()
        assert l_sub == pytest.approx(l_ref, rel=1e-5)
        for name in g_ref:
            a, b = g_sub[name].ravel(), g_ref[name].ravel()
            assert np.allclose(a, b, rtol=1e-4, atol=1e-6 * np.abs(b).max()), name
        return l_ref, g_ref

    F.set_records(recs)
    l0, g0 = check(0)
    ol, og, _ = OF.train_loss(recs[0::k].astype(np.float64))
    assert l0 == pytest.approx(ol, rel=2e-2)
    gv, ov = g0["W3"].astype(np.float64).ravel(), og[3].ravel()
    assert gv @ ov / (np.linalg.norm(gv) * np.linalg.norm(ov)) > 0.9999
    # one Adam step on the subset moves the stratum to o = 2654435761 mod k
    F.train_step(exec_=api.exec_defaults(train_samples=m))
    check(2654435761 % k)


def test_online_training_in_minibatches(api):
    # train_samples = m: after each batch of one walk per point the field
    # takes ceil(n / m) Adam steps over the batch's n records; the estimate
    # stays unbiased
    sc = wi.half_disk(48, 12)
    S = api.Scene(sc)
    pts = _interior(sc, 64, 12)
    F = api.Field(2, *sc.padded_bbox())
    m, v, st = api.solve(S, pts, 2048, eps=1e-3, maxsteps=256, seed=21, guided=True, field=F, train=1,
                         train_until_wpp=8, train_samples=256)
    n_rec = st["records"]                # records of the last training batch
    assert n_rec > 256 and st["train_steps"] >= 8 * 2
    F2 = api.Field(2, *sc.padded_bbox())
    m2, v2, st2 = api.solve(S, pts, 8, eps=1e-3, maxsteps=256, seed=21, guided=True, field=F2, train=1,
                            train_until_wpp=8, train_samples=0)
    assert st2["train_steps"] == 8
    ex = wi.eval_fn(sc.exact, pts)
    z = (m - ex) / np.sqrt(v)
    assert np.all(np.isfinite(m)) and np.all(np.abs(z) < 4.0), z


def test_online_training_runs_and_stays_unbiased(api):
    sc = wi.half_disk(48, 12)
    S = api.Scene(sc)
    lo, hi = S.bbox()
    F = api.Field(2, lo, hi)
    pts = _interior(sc, 256, 9)
    m, v, st = api.solve(S, pts, 64, eps=1e-3, maxsteps=512, seed=4, guided=True, field=F, train=1,
                         train_until_wpp=16)
    assert st["train_steps"] == 16
    ex = wi.eval_fn(sc.exact, pts)
    z = (m - ex) / np.sqrt(v)
    assert np.mean(np.abs(z) < 4.0) > 0.98
    p = F.get_params()
    assert np.all(np.isfinite(p["W1"])) and np.all(np.isfinite(p["grid"]))


def test_training_batches_of_several_walks_per_point(api):
    # batch_wpp = B: the field trains after each batch of B walks per point
    # (the last batch clipped at train_until_wpp), so every walk of the first
    # batch uses the initial field: the estimate equals a frozen-field solve.
    # The warp-specialised kernel runs a batch in one launch, the wavefront in
    # B launches of one walk per point; both gather the same records.
    sc = wi.half_disk(48, 12)
    S = api.Scene(sc)
    pts = _interior(sc, 256, 14)
    lo, hi = S.bbox()
    common = dict(eps=1e-3, maxsteps=256, seed=23, guided=True)
    F0 = api.Field(2, lo, hi, seed=5)
    m0, _, s0 = api.solve(S, pts, 4, field=F0, **common)
    init = F0.get_params()
    res = []
    for kern in (1, 2):
        F = api.Field(2, lo, hi, seed=5)
        m, v, st = api.solve(S, pts, 4, field=F, train=1, train_until_wpp=4, batch_wpp=16, guided_kernel=kern,
                             **common)
        assert st["train_steps"] == 1 and st["walk_steps"] == s0["walk_steps"]
        assert np.allclose(m, m0, rtol=1e-9, atol=1e-12)
        res.append((st["records"], F.get_params()))
    (r1, p1), (r2, p2) = res
    assert r1 == r2 and r1 > 4 * 200
    # one Adam step on the same records gathered in another order: equal up
    # to the order of the gradient sums (a first Adam step moves an entry by
    # about lr sign(g), so an entry whose sum cancels to rounding may differ)
    for k in ("W1", "W3", "grid"):
        assert not np.array_equal(p1[k], init[k])
        assert np.mean(np.isclose(p1[k], p2[k], rtol=1e-3, atol=1e-6)) > 0.999, k
    # batches of 16 and 8 walks per point, then 16 walks without training
    F = api.Field(2, lo, hi, seed=5)
    m, v, st = api.solve(S, pts, 40, field=F, train=1, train_until_wpp=24, batch_wpp=16, **common)
    assert st["train_steps"] == 2 and st["walks"] == 40 * s0["walks"] // 4
    ex = wi.eval_fn(sc.exact, pts)
    z = (m - ex) / np.sqrt(v)
    assert np.all(np.isfinite(m)) and np.mean(np.abs(z) < 4.0) > 0.98
    with pytest.raises(Exception):
        api.solve(S, pts, 2, field=F, train=1, batch_wpp=-1, **common)
    with pytest.raises(Exception):
        api.solve(S, pts, 2, field=F, walker_warps=20, **common)


def test_guided_walks_stay_inside_star(api):
    # A walker that rounding leaves a hair outside a Neumann segment next to
    # a reflex vertex must not take the neighbouring segment's entry
    # crossing as a hit (which flips its side and lets it wander off, where
    # the decoded mixture is meaningless): walks cast exit-only rays.
    # Uniform directions through the guided kernel (c = 0) reproduced such
    # escapes as NaN estimates on this scene before exit-only casts.
    sc, pts = wi.config_star_guided(res=512)
    S = api.Scene(sc)
    lo, hi = S.bbox()
    F = api.Field(2, lo, hi, seed=1)
    pd = torch.tensor(pts, dtype=torch.float64, device="cuda")
    for kw in (dict(c_mode=1, c_fixed=0.0), dict()):
        m, v, st = api.solve(S, pd, 8, eps=1e-3, maxsteps=128, guided=True, field=F, seed=7, **kw)
        assert np.all(np.isfinite(m.cpu().numpy())), kw
    mp, _, _ = api.solve(S, pd, 8, eps=1e-3, maxsteps=128, seed=7)
    mg, _, _ = api.solve(S, pd, 8, eps=1e-3, maxsteps=128, guided=True, field=F, seed=7, c_mode=1, c_fixed=0.0)
    assert np.allclose(mg.cpu().numpy(), mp.cpu().numpy(), rtol=1e-6, atol=1e-7)
    # every recorded walk position lies inside the boundary
    m, v, st = api.solve(S, pd, 1, eps=1e-3, maxsteps=128, guided=True, field=F, seed=8, c_mode=1, c_fixed=0.0,
                         train=1, walk_begin=3)
    rec = F.get_records()
    assert len(rec) > 1000 and np.all(np.isfinite(rec))
    x = rec[:, :2].astype(np.float64)
    onN = rec[:, 9] == 1
    # interior records: inside, up to rounding at the boundary
    off = x[~onN]
    out = off[~wi.inside_star_polygon(sc, off)]
    assert len(out) <= 1e-5 * len(off), len(out)
    if len(out):
        assert _seg_dist_all(sc, out).max() < 1e-5, out[:5]
    # records on the Neumann boundary: on a segment (a few ulps either side)
    rng = np.random.default_rng(0)
    onb = x[onN][rng.choice(int(onN.sum()), min(4000, int(onN.sum())), replace=False)]
    assert _seg_dist_all(sc, onb).max() < 1e-5


def _seg_dist_all(sc, pts):
    a = sc.verts[sc.prims[:, 0]]
    b = sc.verts[sc.prims[:, 1]]
    return np.array([_seg_dist(p[None], a, b).min() for p in pts])


@pytest.mark.parametrize("dim", [2, 3])
def test_wavefront_equals_warp_specialised(api, dim):
    # the two guided kernels draw the same random numbers and decode the same
    # FP16 rows, so with a frozen field their estimates agree up to the order
    # of the FP64 atomic sums; more walks than slots exercises slot refill,
    # the warp-specialised kernel runs with 16 and 28 walker warps, and the
    # automatic choice runs a frozen solve on the wavefront
    sc = wi.star_polyline(512, seed=3) if dim == 2 else wi.displaced_icosphere(subdiv=3, seed=4)
    S = api.Scene(sc)
    F, _, _ = _field_pair(api, dim, 21, sc, w_scale=1.2)
    pts = _interior(sc, 300, 13, margin=0.02)
    pd = torch.tensor(pts, dtype=torch.float64, device="cuda")
    out = []
    for kern, slots, ww in ((1, 0, 0), (1, 0, 28), (2, 0, 0), (2, 1000, 0), (0, 0, 0)):
        m, v, st = api.solve(S, pd, 24, eps=1e-3, maxsteps=256, guided=True, field=F, seed=31, guided_kernel=kern,
                             wavefront_slots=slots, walker_warps=ww)
        out.append((m.cpu().numpy(), v.cpu().numpy(), st))
    m1, v1, s1 = out[0]
    for m0, v0, s0 in out[1:]:
        assert s0["walk_steps"] == s1["walk_steps"] and s0["walks"] == s1["walks"]
        assert np.allclose(m0, m1, rtol=1e-9, atol=1e-12)
        assert np.allclose(v0, v1, rtol=1e-6, atol=1e-12)
