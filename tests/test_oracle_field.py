"""Pins of the oracle's neural field (Sec. 5.2) and normalisation map
(Tab. reg_map): level resolutions, exact reproduction of affine lattice data
by the interpolation, hashing into the table, the ReLU MLP through a
positive-orthant identity, and the ranges of the mapped parameters."""
import numpy as np
import pytest

import oracle
import wost_inputs as wi


def _field(dim=2, seed=0, **kw):
    fp = wi.random_field_params(dim, seed, lo=[-1.5] * dim, hi=[1.5] * dim, **kw)
    return oracle.FieldParams(**fp)


def test_level_resolutions():
    f = oracle.Field(_field(2))
    res = [f.level_res(l) for l in range(16)]
    assert res[0] == 16 and res[-1] == 2048
    assert all(b > a for a, b in zip(res, res[1:]))
    ratios = np.array(res[1:]) / np.array(res[:-1])
    assert np.allclose(ratios, 128 ** (1 / 15), atol=0.08)
    f3 = oracle.Field(_field(3, max_res=512))
    assert f3.level_res(15) == 512


def test_interpolation_reproduces_affine_lattice_data():
    # On a densely indexed level, lattice values a.i + b (i = integer vertex
    # coordinates) are reproduced exactly for any x by multilinear
    # interpolation: feature = a.(u N) + b with u the unit-box coordinate.
    for dim in (2, 3):
        fp = _field(dim, L=4, log2T=16 if dim == 2 else 18, base_res=8, max_res=32)
        T = 1 << fp.log2T
        f0 = oracle.Field(fp)
        rng = np.random.default_rng(dim)
        a = rng.normal(size=dim)
        b = 0.3
        grid = np.zeros((fp.L, T, fp.F))
        for l in range(fp.L):
            N = f0.level_res(l)
            side = N + 1
            assert side ** dim <= T
            idx = np.arange(side ** dim)
            coords = [(idx // side ** k) % side for k in range(dim)]
            val = sum(a[k] * coords[k] for k in range(dim)) + b
            grid[l, :side ** dim, 0] = val
            grid[l, :side ** dim, 1] = -2 * val
        fp.grid = grid
        f = oracle.Field(fp)
        x = rng.uniform(-1.4, 1.4, (50, dim))
        feat = f.encode(x).reshape(50, fp.L, fp.F)
        u = (x - fp.lo) / (fp.hi - fp.lo)
        for l in range(fp.L):
            N = f.level_res(l)
            ref = (u * N) @ a + b
            assert np.allclose(feat[:, l, 0], ref, atol=1e-12)
            assert np.allclose(feat[:, l, 1], -2 * ref, atol=1e-12)


def test_hashed_levels_use_the_table_and_are_continuous():
    fp = _field(2, seed=3)
    f = oracle.Field(fp)
    # a hashed level (2049^2 > 2^16): perturbing one table entry changes the
    # feature only for points whose cell corners hash to it; and the encoding
    # is continuous across cell boundaries
    rng = np.random.default_rng(0)
    x = rng.uniform(-1.2, 1.2, (20, 2))
    e0 = f.encode(x)
    dx = 1e-9
    e1 = f.encode(x + dx)
    assert np.abs(e1 - e0).max() < 1e-4
    fp2 = _field(2, seed=3)
    fp2.grid = fp.grid.copy()
    fp2.grid[15] = 0.0
    f2 = oracle.Field(fp2)
    e2 = f2.encode(x).reshape(20, 16, 2)
    assert np.all(e2[:, 15] == 0) and np.any(e2[:, 14] != 0)


def test_mlp_positive_orthant_is_a_matrix_product():
    # With non-negative weights and features every ReLU is the identity, so
    # the network equals W3 W2 W1 feat + b3 (associativity, no per-layer loop).
    fp = _field(2, seed=5)
    fp.grid = np.abs(fp.grid)
    fp.W1, fp.W2 = np.abs(fp.W1), np.abs(fp.W2)
    f = oracle.Field(fp)
    x = np.random.default_rng(1).uniform(-1, 1, (10, 2))
    raw = f.forward(x)
    feat = f.encode(x)
    M = fp.W3 @ (fp.W2 @ fp.W1)
    assert np.allclose(raw, feat @ M.T + fp.b3, rtol=1e-12, atol=1e-12)
    # and negating W1 kills every hidden unit: output = b3
    fp.W1 = -fp.W1
    assert np.allclose(oracle.Field(fp).forward(x), fp.b3[None], atol=0)


def test_theta_map_ranges():
    fp = _field(3, seed=7)
    f = oracle.Field(fp)
    rng = np.random.default_rng(2)
    for _ in range(20):
        raw = rng.normal(size=fp.nout) * 5
        mu, kap, lam, c = f.theta(raw)
        assert np.allclose(np.linalg.norm(mu, axis=1), 1)
        assert np.all(kap >= np.exp(-8) * (1 - 1e-15)) and np.all(kap <= np.exp(8) * (1 + 1e-15))
        assert lam.sum() == pytest.approx(1) and np.all(lam > 0)
        assert 0 < c < 1
        K, d = fp.K, fp.dim
        # kappa' inside the clamp maps through exp; lambda is invariant to a shift of lambda'
        i = np.abs(raw[K * d:K * d + K]) < 8
        assert np.allclose(np.log(kap[i]), raw[K * d:K * d + K][i])
        raw2 = raw.copy()
        raw2[K * d + K:K * d + 2 * K] += 3.0
        assert np.allclose(f.theta(raw2)[2], lam)
        assert c == pytest.approx(1 / (1 + np.exp(-raw[-1])))


# ---------------------------------------------------------------------------
# dense-grid encoding (the paper's DenseGrid, Sec. 5.2)
# ---------------------------------------------------------------------------
def test_dense_grid_layout_and_affine_reproduction():
    # every level dense, level l at entry offset sum_{j<l} (N_j + 1)^d; affine
    # lattice data a.i + b is reproduced exactly at every level, the finest
    # ones included (which the hash grid would hash)
    for dim, max_res in ((2, 256), (3, 48)):
        fp = _field(dim, L=6, base_res=8, max_res=max_res, grid_type=1)
        f0 = oracle.Field(fp)
        res = [f0.level_res(l) for l in range(fp.L)]
        assert res == wi.level_resolutions(fp.L, 8, max_res)
        sizes = [(n + 1) ** dim for n in res]
        assert fp.grid.shape == (sum(sizes), fp.F)
        rng = np.random.default_rng(10 + dim)
        a = rng.normal(size=dim)
        b = -0.7
        grid = np.zeros_like(fp.grid)
        off = 0
        for l, n in enumerate(res):
            side = n + 1
            idx = np.arange(side ** dim)
            coords = [(idx // side ** k) % side for k in range(dim)]
            val = sum(a[k] * coords[k] for k in range(dim)) + b + l     # level-distinct offset
            grid[off:off + side ** dim, 0] = val
            grid[off:off + side ** dim, 1] = 3 * val
            off += side ** dim
        fp.grid = grid
        f = oracle.Field(fp)
        x = rng.uniform(-1.45, 1.45, (60, dim))
        feat = f.encode(x).reshape(60, fp.L, fp.F)
        u = (x - fp.lo) / (fp.hi - fp.lo)
        for l, n in enumerate(res):
            ref = (u * n) @ a + b + l
            assert np.allclose(feat[:, l, 0], ref, atol=1e-10)
            assert np.allclose(feat[:, l, 1], 3 * ref, atol=1e-10)


def test_dense_grid_equals_hash_grid_on_its_dense_levels():
    # the hash grid stores its coarse levels densely at the same lattice
    # index: copying those levels into a dense grid gives the same features
    dim = 2
    fh = _field(dim, seed=4, L=5, log2T=12, base_res=8, max_res=128)
    fd = _field(dim, seed=4, L=5, log2T=12, base_res=8, max_res=128, grid_type=1)
    res = wi.level_resolutions(5, 8, 128)
    off = 0
    dense_levels = []
    for l, n in enumerate(res):
        m = (n + 1) ** dim
        if m <= 1 << 12:
            fd.grid[off:off + m] = fh.grid[l, :m]
            dense_levels.append(l)
        off += m
    assert len(dense_levels) >= 2
    x = np.random.default_rng(3).uniform(-1.4, 1.4, (40, dim))
    eh = oracle.Field(fh).encode(x).reshape(40, 5, 2)
    ed = oracle.Field(fd).encode(x).reshape(40, 5, 2)
    for l in dense_levels:
        assert np.array_equal(eh[:, l], ed[:, l])
    assert not np.allclose(eh[:, -1], ed[:, -1])
