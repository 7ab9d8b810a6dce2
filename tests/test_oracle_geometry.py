"""Pins of the oracle's brute-force geometric queries against independent
characterisations: densely sampled boundaries, side-of-line/plane silhouette
tests, winding-number marching along rays, and crossing-number insideness."""
import numpy as np
import pytest

import oracle
import wost_inputs as wi


def _sample_segments(a, b, m):
    t = np.linspace(0, 1, m)[None, :, None]
    return (a[:, None, :] * (1 - t) + b[:, None, :] * t)


def test_closest_point_2d_vs_dense_sampling():
    sc = wi.star_polyline(256, seed=5)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(0)
    pts = rng.uniform(-1.3, 1.3, (300, 2))
    idx, dist, xb = S.closest_dirichlet(pts)
    D = np.where(sc.bc == 0)[0]
    a, b = sc.verts[sc.prims[D, 0]], sc.verts[sc.prims[D, 1]]
    samp = _sample_segments(a, b, 400).reshape(-1, 2)
    seglen = np.linalg.norm(b - a, axis=1).max()
    dd = np.linalg.norm(pts[:, None, :] - samp[None], axis=2).min(1)
    # the sampled minimum can only be larger, by at most half a sample spacing
    assert np.all(dist <= dd + 1e-12)
    assert np.all(dd - dist <= seglen / 399 / 2 + 1e-12)
    # returned point is at the returned distance and lies on the returned primitive
    assert np.allclose(np.linalg.norm(pts - xb, axis=1), dist, atol=1e-12)
    assert np.all(sc.bc[idx] == 0)
    pa, pb = sc.verts[sc.prims[idx, 0]], sc.verts[sc.prims[idx, 1]]
    cr = np.abs((pb - pa)[:, 0] * (xb - pa)[:, 1] - (pb - pa)[:, 1] * (xb - pa)[:, 0])
    assert np.all(cr <= 1e-12)


def test_closest_point_3d_vs_dense_sampling():
    sc = wi.displaced_icosphere(subdiv=1, seed=3, with_source=False)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(1)
    pts = rng.uniform(-1.0, 1.0, (60, 3))
    idx, dist, xb = S.closest_dirichlet(pts)
    D = np.where(sc.bc == 0)[0]
    tri = sc.verts[sc.prims[D]]                       # (nD, 3, 3)
    m = 60
    u, v = np.meshgrid(np.linspace(0, 1, m), np.linspace(0, 1, m))
    keep = (u + v) <= 1
    u, v = u[keep], v[keep]
    samp = (tri[:, None, 0] * (1 - u - v)[None, :, None] + tri[:, None, 1] * u[None, :, None]
            + tri[:, None, 2] * v[None, :, None]).reshape(-1, 3)
    dd = np.array([np.linalg.norm(samp - p, axis=1).min() for p in pts])
    h = np.linalg.norm(tri[:, 1] - tri[:, 0], axis=1).max() / (m - 1)
    assert np.all(dist <= dd + 1e-12)
    assert np.all(dd - dist <= 2 * h)
    assert np.allclose(np.linalg.norm(pts - xb, axis=1), dist, atol=1e-12)


def _side(o, p, q):
    return np.sign((p[0] - o[0]) * (q[1] - o[1]) - (p[1] - o[1]) * (q[0] - o[0]))


def test_silhouette_2d_side_of_line():
    # A Neumann vertex v with neighbours a (previous) and b (next) is a
    # silhouette from x exactly when a and b lie on the same side of the line
    # through x and v (the sight line grazes the boundary at v).
    sc = wi.star_polyline(96, seed=11, neumann_frac=1.0)
    S = oracle.Scene(sc)
    V = sc.verts
    n = len(V)
    rng = np.random.default_rng(2)
    pts = rng.uniform(-0.6, 0.6, (200, 2))
    _, dist = S.closest_silhouette(pts)
    for x, ds in zip(pts, dist):
        best = np.inf
        for i in range(n):
            a, v, b = V[(i - 1) % n], V[i], V[(i + 1) % n]
            sa, sb = _side(x, v, a), _side(x, v, b)
            if sa != 0 and sa == sb:
                best = min(best, np.linalg.norm(x - v))
        assert ds == pytest.approx(best, rel=1e-12, abs=1e-15)


def test_silhouette_3d_side_of_plane():
    # An interior Neumann edge (a, b) with opposite vertices c1, c2 of its two
    # faces is a silhouette from x when c1 and c2 lie on the same side of the
    # plane through x, a, b; its distance is the point-segment distance.
    sc = wi.displaced_icosphere(subdiv=1, seed=4, neumann_frac=1.0, with_source=False)
    S = oracle.Scene(sc)
    V, P = sc.verts, sc.prims
    edges = {}
    for f, tri in enumerate(P):
        for k in range(3):
            a, b = tri[k], tri[(k + 1) % 3]
            edges.setdefault((min(a, b), max(a, b)), []).append((f, tri[(k + 2) % 3]))
    rng = np.random.default_rng(3)
    pts = rng.uniform(-0.5, 0.5, (40, 3))
    _, dist = S.closest_silhouette(pts)

    def seg_dist(x, a, b):
        t = np.clip(np.dot(x - a, b - a) / np.dot(b - a, b - a), 0, 1)
        return np.linalg.norm(x - (a + t * (b - a)))
    for x, ds in zip(pts, dist):
        best = np.inf
        for (a, b), lst in edges.items():
            assert len(lst) == 2
            nrm = np.cross(V[a] - x, V[b] - x)
            s1 = np.sign(np.dot(nrm, V[lst[0][1]] - x))
            s2 = np.sign(np.dot(nrm, V[lst[1][1]] - x))
            if s1 != 0 and s1 == s2:
                best = min(best, seg_dist(x, V[a], V[b]))
        assert ds == pytest.approx(best, rel=1e-12)


def test_silhouette_point_on_neumann_edge():
    # A walker standing on a Neumann segment next to a reflex corner must see
    # that corner as a silhouette (its own segment is edge-on, the next one
    # faces it from behind); at a convex corner it must not.
    # Domain: L-shape; segment (2,0)->(0,0) then (0,0)->(0,2) is reflex at the origin.
    V = np.array([[2, -1], [2, 0], [0, 0], [0, 2], [-1, 2], [-1, -1]], float)
    P = np.array([[i, (i + 1) % 6] for i in range(6)], np.int32)
    bc = np.array([0, 1, 1, 0, 0, 0], np.uint8)
    sc = wi.Scene("L", 2, V, P, bc, wi.Fn(wi.FN_X2_MINUS_Y2))
    S = oracle.Scene(sc)
    _, d = S.closest_silhouette(np.array([[1.0, 0.0]]))
    assert d[0] == pytest.approx(1.0)      # the reflex vertex at the origin
    # convex case: square with one Neumann corner
    V = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    P = np.array([[i, (i + 1) % 4] for i in range(4)], np.int32)
    bc = np.array([1, 1, 0, 0], np.uint8)
    S = oracle.Scene(wi.Scene("sq", 2, V, P, bc, wi.Fn(wi.FN_X2_MINUS_Y2)))
    _, d = S.closest_silhouette(np.array([[0.5, 0.0]]))
    # vertex (1,0) is convex -> not a silhouette; only the Neumann-set borders
    # (0,0) and (1,1) remain
    assert d[0] == pytest.approx(0.5)


def test_ray_first_hit_2d_vs_marching():
    sc = wi.star_polyline(128, seed=6, neumann_frac=1.0)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(4)
    org = rng.uniform(-0.5, 0.5, (100, 2))
    th = rng.uniform(0, 2 * np.pi, 100)
    dirs = np.stack([np.cos(th), np.sin(th)], 1)
    idx, t = S.ray_neumann(org, dirs, 10.0)
    assert np.all(idx >= 0)
    ts = np.linspace(0, 3, 30001)
    for o, d, ti in zip(org, dirs, t):
        inside = wi.inside_polygon_mask(sc, o[None] + ts[:, None] * d[None])
        first_out = ts[np.argmin(inside)]
        assert abs(first_out - ti) <= 2e-4


def test_ray_first_hit_3d_vs_winding_march():
    sc = wi.displaced_icosphere(subdiv=1, seed=8, neumann_frac=1.0, with_source=False)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(5)
    org = rng.uniform(-0.4, 0.4, (12, 3))
    dirs = rng.normal(size=(12, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    idx, t = S.ray_neumann(org, dirs, 10.0)
    for o, d, ti in zip(org, dirs, t):
        ts = np.linspace(0, 2, 2001)
        w = S.winding(o[None] + ts[:, None] * d[None])
        first_out = ts[np.argmax(w < 0.5)]
        assert abs(first_out - ti) <= 1.5e-3
    # tmax and skip semantics
    i2, t2 = S.ray_neumann(org, dirs, t * 0.5)
    assert np.all(i2 == -1)
    i3, t3 = S.ray_neumann(org + t[:, None] * dirs, dirs, 10.0, skip=idx)
    assert np.all(i3 == -1)                  # leaving a convex-ish shell: nothing further


def test_exit_ray_2d_vs_marching():
    # from inside a closed boundary the first crossing is an exit, so the
    # exit-only cast equals the two-sided one; from outside it skips the
    # entry and returns where the ray leaves the domain again
    sc = wi.star_polyline(128, seed=6, neumann_frac=1.0)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(14)
    org = rng.uniform(-0.5, 0.5, (60, 2))
    th = rng.uniform(0, 2 * np.pi, 60)
    dirs = np.stack([np.cos(th), np.sin(th)], 1)
    i2, t2 = S.ray_neumann(org, dirs, 10.0)
    ie, te = S.ray_neumann(org, dirs, 10.0, exit_only=True)
    assert np.array_equal(i2, ie) and np.allclose(t2, te, rtol=1e-12, atol=1e-14)
    far = 2.0 * np.stack([np.cos(th + np.pi), np.sin(th + np.pi)], 1)   # outside, aimed back across
    i_in, t_in = S.ray_neumann(far, dirs, 10.0)
    i_out, t_out = S.ray_neumann(far, dirs, 10.0, exit_only=True)
    ts = np.linspace(0, 4.5, 45001)
    for o, d, a, b, ia, ib in zip(far, dirs, t_in, t_out, i_in, i_out):
        inside = wi.inside_polygon_mask(sc, o[None] + ts[:, None] * d[None])
        enter = ts[np.argmax(inside)]
        leave = ts[np.argmax(ts > enter) + np.argmin(inside[ts > enter])]
        assert ia >= 0 and ib >= 0 and ia != ib
        assert abs(a - enter) <= 2e-4 and abs(b - leave) <= 2e-4
        n = S.inward_normal(ib)
        assert np.dot(d, n) < 0 < np.dot(d, S.inward_normal(ia))


def test_exit_ray_at_a_vertex():
    # a walk standing on the bottom edge of the unit square at its corner
    # (1, 0), heading barely up (inward for the bottom edge, outward for the
    # right edge), leaves through the right edge at t = 0: the exit cast
    # returns it, with t within the rounding band, not a point far outside
    V = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], float)
    P = np.array([[i, (i + 1) % 4] for i in range(4)], np.int32)
    sc = wi.Scene("square", 2, V, P, np.array([1, 1, 1, 0], np.uint8), wi.Fn(wi.FN_ZERO))
    S = oracle.Scene(sc)
    d = np.array([[1.0, 1e-4]]) / np.hypot(1.0, 1e-4)
    for x0 in ([1.0, 0.0], [1.0 - 1e-12, 0.0], [1.0 + 1e-12, 0.0]):
        i, t = S.ray_neumann(np.array([x0]), d, 10.0, skip=0, exit_only=True)
        assert i[0] == 1 and abs(t[0]) <= 16 * 2 ** -24 * S.scale, (x0, i, t)
    # an inward direction for both edges stays in and exits the top edge
    i, t = S.ray_neumann(np.array([[1.0, 0.0]]), np.array([[-0.6, 0.8]]), 10.0, skip=0, exit_only=True)
    assert i[0] == 2 and abs(t[0] - 1.25) < 1e-12


def test_exit_ray_3d_vs_winding_march():
    sc = wi.displaced_icosphere(subdiv=1, seed=8, neumann_frac=1.0, with_source=False)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(15)
    dirs = rng.normal(size=(10, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    far = -2.0 * dirs
    ie, te = S.ray_neumann(far, dirs, 10.0, exit_only=True)
    for o, d, ti, ii in zip(far, dirs, te, ie):
        ts = np.linspace(0, 4, 4001)
        w = S.winding(o[None] + ts[:, None] * d[None]) > 0.5
        enter = np.argmax(w)
        leave = ts[enter + np.argmin(w[enter:])]
        assert ii >= 0 and abs(ti - leave) <= 3e-3
        assert np.dot(d, S.inward_normal(ii)) < 0


def test_winding_vs_crossing_number():
    sc = wi.star_polyline(200, seed=9)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(6)
    pts = rng.uniform(-1.4, 1.4, (400, 2))
    w = S.winding(pts)
    ins = wi.inside_polygon_mask(sc, pts)
    assert np.all((w > 0.5) == ins)
    assert np.allclose(w, np.round(w), atol=1e-9)


def test_winding_3d_sphere():
    sc = wi.sphere_dirichlet(3)
    S = oracle.Scene(sc)
    rng = np.random.default_rng(7)
    pts = rng.uniform(-1.2, 1.2, (200, 3))
    r = np.linalg.norm(pts, axis=1)
    pts = pts[(r < 0.9) | (r > 1.01)]
    w = S.winding(pts)
    assert np.all((w > 0.5) == (np.linalg.norm(pts, axis=1) < 0.95))
    assert np.allclose(w, np.round(w), atol=1e-8)


def test_mesh_generators_are_closed_and_outward():
    for sc in [wi.sphere_dirichlet(2), wi.slab_box(3), wi.displaced_icosphere(2, 3)]:
        v, f = sc.verts, sc.prims
        vol = np.einsum("ij,ij->i", v[f[:, 0]], np.cross(v[f[:, 1]], v[f[:, 2]])).sum() / 6
        assert vol > 0
        edges = {}
        for tri in f:
            for k in range(3):
                e = (tri[k], tri[(k + 1) % 3])
                edges[e] = edges.get(e, 0) + 1
        for (a, b), c in edges.items():
            assert c == 1 and edges.get((b, a)) == 1
