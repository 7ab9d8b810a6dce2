"""The seeded multi-scene workload generator (no GPU): deterministic,
within its stated ranges, points strictly inside their star polygons."""
import numpy as np

import wost_inputs as wi


def test_config_batch_is_seeded_and_in_range():
    a = wi.config_batch(njobs=12, seed=4, points_range=(100, 2000))
    b = wi.config_batch(njobs=12, seed=4, points_range=(100, 2000))
    c = wi.config_batch(njobs=12, seed=5, points_range=(100, 2000))
    assert len(a) == 12
    for x, y in zip(a, b):
        assert np.array_equal(x.points, y.points) and np.array_equal(x.scene.verts, y.scene.verts)
        assert x.nwalks == y.nwalks and x.seed == y.seed
    assert any(len(x.points) != len(z.points) for x, z in zip(a, c))
    ids = [j.scene.scene_id for j in a]
    assert len(set(ids)) == len(ids)
    for j in a:
        assert 256 <= len(j.scene.prims) <= 16384
        assert 100 <= len(j.points) <= 2000
        assert 8 <= j.nwalks <= 128
        nf = (j.scene.bc == wi.BC_NEUMANN).mean()
        assert 0.19 <= nf <= 0.51
        assert np.all(wi.inside_star_polygon(j.scene, j.points))


def test_star_interior_points_are_uniform_inside():
    sc = wi.star_polyline(512, seed=3)
    p = wi.star_interior_points(sc, 20000, seed=1)
    assert p.shape == (20000, 2) and np.all(wi.inside_star_polygon(sc, p))
    # uniform density: the share of points in the left half matches that
    # half's share of a fine inside-mask of the bounding box
    lo, hi = sc.bbox
    g = wi.grid_points_2d(400, lo, hi)
    inside = wi.inside_star_polygon(sc, g)
    share = (g[inside, 0] < 0).mean()
    assert abs((p[:, 0] < 0).mean() - share) < 0.015
    assert wi.star_interior_points(sc, 0, seed=1).shape == (0, 2)
