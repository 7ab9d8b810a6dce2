"""The FP64 tie-rule helpers of the query parity tests (geom_ties), checked
on the CPU against the oracle: the oracle's own answers (exact FP64) must be
accepted, and planted wrong answers -- another silhouette or primitive that
is not tied, a miss where a strict hit exists -- must be rejected."""
import numpy as np

import geom_ties as gt
import oracle
import wost_inputs as wi


def test_silhouette_rule_accepts_oracle_and_rejects_wrong_elements():
    for dim in (2, 3):
        if dim == 2:
            sc = wi.star_polyline(256, seed=7, neumann_frac=0.6)
            pts = np.random.default_rng(2).uniform(-1.2, 1.2, (300, 2))
        else:
            sc = wi.displaced_icosphere(subdiv=1, seed=4, neumann_frac=0.5, with_source=False)
            pts = np.random.default_rng(3).uniform(-0.8, 0.8, (150, 3))
        O = oracle.Scene(sc)
        el = gt.silhouette_elements(sc)
        assert len(el[0]) == O.nsil
        keys = el[4]
        key_index = {int(k): i for i, k in enumerate(keys)}
        nin = gt.inward_normals(sc)
        oe, od = O.closest_silhouette(pts)
        rejected = 0
        for i in range(len(pts)):
            cand = gt.silhouette_candidates(sc, el, nin, pts[i], O.scale)
            d, strict, maybe = cand
            assert np.all(strict <= maybe)
            if oe[i] < 0:
                assert gt.silhouette_answer_ok(-1, np.inf, key_index, cand, O.scale)
                continue
            assert abs(d[oe[i]] - od[i]) < 1e-12
            assert gt.silhouette_answer_ok(keys[oe[i]], od[i], key_index, cand, O.scale)
            # a strict silhouette clearly farther than the nearest is wrong
            far = np.nonzero(strict & (d > od[i] + 1e-3))[0]
            if len(far):
                assert not gt.silhouette_answer_ok(keys[far[0]], d[far[0]], key_index, cand, O.scale)
                rejected += 1
            # the right element with a wrong distance is wrong
            assert not gt.silhouette_answer_ok(keys[oe[i]], od[i] + 1e-3, key_index, cand, O.scale)
            # an element that is no silhouette from here at all is wrong
            non = np.nonzero(~maybe)[0]
            if len(non):
                assert not gt.silhouette_answer_ok(keys[non[0]], d[non[0]], key_index, cand, O.scale)
        assert rejected > 10


def test_ray_rule_accepts_oracle_and_rejects_wrong_hits():
    for dim in (2, 3):
        if dim == 2:
            sc = wi.star_polyline(256, seed=8, neumann_frac=0.7)
            rng = np.random.default_rng(4)
            org = rng.uniform(-0.6, 0.6, (300, 2))
            th = rng.uniform(0, 2 * np.pi, len(org))
            dirs = np.stack([np.cos(th), np.sin(th)], 1)
        else:
            sc = wi.displaced_icosphere(subdiv=1, seed=9, neumann_frac=0.6, with_source=False)
            rng = np.random.default_rng(5)
            org = rng.uniform(-0.5, 0.5, (200, 3))
            dirs = rng.normal(size=(200, 3))
            dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
        tmax = rng.uniform(0.2, 2.0, len(org))
        O = oracle.Scene(sc)
        for exit_only in (False, True):
            oi, ot = O.ray_neumann(org, dirs, tmax, exit_only=exit_only)
            hits = 0
            for i in range(len(org)):
                cand = gt.ray_candidates(sc, org[i], dirs[i], tmax[i], None, exit_only, O.scale)
                ids, t, strict, maybe, d_t = cand
                assert np.all(strict <= maybe)
                assert gt.ray_answer_ok(oi[i], ot[i] if oi[i] >= 0 else np.inf, cand, O.scale, tmax[i])
                if oi[i] >= 0:
                    hits += 1
                    assert abs(t[ids == oi[i]][0] - ot[i]) < 1e-9
                    # a miss where the oracle hits strictly is wrong
                    if strict[ids == oi[i]][0]:
                        assert not gt.ray_answer_ok(-1, np.inf, cand, O.scale, tmax[i])
                    # a primitive the ray does not cross is wrong
                    other = ids[~maybe]
                    if len(other):
                        assert not gt.ray_answer_ok(other[0], 0.5, cand, O.scale, tmax[i])
                    # a crossing farther along the ray is wrong
                    later = np.nonzero(strict & (t > ot[i] + 1e-3))[0]
                    if len(later):
                        assert not gt.ray_answer_ok(ids[later[0]], t[later[0]], cand, O.scale, tmax[i])
            assert hits > 50
