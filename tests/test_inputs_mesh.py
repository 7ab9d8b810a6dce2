"""The closed-mesh generator behind the large 3D workload (naive surface nets
of a signed function): watertight, outward-wound, with the topology of the
solid it samples (Euler characteristic 2 - 2 genus on manifold meshes)."""
import numpy as np

import wost_inputs as wi


def _edges(P):
    e = np.concatenate([P[:, [0, 1]], P[:, [1, 2]], P[:, [2, 0]]], 0).astype(np.int64)
    return e


def _check_closed(V, P):
    e = _edges(P)
    key = e[:, 0] * len(V) + e[:, 1]
    rev = e[:, 1] * len(V) + e[:, 0]
    # every directed edge appears once and its reverse once: closed, consistently wound
    assert len(np.unique(key)) == len(key)
    assert np.array_equal(np.sort(key), np.sort(rev))
    a, b, c = V[P[:, 0]], V[P[:, 1]], V[P[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6
    return len(V) - len(e) // 2 + len(P), vol


def test_surface_nets_sphere_and_torus():
    V, P = wi.surface_nets(lambda p: np.linalg.norm(p, axis=1) - 0.8, 40, -1.0, 1.0)
    chi, vol = _check_closed(V, P)
    assert chi == 2 and abs(vol - 4 / 3 * np.pi * 0.8 ** 3) < 0.01 * vol
    # torus about z with radii 0.6 and 0.25: genus 1
    def torus(p):
        q = np.linalg.norm(p[:, :2], axis=1) - 0.6
        return np.hypot(q, p[:, 2]) - 0.25
    V, P = wi.surface_nets(torus, 48, -1.0, 1.0)
    chi, vol = _check_closed(V, P)
    assert chi == 0 and abs(vol - 2 * np.pi ** 2 * 0.6 * 0.25 ** 2) < 0.02 * vol


def test_genus3_mesh_small():
    sc = wi.genus3_mesh(n=128)
    V, P = sc.verts, sc.prims
    assert sc.dim == 3 and len(P) > 140000
    assert abs((sc.bc == 1).mean() - 0.3) < 0.002
    a, b, c = V[P[:, 0]], V[P[:, 1]], V[P[:, 2]]
    vol = np.einsum("ij,ij->i", a, np.cross(b, c)).sum() / 6
    assert 2.5 < vol < 4.2
    chi, _ = _check_closed(V, P)
    assert chi == -4                                 # genus 3
    # seeded: identical on a second call
    sc2 = wi.genus3_mesh(n=128)
    assert np.array_equal(sc.verts, sc2.verts) and np.array_equal(sc.bc, sc2.bc)
    # vertices lie on the level set to within a grid cell
    s = wi.genus3_sdf(V, 5)
    assert np.abs(s).max() < 2.5 / 128
