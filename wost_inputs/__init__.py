"""Seeded synthetic inputs shared by the CPU oracle and the CUDA path.

This module only builds *inputs*: boundary meshes, boundary-condition tags,
the analytic data functions (as plain descriptors) and query point sets.
It contains none of the walk-on-stars arithmetic, so both implementations can
use it without sharing method code.

Workload shapes follow the paper's experiments (Sec. 6): 2D polylines with a
Dirichlet/Neumann split (Sec. 6.1, diffusion-curve problems), 3D closed meshes
evaluated on a planar slice (Sec. 6.1, "solving on slices"), K = 8 lobes, dense
evaluation grids.  The paper's own datasets are not used; every scene here is
generated from a seed.

Data-function descriptors (``Fn``) are an interface shared with both sides:
``kind`` is one of the ``FN_*`` codes below and ``params`` a list of doubles.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# ---- analytic data functions (codes are part of the C interface) ----------
FN_ZERO = 0        # 0
FN_CONST = 1       # params[0]
FN_EXP_COS = 2     # exp(a x) cos(a y), a = params[0]
FN_X2_MINUS_Y2 = 3  # x^2 - y^2
FN_SQNORM = 4      # |x|^2                    (Laplacian 2d)
FN_INV_DIST = 5    # 1/|x - c|, c = params[0:3] (harmonic in 3D)
FN_LOG_DIST = 6    # log|x - c|, c = params[0:2] (harmonic in 2D)
FN_GAUSS_SUM = 7   # sum_i A_i exp(-|x-p_i|^2/(2 s^2)); params = [n, s, A_1, p_1(3), ...]
FN_COSH_COS = 8    # cosh(a x) cos(a y), a = params[0]
FN_POLY2 = 9       # c + b.x + sum a_ij x_i x_j; params = [c, bx, by, bz, axx, ayy, azz, axy, axz, ayz]
FN_ATAN2 = 10      # params[0] * atan2(y, x) + params[1] (polar angle, harmonic in 2D)

BC_DIRICHLET = 0
BC_NEUMANN = 1


@dataclasses.dataclass
class Fn:
    kind: int = FN_ZERO
    params: List[float] = dataclasses.field(default_factory=list)


@dataclasses.dataclass
class Scene:
    """A closed boundary: ``prims`` index ``verts``; 2D segments run
    counter-clockwise (domain on the left), 3D triangles wind
    counter-clockwise seen from outside (outward normals)."""
    name: str
    dim: int
    verts: np.ndarray          # (nv, dim) float64
    prims: np.ndarray          # (np, dim) int32
    bc: np.ndarray             # (np,) uint8, BC_DIRICHLET / BC_NEUMANN
    g: Fn                      # Dirichlet data
    f: Fn = dataclasses.field(default_factory=Fn)   # source term (Laplacian u = f)
    h: Fn = dataclasses.field(default_factory=Fn)   # Neumann flux du/dn, n pointing into the domain
    exact: Optional[Fn] = None  # closed-form solution when one exists
    scene_id: int = 0

    def __post_init__(self):
        self.verts = np.ascontiguousarray(self.verts, dtype=np.float64)
        self.prims = np.ascontiguousarray(self.prims, dtype=np.int32)
        self.bc = np.ascontiguousarray(self.bc, dtype=np.uint8)

    @property
    def bbox(self):
        return self.verts.min(0), self.verts.max(0)

    def padded_bbox(self, pad=0.05):
        lo, hi = self.bbox
        ext = hi - lo
        return lo - pad * ext, hi + pad * ext


def eval_fn(fn: Fn, x: np.ndarray) -> np.ndarray:
    """Evaluate a data descriptor on points (n, d) -- used by tests and the
    bench to form closed-form references; not part of either solver."""
    x = np.asarray(x, dtype=np.float64)
    k, p = fn.kind, fn.params
    if k == FN_ZERO:
        return np.zeros(len(x))
    if k == FN_CONST:
        return np.full(len(x), p[0])
    if k == FN_EXP_COS:
        return np.exp(p[0] * x[:, 0]) * np.cos(p[0] * x[:, 1])
    if k == FN_X2_MINUS_Y2:
        return x[:, 0] ** 2 - x[:, 1] ** 2
    if k == FN_SQNORM:
        return (x ** 2).sum(1)
    if k == FN_INV_DIST:
        c = np.array(p[: x.shape[1]])
        return 1.0 / np.linalg.norm(x - c, axis=1)
    if k == FN_LOG_DIST:
        c = np.array(p[: x.shape[1]])
        return np.log(np.linalg.norm(x - c, axis=1))
    if k == FN_COSH_COS:
        return np.cosh(p[0] * x[:, 0]) * np.cos(p[0] * x[:, 1])
    if k == FN_POLY2:
        X, Y = x[:, 0], x[:, 1]
        Z = x[:, 2] if x.shape[1] == 3 else np.zeros(len(x))
        q = list(p) + [0.0] * (10 - len(p))
        return (q[0] + q[1] * X + q[2] * Y + q[3] * Z + q[4] * X * X + q[5] * Y * Y + q[6] * Z * Z
                + q[7] * X * Y + q[8] * X * Z + q[9] * Y * Z)
    if k == FN_ATAN2:
        return p[0] * np.arctan2(x[:, 1], x[:, 0]) + (p[1] if len(p) > 1 else 0.0)
    if k == FN_GAUSS_SUM:
        n, s = int(p[0]), p[1]
        out = np.zeros(len(x))
        for i in range(n):
            a = p[2 + 4 * i]
            c = np.array(p[3 + 4 * i: 3 + 4 * i + x.shape[1]])
            out += a * np.exp(-((x - c) ** 2).sum(1) / (2 * s * s))
        return out
    raise ValueError(f"unknown fn kind {k}")


# ---- 2D scenes --------------------------------------------------------------

def _closed_loop(n):
    i = np.arange(n, dtype=np.int32)
    return np.stack([i, (i + 1) % n], 1)


def ngon(n: int = 64, radius: float = 1.0, g: Optional[Fn] = None, exact=True) -> Scene:
    """Regular n-gon inscribed in a circle, all Dirichlet (64 segments,
    g = e^x cos y is the small 2D Laplace workload)."""
    th = 2 * np.pi * np.arange(n) / n
    v = radius * np.stack([np.cos(th), np.sin(th)], 1)
    g = g or Fn(FN_EXP_COS, [1.0])
    return Scene(f"ngon{n}", 2, v, _closed_loop(n), np.zeros(n, np.uint8), g,
                 exact=g if exact else None)


def star_polyline(nseg: int = 4096, seed: int = 2, amp: float = 0.3, nmodes: int = 5,
                  neumann_frac: float = 0.4, g: Optional[Fn] = None) -> Scene:
    """Star-shaped polyline r(t) = 1 + amp * sum_j a_j cos(m_j t + phi_j) with
    distinct m_j in 1..8, a_j ~ U(0,1) normalised to sum 1, phi_j ~ U(0, 2 pi);
    a contiguous run of ``neumann_frac`` of the segments (seeded offset) is
    zero-flux Neumann, the rest Dirichlet with g = x^2 - y^2."""
    rng = np.random.default_rng(seed)
    m = rng.choice(np.arange(1, 9), size=nmodes, replace=False)
    a = rng.uniform(0, 1, nmodes)
    a /= a.sum()
    phi = rng.uniform(0, 2 * np.pi, nmodes)
    th = 2 * np.pi * np.arange(nseg) / nseg
    r = 1 + amp * (a[None, :] * np.cos(m[None, :] * th[:, None] + phi[None, :])).sum(1)
    v = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    bc = np.zeros(nseg, np.uint8)
    nn = int(round(neumann_frac * nseg))
    off = int(rng.integers(0, nseg))
    bc[(off + np.arange(nn)) % nseg] = BC_NEUMANN
    return Scene(f"star{nseg}_s{seed}", 2, v, _closed_loop(nseg), bc,
                 g or Fn(FN_X2_MINUS_Y2))


def half_disk(narc: int = 64, nflat: int = 16, g: Optional[Fn] = None) -> Scene:
    """Upper half of the unit disk: the flat edge on y = 0 is zero-flux
    Neumann, the arc Dirichlet.  Any g with dg/dy = 0 on y = 0 (x^2 - y^2,
    e^x cos y, |x|^2 for the Poisson case) is then the exact solution."""
    th = np.pi * np.arange(narc + 1) / narc
    arc = np.stack([np.cos(th), np.sin(th)], 1)          # (1,0) -> (-1,0) CCW
    xs = -1 + 2 * np.arange(1, nflat) / nflat             # interior flat vertices
    flat = np.stack([xs, np.zeros_like(xs)], 1)           # (-1,0) -> (1,0)
    v = np.concatenate([arc, flat], 0)
    n = len(v)
    prims = _closed_loop(n)
    bc = np.zeros(n, np.uint8)
    bc[narc:] = BC_NEUMANN                                # segments from (-1,0) back to (1,0)
    g = g or Fn(FN_X2_MINUS_Y2)
    return Scene("half_disk", 2, v, prims, bc, g, exact=g)


def half_disk_flux(narc: int = 64, nflat: int = 16, poisson: bool = False) -> Scene:
    """Upper half disk with a nonzero Neumann flux on the flat edge y = 0
    (normal (0, 1) into the domain).  Laplace: u = x^2 - y^2 + x y + y, so
    h = du/dy(y = 0) = 1 + x.  Poisson (f = 4): u = x^2 + y^2 + y, h = 1."""
    sc = half_disk(narc, nflat)
    if poisson:
        u = Fn(FN_POLY2, [0, 0, 1, 0, 1, 1, 0, 0, 0, 0])
        sc.f = Fn(FN_CONST, [4.0])
        sc.h = Fn(FN_CONST, [1.0])
    else:
        u = Fn(FN_POLY2, [0, 0, 1, 0, 1, -1, 0, 1, 0, 0])
        sc.h = Fn(FN_POLY2, [1, 1, 0, 0, 0, 0, 0, 0, 0, 0])
    sc.g = sc.exact = u
    sc.name = "half_disk_flux"
    return sc


def rectangle_channel(nx: int = 16, ny: int = 8, a: float = math.pi) -> Scene:
    """[-1,1] x [0,1]: the edges y = 0 and y = 1 are zero-flux Neumann, x = +-1
    Dirichlet with g = cosh(a x) cos(a y), exact for a = pi (dg/dy = 0 on both
    Neumann edges).  Walks bounce between two Neumann walls."""
    pts = []
    for i in range(nx):                       # bottom, left to right
        pts.append((-1 + 2 * i / nx, 0.0))
    for j in range(ny):                       # right, bottom to top
        pts.append((1.0, j / ny))
    for i in range(nx):                       # top, right to left
        pts.append((1 - 2 * i / nx, 1.0))
    for j in range(ny):                       # left, top to bottom
        pts.append((-1.0, 1 - j / ny))
    v = np.array(pts)
    n = len(v)
    bc = np.zeros(n, np.uint8)
    bc[:nx] = BC_NEUMANN
    bc[nx + ny: 2 * nx + ny] = BC_NEUMANN
    g = Fn(FN_COSH_COS, [a])
    return Scene("channel2d", 2, v, _closed_loop(n), bc, g, exact=g)


def annulus_sector(r_in: float = 0.9, r_out: float = 1.0, theta_max: float = 0.95 * math.pi,
                   narc: int = 1024) -> Scene:
    """The thin annulus sector r_in < |x| < r_out, 0 < angle < theta_max:
    zero-flux Neumann arcs, Dirichlet radial ends with g = angle / theta_max,
    the polar angle being harmonic with zero normal derivative on circles
    (exact for the curved domain; the polygon's chords put a small error on
    it).  The inner circle's silhouette keeps the star radius near the
    annulus width, so walks from the middle take hundreds of steps."""
    th = theta_max * np.arange(narc + 1) / narc
    outer = np.stack([r_out * np.cos(th), r_out * np.sin(th)], 1)          # CCW, domain on the left
    inner = np.stack([r_in * np.cos(th[::-1]), r_in * np.sin(th[::-1])], 1)  # CW back to angle 0
    v = np.concatenate([outer, inner], 0)
    n = len(v)
    prims = _closed_loop(n)
    bc = np.ones(n, np.uint8)
    bc[narc] = BC_DIRICHLET          # outer end -> inner end at theta_max
    bc[n - 1] = BC_DIRICHLET         # inner start -> outer start at angle 0
    g = Fn(FN_ATAN2, [1.0 / theta_max, 0.0])
    return Scene("annulus_sector", 2, v, prims, bc, g, exact=g)


# ---- 3D scenes --------------------------------------------------------------

def icosphere(subdiv: int):
    """Unit icosphere: 20 * 4^subdiv outward-wound triangles."""
    t = (1 + 5 ** 0.5) / 2
    v = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t),
         (0, -1, -t), (0, 1, -t), (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    f = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4),
         (11, 10, 2), (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8),
         (3, 8, 9), (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    verts = [np.array(p, float) / np.linalg.norm(p) for p in v]
    faces = f
    for _ in range(subdiv):
        cache = {}
        new_faces = []

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                p = verts[a] + verts[b]
                verts.append(p / np.linalg.norm(p))
                cache[key] = len(verts) - 1
            return cache[key]
        for (a, b, c) in faces:
            ab, bc_, ca = mid(a, b), mid(b, c), mid(c, a)
            new_faces += [(a, ab, ca), (b, bc_, ab), (c, ca, bc_), (ab, bc_, ca)]
        faces = new_faces
    return np.array(verts), np.array(faces, np.int32)


class Perlin3:
    """Improved gradient noise (Perlin 2002 construction) with a seeded
    permutation table; used only to displace generated meshes."""

    _G = np.array([(1, 1, 0), (-1, 1, 0), (1, -1, 0), (-1, -1, 0), (1, 0, 1), (-1, 0, 1),
                   (1, 0, -1), (-1, 0, -1), (0, 1, 1), (0, -1, 1), (0, 1, -1), (0, -1, -1)], float)

    def __init__(self, seed: int):
        rng = np.random.default_rng(seed)
        p = rng.permutation(256)
        self.p = np.concatenate([p, p]).astype(np.int64)
        self.gi = rng.integers(0, 12, 256)

    @staticmethod
    def _fade(t):
        return t * t * t * (t * (t * 6 - 15) + 10)

    def __call__(self, x: np.ndarray) -> np.ndarray:
        x = np.asarray(x, float)
        i0 = np.floor(x).astype(np.int64)
        fr = x - i0
        i0 &= 255
        u = self._fade(fr)
        out = 0.0
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    h = self.p[self.p[self.p[i0[:, 0] + dx] + i0[:, 1] + dy] + i0[:, 2] + dz]
                    g = self._G[self.gi[h & 255]]
                    d = fr - np.array([dx, dy, dz], float)
                    w = ((u[:, 0] if dx else 1 - u[:, 0]) * (u[:, 1] if dy else 1 - u[:, 1])
                         * (u[:, 2] if dz else 1 - u[:, 2]))
                    out = out + w * (g * d).sum(1)
        return out


def _cap_neumann(verts, prims, frac, axis):
    cen = verts[prims].mean(1)
    dirs = cen / np.linalg.norm(cen, axis=1, keepdims=True)
    score = dirs @ axis
    n = int(round(frac * len(prims)))
    bc = np.zeros(len(prims), np.uint8)
    bc[np.argsort(-score, kind="stable")[:n]] = BC_NEUMANN
    return bc


def displaced_icosphere(subdiv: int = 6, seed: int = 3, amp: float = 0.15, freq: float = 2.0,
                        neumann_frac: float = 0.3, with_source: bool = True) -> Scene:
    """Icosphere (20 * 4^subdiv triangles, 81,920 at subdiv 6) radially
    displaced by amp * Perlin noise; the Neumann set is the 30% of faces
    whose centroid direction best aligns with a seeded axis (one cap).
    Dirichlet g = 1/|x - c|, c = (2.5, 0, 0); source = 4 seeded Gaussians
    (sigma 0.1, amplitudes U(-4, 4), centres inside)."""
    rng = np.random.default_rng(seed)
    v, f = icosphere(subdiv)
    noise = Perlin3(seed)
    v = v * (1 + amp * noise(v * freq + 17.0))[:, None]
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    bc = _cap_neumann(v, f, neumann_frac, axis)
    src = Fn()
    if with_source:
        params = [4.0, 0.1]
        for _ in range(4):
            a = rng.uniform(-4, 4)
            d = rng.normal(size=3)
            c = d / np.linalg.norm(d) * rng.uniform(0, 0.5)
            params += [a, *c]
        src = Fn(FN_GAUSS_SUM, params)
    return Scene(f"icosphere{subdiv}_s{seed}", 3, v, f, bc, Fn(FN_INV_DIST, [2.5, 0.0, 0.0]), f=src)


def _tunnel_lines(rng, count=3, radius=0.2, reach=0.45, min_gap=0.5):
    """Seeded lines (point, unit direction) crossing the unit ball, pairwise
    at least min_gap apart, so the tunnels around them are disjoint."""
    lines = []
    while len(lines) < count:
        a = rng.normal(size=3)
        a /= np.linalg.norm(a)
        p = rng.normal(size=3)
        p -= (p @ a) * a
        p *= rng.uniform(0.0, reach) / max(np.linalg.norm(p), 1e-12)
        ok = True
        for q, b in lines:
            n = np.cross(a, b)
            dist = abs((p - q) @ n) / np.linalg.norm(n) if np.linalg.norm(n) > 1e-9 else \
                np.linalg.norm(np.cross(p - q, a))
            ok &= dist > min_gap
        if ok:
            lines.append((p, a))
    return lines


def genus3_sdf(pts: np.ndarray, seed: int = 5, amp: float = 0.15, freq: float = 2.0, radius: float = 0.2,
               blend: float = 0.04):
    """Signed distance-like function (negative inside) of the displaced unit
    sphere minus three disjoint cylinders of the given radius along seeded
    lines: smax(|p| - R(p/|p|), -(dist_i - radius)), where smax is the
    polynomial smooth maximum max(a, b) + k h^2 / 4, h = max(k - |a - b|, 0) / k
    with k = blend, which rounds the tunnel rims so that no crease is sharper
    than the meshing grid.  R is evaluated only in the radial band where the
    displaced surface can lie."""
    rng = np.random.default_rng(seed)
    noise = Perlin3(seed)
    lines = _tunnel_lines(rng, radius=radius)
    pts = np.asarray(pts, np.float64)
    r = np.linalg.norm(pts, axis=1)
    d = r - 1.0
    band = (r > 1 - 1.2 * amp) & (r < 1 + 1.2 * amp)
    if band.any():
        dirs = pts[band] / r[band][:, None]
        d[band] = r[band] - (1 + amp * noise(dirs * freq + 17.0))
    for p0, a in lines:
        q = pts - p0
        q -= (q @ a)[:, None] * a
        e = radius - np.linalg.norm(q, axis=1)
        h = np.maximum(blend - np.abs(d - e), 0.0) / blend
        d = np.maximum(d, e) + 0.25 * blend * h * h
    return d


def surface_nets(sdf, n: int, lo: float, hi: float, chunk: int = 1 << 22):
    """Naive surface nets of the zero level set of sdf (negative inside) on an
    n^3-cell grid over [lo, hi]^3: one vertex per cell with a sign change (the
    mean of its edges' linear crossings), one quad per crossing grid edge over
    the four cells sharing it, wound counter-clockwise seen from outside, split
    into two triangles.  Returns (verts, tris)."""
    h = (hi - lo) / n
    axis = lo + h * np.arange(n + 1)
    X, Y, Z = np.meshgrid(axis, axis, axis, indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    del X, Y, Z
    s = np.empty(len(P))
    for b in range(0, len(P), chunk):
        s[b:b + chunk] = sdf(P[b:b + chunk])
    del P
    s = s.reshape(n + 1, n + 1, n + 1)
    inside = s < 0
    assert not inside[[0, -1]].any() and not inside[:, [0, -1]].any() and not inside[:, :, [0, -1]].any()
    cell_ids, cross_pts, quads, flips = [], [], [], []

    def cid(i, j, k):
        return (i * n + j) * n + k

    for ax in range(3):
        sl0 = [slice(None)] * 3
        sl1 = [slice(None)] * 3
        sl0[ax] = slice(0, n)
        sl1[ax] = slice(1, n + 1)
        ch = inside[tuple(sl0)] != inside[tuple(sl1)]
        idx = np.argwhere(ch)                      # lower endpoint (i, j, k)
        s0 = s[tuple(sl0)][ch]
        s1 = s[tuple(sl1)][ch]
        t = s0 / (s0 - s1)
        p = lo + h * idx.astype(np.float64)
        p[:, ax] += h * t
        i, j, k = idx[:, 0], idx[:, 1], idx[:, 2]
        # the four cells around the edge, counter-clockwise about +axis
        if ax == 0:
            cs = [cid(i, j - 1, k - 1), cid(i, j, k - 1), cid(i, j, k), cid(i, j - 1, k)]
        elif ax == 1:
            cs = [cid(i - 1, j, k - 1), cid(i - 1, j, k), cid(i, j, k), cid(i, j, k - 1)]
        else:
            cs = [cid(i - 1, j - 1, k), cid(i, j - 1, k), cid(i, j, k), cid(i - 1, j, k)]
        cs = np.stack(cs, 1)
        for c in range(4):
            cell_ids.append(cs[:, c])
            cross_pts.append(p)
        quads.append(cs)
        flips.append(s0 >= 0)                       # outside (not s < 0) at the lower end: outward is -axis
    ids = np.concatenate(cell_ids)
    pts = np.concatenate(cross_pts, 0)
    uniq, inv = np.unique(ids, return_inverse=True)
    cnt = np.bincount(inv, minlength=len(uniq))
    verts = np.stack([np.bincount(inv, weights=pts[:, d], minlength=len(uniq)) / cnt for d in range(3)], 1)
    q = np.searchsorted(uniq, np.concatenate(quads, 0))
    flip = np.concatenate(flips)
    q[flip] = q[flip][:, ::-1]
    tris = np.concatenate([q[:, [0, 1, 2]], q[:, [0, 2, 3]]], 0).astype(np.int32)
    return verts, tris


def genus3_mesh(n: int = 330, seed: int = 5, neumann_frac: float = 0.3) -> Scene:
    """The genus-3 solid (displaced sphere minus three disjoint tunnels) as a
    naive-surface-nets mesh on an n^3 grid over [-1.25, 1.25]^3 (about 1 M
    triangles at n = 330); the Neumann set is the neumann_frac of faces whose
    centroid direction best aligns with a seeded axis; Dirichlet g = 1/|x - c|,
    c = (2.5, 0, 0); no source."""
    verts, tris = surface_nets(lambda p: genus3_sdf(p, seed), n, -1.25, 1.25)
    rng = np.random.default_rng(seed + 1000)
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    bc = _cap_neumann(verts, tris, neumann_frac, axis)
    return Scene(f"genus3_n{n}_s{seed}", 3, verts, tris, bc, Fn(FN_INV_DIST, [2.5, 0.0, 0.0]))


def config_genus3(res: int = 1024, n: int = 330, seed: int = 5, margin: float = 0.02):
    """The large 3D workload: the genus-3 mesh and the res x res cell centres
    of the slice z = 0 over its bounding box, kept where the solid's signed
    function is below -margin (inside, off the boundary)."""
    sc = genus3_mesh(n, seed)
    lo, hi = sc.bbox
    pts = slice_points_3d(res, lo, hi, 0.0)
    return sc, pts[genus3_sdf(pts, seed) < -margin]


def slab_box(n: int = 4) -> Scene:
    """Box [-1,1]^2 x [0,1] triangulated with n x n quads per face; the
    faces z = 0 and z = 1 are zero-flux Neumann, the side faces Dirichlet with
    g = x^2 - y^2 (harmonic, z-independent, hence exact)."""
    verts, tris, bcs = [], [], []

    def face(origin, du, dv, neumann):
        base = len(verts)
        for j in range(n + 1):
            for i in range(n + 1):
                verts.append(origin + du * (i / n) + dv * (j / n))
        for j in range(n):
            for i in range(n):
                a = base + j * (n + 1) + i
                b, c, d = a + 1, a + n + 2, a + n + 1
                tris.extend([(a, b, c), (a, c, d)])
                bcs.extend([neumann, neumann])
    O = np.array
    # each face: du x dv points outward
    face(O([-1., -1., 0.]), O([0., 2., 0.]), O([2., 0., 0.]), 1)   # z=0, normal -z
    face(O([-1., -1., 1.]), O([2., 0., 0.]), O([0., 2., 0.]), 1)   # z=1, normal +z
    face(O([-1., -1., 0.]), O([2., 0., 0.]), O([0., 0., 1.]), 0)   # y=-1, normal -y
    face(O([-1., 1., 0.]), O([0., 0., 1.]), O([2., 0., 0.]), 0)    # y=+1, normal +y
    face(O([-1., -1., 0.]), O([0., 0., 1.]), O([0., 2., 0.]), 0)   # x=-1, normal -x
    face(O([1., -1., 0.]), O([0., 2., 0.]), O([0., 0., 1.]), 0)    # x=+1, normal +x
    verts = np.array(verts)
    # weld duplicate vertices so that edges are shared (needed for silhouettes)
    key = np.round(verts * 1e9).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    verts = verts[first]
    tris = inv.reshape(-1)[np.array(tris)]
    g = Fn(FN_X2_MINUS_Y2)
    return Scene("slab_box", 3, verts, tris.astype(np.int32), np.array(bcs, np.uint8), g, exact=g)


def slab_box_flux(n: int = 3) -> Scene:
    """The slab box with a nonzero flux through both Neumann planes:
    u = x^2 - y^2 + z + x z, du/dz = 1 + x; the normal into the domain is +z
    on z = 0 and -z on z = 1, so h = (1 + x)(1 - 2 z)."""
    sc = slab_box(n)
    u = Fn(FN_POLY2, [0, 0, 0, 1, 1, -1, 0, 0, 1, 0])
    sc.g = sc.exact = u
    sc.h = Fn(FN_POLY2, [1, 1, 0, -2, 0, 0, 0, 0, -2, 0])
    sc.name = "slab_box_flux"
    return sc


def sphere_dirichlet(subdiv: int = 3, g: Optional[Fn] = None) -> Scene:
    """Unit icosphere, all Dirichlet (g = 1/|x - c| with c outside is exact)."""
    v, f = icosphere(subdiv)
    g = g or Fn(FN_INV_DIST, [2.5, 0.0, 0.0])
    return Scene(f"sphere{subdiv}", 3, v, f, np.zeros(len(f), np.uint8), g, exact=g)


# ---- query point sets -------------------------------------------------------

def grid_points_2d(n: int, lo, hi) -> np.ndarray:
    """n x n cell centres of the box [lo, hi] (row-major, x fastest)."""
    xs = lo[0] + (np.arange(n) + 0.5) / n * (hi[0] - lo[0])
    ys = lo[1] + (np.arange(n) + 0.5) / n * (hi[1] - lo[1])
    X, Y = np.meshgrid(xs, ys)
    return np.stack([X.ravel(), Y.ravel()], 1)


def slice_points_3d(n: int, lo, hi, z: float = 0.0) -> np.ndarray:
    """n x n cell centres of the plane z = const over [lo, hi] in x, y."""
    p2 = grid_points_2d(n, lo[:2], hi[:2])
    return np.concatenate([p2, np.full((len(p2), 1), z)], 1)


def inside_polygon_mask(scene: Scene, pts: np.ndarray) -> np.ndarray:
    """Crossing-number test of 2D points against the scene polygon (input
    masking only)."""
    a = scene.verts[scene.prims[:, 0]]
    b = scene.verts[scene.prims[:, 1]]
    x, y = pts[:, 0:1], pts[:, 1:2]
    cond = (a[None, :, 1] > y) != (b[None, :, 1] > y)
    with np.errstate(divide="ignore", invalid="ignore"):
        xint = a[None, :, 0] + (y - a[None, :, 1]) * (b[None, :, 0] - a[None, :, 0]) / (b[None, :, 1] - a[None, :, 1])
    cross = cond & (x < xint)
    return (cross.sum(1) % 2) == 1


def inside_polygon_mask_chunked(scene: Scene, pts: np.ndarray, chunk: int = 4096) -> np.ndarray:
    out = np.zeros(len(pts), bool)
    for s in range(0, len(pts), chunk):
        out[s:s + chunk] = inside_polygon_mask(scene, pts[s:s + chunk])
    return out


def config_small_laplace():
    """64-segment polyline approximating the unit circle, all Dirichlet,
    g = e^x cos y; 32 x 32 grid of [-1,1]^2 clipped to the interior."""
    sc = ngon(64)
    pts = grid_points_2d(32, (-1, -1), (1, 1))
    pts = pts[inside_polygon_mask(sc, pts)]
    return sc, pts


def inside_star_polygon(sc: Scene, pts: np.ndarray) -> np.ndarray:
    """Exact insideness for a polygon whose vertices are sorted by angle
    around the origin (star-shaped w.r.t. 0): find the edge spanning each
    point's direction and compare the point with that edge's line."""
    v = sc.verts
    ang = np.arctan2(v[:, 1], v[:, 0]) % (2 * np.pi)
    order = np.argsort(ang)
    va, aa = v[order], ang[order]
    th = np.arctan2(pts[:, 1], pts[:, 0]) % (2 * np.pi)
    j = np.searchsorted(aa, th, side="right")
    a = va[(j - 1) % len(va)]
    b = va[j % len(va)]
    # inside iff p is on the origin's side of the line a-b
    cross_p = (b[:, 0] - a[:, 0]) * (pts[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (pts[:, 0] - a[:, 0])
    cross_o = (b[:, 0] - a[:, 0]) * (0 - a[:, 1]) - (b[:, 1] - a[:, 1]) * (0 - a[:, 0])
    return np.sign(cross_p) == np.sign(cross_o)


def config_star_guided(res: int = 512, nseg: int = 4096, seed: int = 2):
    """4096-segment seeded star polyline, 40% zero-flux Neumann arc, Dirichlet
    x^2 - y^2; res x res grid over the bounding box masked to the interior."""
    sc = star_polyline(nseg, seed)
    lo, hi = sc.bbox
    pts = grid_points_2d(res, lo, hi)
    pts = pts[inside_star_polygon(sc, pts)]
    return sc, pts


def star_interior_points(sc: Scene, n: int, seed: int) -> np.ndarray:
    """n seeded points uniform in the interior of a star polygon (rejection
    from its bounding box)."""
    rng = np.random.default_rng(seed)
    lo, hi = sc.bbox
    out = []
    have = 0
    while have < n:
        cand = lo + (hi - lo) * rng.uniform(0, 1, (max(2 * (n - have), 64), 2))
        cand = cand[inside_star_polygon(sc, cand)]
        out.append(cand)
        have += len(cand)
    return np.concatenate(out, 0)[:n] if n > 0 else np.zeros((0, 2))


@dataclasses.dataclass
class BatchJob:
    scene: Scene
    points: np.ndarray
    nwalks: int
    seed: int = 1


def _log_uniform_int(rng, lo, hi):
    return int(round(math.exp(rng.uniform(math.log(lo), math.log(hi)))))


def config_batch(njobs: int = 64, seed: int = 4, seg_range=(256, 16384), neumann_range=(0.2, 0.5),
                 points_range=(1024, 262144), wpp_range=(8, 128)):
    """Many independent 2D problems of uneven size: njobs seeded star
    polylines (as star_polyline) with log-uniform segment counts in
    seg_range and a Neumann fraction uniform in neumann_range; each job has a
    log-uniform number of interior query points in points_range and a
    log-uniform walk count in wpp_range.  Job j has scene_id j + 1 and walk
    seed 1000 * seed + j."""
    rng = np.random.default_rng(seed)
    jobs = []
    for j in range(njobs):
        nseg = _log_uniform_int(rng, *seg_range)
        nf = float(rng.uniform(*neumann_range))
        npts = _log_uniform_int(rng, *points_range)
        wpp = _log_uniform_int(rng, *wpp_range)
        sc = star_polyline(nseg, seed=100000 * seed + j, neumann_frac=nf)
        sc.scene_id = j + 1
        pts = star_interior_points(sc, npts, seed=200000 * seed + j)
        jobs.append(BatchJob(sc, pts, wpp, seed=1000 * seed + j))
    return jobs


def config_3d_guided(res: int = 256, subdiv: int = 6, seed: int = 3, neumann_frac: float = 0.3,
                     with_source: bool = True, margin: float = 0.01):
    """The displaced icosphere (81,920 triangles at subdiv 6) with its Neumann
    cap, Gaussian sources and g = 1/|x - c|; query points are the res x res
    cell centres of the slice z = 0 over the bounding box, kept where |p| is
    below (1 - margin) of the displaced radius in p's direction (the surface
    is star-shaped about the origin)."""
    sc = displaced_icosphere(subdiv, seed, neumann_frac=neumann_frac, with_source=with_source)
    lo, hi = sc.bbox
    pts = slice_points_3d(res, lo, hi, 0.0)
    noise = Perlin3(seed)
    rad = np.linalg.norm(pts, axis=1)
    d = pts / np.maximum(rad, 1e-12)[:, None]
    r_surf = 1 + 0.15 * noise(d * 2.0 + 17.0)
    return sc, pts[rad < (1 - margin) * r_surf]


def subsample(pts: np.ndarray, n: int, seed: int = 0) -> np.ndarray:
    if n >= len(pts):
        return pts
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(len(pts), n, replace=False))
    return pts[idx]


# ---- neural-field parameters for tests (exchange layout) ---------------------

def level_resolutions(L: int, base_res: int, max_res: int):
    """N_l = floor(N_min b^l), b such that N_{L-1} = N_max (both encodings)."""
    if L == 1:
        return [base_res]
    b = math.exp((math.log(max_res) - math.log(base_res)) / (L - 1))
    return [int(math.floor(base_res * b ** l + 1e-6)) for l in range(L)]


def dense_grid_entries(dim: int, L: int, base_res: int, max_res: int) -> int:
    """Lattice entries of the dense-grid encoding: sum_l (N_l + 1)^d."""
    return sum((n + 1) ** dim for n in level_resolutions(L, base_res, max_res))


def random_field_params(dim: int, seed: int, lo, hi, K: int = 8, L: int = 16, log2T: int = 16,
                        F: int = 2, H: int = 64, base_res: int = 16, max_res: Optional[int] = None,
                        grid_scale: float = 0.5, w_scale: float = 1.0, grid_type: int = 0):
    """Seeded field parameters in the exchange layout used by both
    implementations: grid (L, 2^log2T, F), W1 (H, L*F), W2 (H, H),
    W3 (nout, H), b3 (nout) with nout = (dim + 2) K + 1.  Returned as a dict
    of float64 arrays plus the shape/box metadata."""
    rng = np.random.default_rng(seed)
    if max_res is None:
        max_res = 2048 if dim == 2 else 512
    T = 1 << log2T
    nin = L * F
    nout = (dim + 2) * K + 1
    if grid_type == 1:
        grid = rng.uniform(-grid_scale, grid_scale, (dense_grid_entries(dim, L, base_res, max_res), F))
    else:
        grid = rng.uniform(-grid_scale, grid_scale, (L, T, F))
    W1 = rng.uniform(-1, 1, (H, nin)) * w_scale * math.sqrt(6.0 / nin)
    W2 = rng.uniform(-1, 1, (H, H)) * w_scale * math.sqrt(6.0 / H)
    W3 = rng.uniform(-1, 1, (nout, H)) * w_scale * math.sqrt(6.0 / H) * 0.5
    b3 = rng.normal(size=nout) * 0.5
    return dict(dim=dim, K=K, L=L, log2T=log2T, F=F, H=H, base_res=base_res, max_res=max_res,
                lo=np.asarray(lo, float), hi=np.asarray(hi, float),
                grid=grid, W1=W1, W2=W2, W3=W3, b3=b3, grid_type=grid_type)


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (ties to even) and return
    them as float64 -- lets both implementations start from bit-identical
    low-precision parameters."""
    f = np.asarray(a, np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def round_to_fp16(a: np.ndarray) -> np.ndarray:
    return np.asarray(a, np.float16).astype(np.float64)
