"""FP64 reference geometry for the tie rule of the query parity tests.

The GPU runs its boundary queries in FP32 and re-tests only some decisions in
FP64; the oracle runs everything in FP64.  Both must return the same primitive
except where rounding may legitimately decide: two candidates at equal
distance (a tie), or a candidate whose own decision (silhouette side, ray
parameter range, exit orientation) lies within the rounding band of its
threshold.  The helpers below compute, independently of both
implementations, each candidate's FP64 value and whether its decision is
"strict" (cannot flip under FP32 rounding of the inputs and the arithmetic)
or "borderline"; a test then accepts a GPU answer only if it lies between
the strict and the permissive reading.

Rounding bands: an FP32 quantity computed from FP32 inputs of magnitude M
carries an absolute error of a few units of 2^-24 M; divided by a
determinant it is scaled by the ray/primitive condition number.  The bands
use 32 units (a factor of 4 to 8 over the operation counts) so that only
decisions that rounding can really move are accepted.
"""
import numpy as np

U = 2.0 ** -24


def tie_band(d, scale):
    """Distances closer than this are a tie (the rule for closest-point and
    silhouette indices): 8 units of 2^-24 of (distance + scene scale)."""
    return 8 * U * (np.abs(d) + scale)


# ---------------------------------------------------------------------------
# silhouettes
# ---------------------------------------------------------------------------
def inward_normals(sc):
    V, P = sc.verts, sc.prims
    if sc.dim == 2:
        e = V[P[:, 1]] - V[P[:, 0]]
        n = np.stack([-e[:, 1], e[:, 0]], 1)
    else:
        n = -np.cross(V[P[:, 1]] - V[P[:, 0]], V[P[:, 2]] - V[P[:, 0]])
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def silhouette_elements(sc):
    """Silhouette elements of the Neumann boundary in the oracle's order:
    2D Neumann vertices (ascending), 3D Neumann edges (a < b, ascending).
    Returns (a, b, f0, f1, key): element endpoints (a == b in 2D), the two
    adjacent Neumann primitives (-1 when the element borders the Neumann set:
    always a silhouette) and the GPU's element key."""
    P, bc = sc.prims, sc.bc
    neu = np.nonzero(bc == 1)[0]
    if sc.dim == 2:
        out_seg, in_seg = {}, {}
        for i in neu:
            out_seg[P[i, 0]] = i
            in_seg[P[i, 1]] = i
        verts = sorted(set(out_seg) | set(in_seg))
        a = np.array(verts)
        f0 = np.array([in_seg.get(v, -1) for v in verts])
        f1 = np.array([out_seg.get(v, -1) for v in verts])
        both = (f0 >= 0) & (f1 >= 0)
        f0, f1 = np.where(both, f0, -1), np.where(both, f1, -1)
        return a, a.copy(), f0, f1, a.astype(np.int64)
    faces = {}
    for i in neu:
        for k in range(3):
            u, v = P[i, k], P[i, (k + 1) % 3]
            faces.setdefault((min(u, v), max(u, v)), []).append(i)
    keys = sorted(faces)
    a = np.array([k[0] for k in keys])
    b = np.array([k[1] for k in keys])
    f0 = np.array([faces[k][0] if len(faces[k]) == 2 else -1 for k in keys])
    f1 = np.array([faces[k][1] if len(faces[k]) == 2 else -1 for k in keys])
    return a, b, f0, f1, a.astype(np.int64) * len(sc.verts) + b


def _point_seg_dist(x, A, B):
    e = B - A
    ee = (e * e).sum(1)
    t = np.where(ee > 0, ((x - A) * e).sum(1) / np.where(ee > 0, ee, 1), 0.0)
    t = np.clip(t, 0, 1)
    return np.linalg.norm(x - (A + t[:, None] * e), axis=1)


def silhouette_candidates(sc, el, nin, x, scale):
    """For one query x: FP64 distance to every element, and its strict /
    permissive silhouette status (edge-on tolerance tau = 1e-6 scale; a
    classification value within its rounding band of +-tau is borderline)."""
    a, b, f0, f1, _ = el
    V = sc.verts
    A, B = V[a], V[b]
    d = _point_seg_dist(x, A, B)
    always = f0 < 0
    r = x - A
    rn = np.linalg.norm(r, axis=1)
    tau = 1e-6 * scale
    g0 = np.where(always, 0, f0)
    g1 = np.where(always, 0, f1)
    o0 = (nin[g0] * r).sum(1)
    o1 = (nin[g1] * r).sum(1)
    band = 32 * U * (rn + np.linalg.norm(x) + np.linalg.norm(A, axis=1))

    def cls(o, shift):
        return np.where(o + shift > tau, 1, np.where(o + shift < -tau, -1, 0))

    def sil(c0, c1):
        return ((c0 == -1) & (c1 >= 0)) | ((c1 == -1) & (c0 >= 0))

    exact = sil(cls(o0, 0), cls(o1, 0))
    # every combination of the two values moved by +-band
    outcomes = [sil(cls(o0, s0), cls(o1, s1)) for s0 in (-band, 0, band) for s1 in (-band, 0, band)]
    allsil = np.all(outcomes, axis=0)
    anysil = np.any(outcomes, axis=0)
    strict = always | (exact & allsil)
    maybe = always | anysil
    return d, strict, maybe


def silhouette_answer_ok(gk, gd, key_index, cand, scale):
    """The GPU's (key, FP32 distance) is a valid answer for one query."""
    d, strict, maybe = cand
    inf = np.inf
    lo = d[maybe].min() if maybe.any() else inf       # nearest if every borderline element counts
    hi = d[strict].min() if strict.any() else inf     # nearest over strict silhouettes only
    if gk < 0:
        return not strict.any() and np.isinf(gd)
    e = key_index.get(int(gk))
    if e is None or not maybe[e]:
        return False
    band = tie_band(d[e], scale)
    return (lo - band <= d[e] <= hi + band) and abs(gd - d[e]) <= 1e-6 * scale + 2e-7 * d[e]


# ---------------------------------------------------------------------------
# ray casts against the Neumann primitives
# ---------------------------------------------------------------------------
def ray_candidates(sc, x, v, tmax, skip, exit_only, scale):
    """For one ray x + t v: FP64 crossing parameter with every Neumann
    primitive, and whether it is a strict / permissive hit of the cast.
    Two-sided cast: t in (0, tmax], the crossing inside the primitive.
    Exit-only cast (the walk's): v against the inward normal, t in
    (-b, tmax], the crossing within about b of the primitive, b = 16 2^-24
    scale.  Returns (prim ids, t, strict, maybe)."""
    V, P, bc = sc.verts, sc.prims, sc.bc
    ids = np.nonzero(bc == 1)[0]
    if skip is not None and skip >= 0:
        ids = ids[ids != skip]
    b = 16 * U * scale if exit_only else 0.0
    vn = np.linalg.norm(v)
    if sc.dim == 2:
        A, B = V[P[ids, 0]], V[P[ids, 1]]
        e = B - A
        L = np.linalg.norm(e, axis=1)
        ax = A - x
        den = v[0] * e[:, 1] - v[1] * e[:, 0]
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (ax[:, 0] * e[:, 1] - ax[:, 1] * e[:, 0]) / den
            s = (ax[:, 0] * v[1] - ax[:, 1] * v[0]) / den
            kap = (np.linalg.norm(ax, axis=1) + L) * vn / np.abs(den)
        eta = b / L
        params = [(s, -eta, 1 + eta, 32 * U * kap)]
        d_t = 32 * U * kap * (L + np.linalg.norm(ax, axis=1))
        d_den = 32 * U * L * vn
    else:
        A, B, Cc = V[P[ids, 0]], V[P[ids, 1]], V[P[ids, 2]]
        e1, e2 = B - A, Cc - A
        pv = np.cross(v[None, :], e2)
        det = (e1 * pv).sum(1)
        tv = x - A
        qv = np.cross(tv, e1)
        with np.errstate(divide="ignore", invalid="ignore"):
            u = (tv * pv).sum(1) / det
            w = (qv * v[None, :]).sum(1) / det
            t = (e2 * qv).sum(1) / det
            n1, n2 = np.linalg.norm(e1, axis=1), np.linalg.norm(e2, axis=1)
            nt = np.linalg.norm(tv, axis=1)
            kap = n1 * n2 * vn / np.abs(det) * (1 + (nt + n1 + n2) / np.minimum(n1, n2))
        nrm = np.linalg.norm(np.cross(e1, e2), axis=1)
        l2 = np.maximum(np.maximum(n1 ** 2, n2 ** 2), np.linalg.norm(e2 - e1, axis=1) ** 2)
        eta = b * np.sqrt(l2) / nrm
        params = [(u, -eta, 1 + eta, 32 * U * kap), (w, -eta, np.inf, 32 * U * kap),
                  (u + w, -np.inf, 1 + eta, 64 * U * kap)]
        d_t = 32 * U * kap * (nt + n1 + n2)
        d_den = 32 * U * n1 * n2 * vn
        den = -det          # exit iff det < 0
    d_t = np.nan_to_num(d_t, nan=np.inf, posinf=np.inf)
    band = 16 * U * (scale + tmax)
    if exit_only:
        o_strict, o_maybe = den > d_den, den > -d_den
    else:
        o_strict, o_maybe = np.abs(den) > d_den, np.ones(len(ids), bool)
    strict, maybe = o_strict.copy(), o_maybe.copy()
    for q, lo, hi, dq in params:
        dq = np.nan_to_num(dq, nan=np.inf, posinf=np.inf)
        strict &= (q > lo + dq) & (q < hi - dq)
        maybe &= (q >= lo - dq) & (q <= hi + dq)
    tlo = -b
    strict &= (t > tlo + d_t) & (t <= tmax - np.maximum(d_t, band))
    maybe &= (t > tlo - d_t) & (t <= tmax + np.maximum(d_t, band))
    strict &= np.isfinite(t)
    maybe &= np.isfinite(t) | ~np.isfinite(d_t)
    return ids, np.where(np.isfinite(t), t, np.inf), strict, maybe, d_t


def ray_answer_ok(gi, gt, cand, scale, tmax):
    """The GPU's (primitive id, FP32 t) is a valid answer for one ray."""
    ids, t, strict, maybe, d_t = cand
    inf = np.inf
    lo = t[maybe].min() if maybe.any() else inf
    hi = t[strict].min() if strict.any() else inf
    band = 16 * U * (scale + tmax)
    if gi < 0:
        return not strict.any()
    j = np.nonzero(ids == gi)[0]
    if len(j) == 0 or not maybe[j[0]]:
        return False
    j = j[0]
    tol = max(d_t[j], band) if np.isfinite(d_t[j]) else inf
    return (lo - tol <= t[j] <= hi + tol) and abs(gt - t[j]) <= max(tol, 1e-5 * (1 + abs(t[j])))
