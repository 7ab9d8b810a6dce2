"""CPU FP64 oracle for guided walk on stars -- TEST INFRASTRUCTURE ONLY.

Plain, slow restatement of the paper's method (arXiv 2410.18944) in C
(``oracle/*.c``), loaded through ctypes.  Only ``tests/``, the smoke check and
the benchmark's CPU-baseline leg may import this package; the CUDA library and
its Python binding never do.  Nothing here is shared with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = ["philox.c", "scene.c", "vmf.c", "field.c", "walk.c", "train.c"]
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

REC = 12  # doubles per training record: x[3], nu[3], n[3], on_neumann, q, target


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2)."""
    srcs = [os.path.join(_HERE, s) for s in _SRC]
    hdr = os.path.join(_HERE, "oracle.h")
    if not force and os.path.exists(_LIB_PATH):
        t = os.path.getmtime(_LIB_PATH)
        if all(os.path.getmtime(s) <= t for s in srcs + [hdr]):
            return _LIB_PATH
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm", "-lpthread"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int32)
_u32p = C.POINTER(C.c_uint32)


class Params(C.Structure):
    _fields_ = [("eps", C.c_double), ("maxsteps", C.c_int), ("guided", C.c_int),
                ("c_mode", C.c_int), ("c_fixed", C.c_double), ("reflect", C.c_int),
                ("seed", C.c_uint64), ("scene_id", C.c_uint32), ("nthreads", C.c_int),
                ("rr_depth", C.c_int), ("rr_survival", C.c_double)]


class _Field(C.Structure):
    _fields_ = [("dim", C.c_int), ("K", C.c_int), ("L", C.c_int), ("log2T", C.c_int),
                ("F", C.c_int), ("H", C.c_int), ("base_res", C.c_int), ("max_res", C.c_int),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3),
                ("grid", _dp), ("W1", _dp), ("W2", _dp), ("W3", _dp), ("b3", _dp), ("grid_type", C.c_int)]


def _declare(L):
    L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.orc_u01.restype = C.c_double
    L.orc_u01.argtypes = [C.c_uint32]
    L.orc_scene_create.restype = C.c_void_p
    L.orc_scene_create.argtypes = [C.c_int, C.c_int, _dp, C.c_int, _ip, C.POINTER(C.c_uint8),
                                   C.c_int, _dp, C.c_int, C.c_int, _dp, C.c_int, C.c_int, _dp, C.c_int]
    L.orc_neumann_sample.argtypes = [C.c_void_p, _dp, C.c_double, _u32p, C.c_uint32, C.c_uint32, C.c_uint32,
                                     _dp, _dp]
    L.orc_scene_free.argtypes = [C.c_void_p]
    L.orc_scene_nsil.argtypes = [C.c_void_p]
    L.orc_scene_scale.argtypes = [C.c_void_p]
    L.orc_scene_scale.restype = C.c_double
    L.orc_eval_fn.restype = C.c_double
    L.orc_eval_fn.argtypes = [C.c_int, _dp, C.c_int, _dp]
    L.orc_closest_dirichlet.argtypes = [C.c_void_p, _dp, _dp, _dp]
    L.orc_closest_silhouette.argtypes = [C.c_void_p, _dp, _dp]
    L.orc_ray_neumann.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, _dp]
    L.orc_ray_neumann_exit.argtypes = [C.c_void_p, _dp, _dp, C.c_double, C.c_int, _dp]
    L.orc_winding.restype = C.c_double
    L.orc_winding.argtypes = [C.c_void_p, _dp]
    L.orc_inward_normal.argtypes = [C.c_void_p, C.c_int, _dp]
    L.orc_i0e.restype = C.c_double
    L.orc_i0e.argtypes = [C.c_double]
    L.orc_i1e.restype = C.c_double
    L.orc_i1e.argtypes = [C.c_double]
    L.orc_vmf_pdf.restype = C.c_double
    L.orc_vmf_pdf.argtypes = [C.c_int, C.c_double, _dp, _dp]
    L.orc_vmf_mean_cos.restype = C.c_double
    L.orc_vmf_mean_cos.argtypes = [C.c_int, C.c_double]
    L.orc_vmf2_sample_angle.restype = C.c_double
    L.orc_vmf2_sample_angle.argtypes = [C.c_double, _u32p, C.c_uint32, C.c_uint32, C.c_uint32, _ip]
    L.orc_vmf3_sample.argtypes = [C.c_double, _dp, C.c_double, C.c_double, _dp]
    L.orc_guided_draw.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, C.c_double, _u32p, C.c_uint32, C.c_uint32,
                                  C.c_uint32, _dp]
    L.orc_mixture_pdf.restype = C.c_double
    L.orc_mixture_pdf.argtypes = [C.c_int, C.c_int, _dp, _dp, _dp, _dp]
    L.orc_field_nout.argtypes = [C.POINTER(_Field)]
    L.orc_field_entries.restype = C.c_int64
    L.orc_field_entries.argtypes = [C.POINTER(_Field)]
    L.orc_level_res.argtypes = [C.POINTER(_Field), C.c_int]
    L.orc_field_encode.argtypes = [C.POINTER(_Field), _dp, _dp]
    L.orc_field_forward.argtypes = [C.POINTER(_Field), _dp, _dp]
    L.orc_theta_map.argtypes = [C.POINTER(_Field), _dp, _dp, _dp, _dp, _dp]
    L.orc_point_status.argtypes = [C.c_void_p, _dp, C.c_double, _dp]
    L.orc_walk.restype = C.c_double
    L.orc_walk.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(Params), C.c_uint32, C.c_uint32, _dp,
                           _ip, _ip, _dp, C.c_int, _ip]
    L.orc_walk_terms.restype = C.c_double
    L.orc_walk_terms.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(Params), C.c_uint32, C.c_uint32, _dp,
                                 _ip, _ip, _dp, C.c_int, _ip, _dp]
    L.orc_solve.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(Params), _dp, C.c_int, C.c_int, C.c_int,
                            _dp, _dp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), _dp, _ip]
    L.orc_train_loss.restype = C.c_double
    L.orc_train_loss.argtypes = [C.POINTER(_Field), _dp, C.c_int, C.c_double, C.c_int, C.c_double, C.c_int,
                                 _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.orc_adam.argtypes = [_dp, _dp, _dp, _dp, C.c_int64, C.c_double, C.c_double, C.c_double,
                           C.c_double, C.c_int]


def _d(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def philox(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [o[i] for i in range(4)]


def eval_fn(kind, params, x):
    x = _f64(x)
    p = _f64(list(params) + [0.0] * 8)
    return np.array([lib().orc_eval_fn(kind, _d(p), x.shape[1], _d(xi)) for xi in x])


# ---- scene ------------------------------------------------------------------

class Scene:
    """Oracle-side copy of a ``wost_inputs.Scene``."""

    def __init__(self, sc):
        self.src = sc
        self.dim = sc.dim
        V = _f64(sc.verts)
        P = np.ascontiguousarray(sc.prims, np.int32)
        bc = np.ascontiguousarray(sc.bc, np.uint8)
        g = _f64(list(sc.g.params) + [0.0] * 10)
        f = _f64(list(sc.f.params) + [0.0] * 10)
        h = _f64(list(sc.h.params) + [0.0] * 10)
        self._h = lib().orc_scene_create(sc.dim, len(V), _d(V), len(P), P.ctypes.data_as(_ip),
                                         bc.ctypes.data_as(C.POINTER(C.c_uint8)), sc.g.kind, _d(g),
                                         len(g), sc.f.kind, _d(f), len(f), sc.h.kind, _d(h), len(h))

    def __del__(self):
        if getattr(self, "_h", None) and lib is not None:
            try:
                lib().orc_scene_free(self._h)
            except Exception:
                pass
            self._h = None

    @property
    def nsil(self):
        return lib().orc_scene_nsil(self._h)

    @property
    def scale(self):
        return lib().orc_scene_scale(self._h)

    def closest_dirichlet(self, pts):
        pts = _f64(pts)
        n = len(pts)
        idx = np.zeros(n, np.int32)
        dist = np.zeros(n)
        xb = np.zeros((n, 3))
        d = C.c_double()
        for i in range(n):
            q = np.zeros(3)
            idx[i] = lib().orc_closest_dirichlet(self._h, _d(pts[i]), C.byref(d), _d(q))
            dist[i] = d.value
            xb[i] = q
        return idx, dist, xb[:, :self.dim]

    def closest_silhouette(self, pts):
        pts = _f64(pts)
        n = len(pts)
        idx = np.zeros(n, np.int32)
        dist = np.zeros(n)
        d = C.c_double()
        for i in range(n):
            idx[i] = lib().orc_closest_silhouette(self._h, _d(pts[i]), C.byref(d))
            dist[i] = d.value
        return idx, dist

    def ray_neumann(self, org, dirs, tmax, skip=None, exit_only=False):
        """First Neumann hit per ray (all hits, or with exit_only the first
        primitive the ray leaves the domain through, as the walks cast)."""
        org, dirs = _f64(org), _f64(dirs)
        n = len(org)
        tmax = np.broadcast_to(np.asarray(tmax, float), (n,))
        skip = np.full(n, -1, np.int32) if skip is None else np.broadcast_to(np.asarray(skip, np.int32), (n,))
        idx = np.zeros(n, np.int32)
        t = np.zeros(n)
        tt = C.c_double()
        fn = lib().orc_ray_neumann_exit if exit_only else lib().orc_ray_neumann
        for i in range(n):
            idx[i] = fn(self._h, _d(org[i]), _d(dirs[i]), float(tmax[i]), int(skip[i]), C.byref(tt))
            t[i] = tt.value
        return idx, t

    def neumann_sample(self, x, r, key, pid, wid, step):
        """(primitive, z, W) of the <N> sample at x within radius r."""
        x3 = np.zeros(3)
        x3[:self.dim] = x
        z = np.zeros(3)
        W = C.c_double()
        k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
        i = lib().orc_neumann_sample(self._h, _d(x3), float(r), k, pid, wid, step, _d(z), C.byref(W))
        return i, z[:self.dim], W.value

    def winding(self, pts):
        pts = _f64(pts)
        return np.array([lib().orc_winding(self._h, _d(p)) for p in pts])

    def inward_normal(self, prim):
        n = np.zeros(3)
        lib().orc_inward_normal(self._h, int(prim), _d(n))
        return n[:self.dim]

    def point_status(self, pts, eps):
        pts = _f64(pts)
        st = np.zeros(len(pts), np.int32)
        val = np.zeros(len(pts))
        v = C.c_double()
        for i, p in enumerate(pts):
            st[i] = lib().orc_point_status(self._h, _d(p), eps, C.byref(v))
            val[i] = v.value
        return st, val


# ---- vMF --------------------------------------------------------------------

def i0e(x):
    return lib().orc_i0e(float(x))


def i1e(x):
    return lib().orc_i1e(float(x))


def vmf_pdf(dim, kappa, mu, nu):
    mu, nu = _f64(mu), _f64(nu)
    return lib().orc_vmf_pdf(dim, float(kappa), _d(mu), _d(nu))


def vmf_mean_cos(dim, kappa):
    return lib().orc_vmf_mean_cos(dim, float(kappa))


def vmf2_sample_angle(kappa, key, pid, wid, step):
    k = (C.c_uint32 * 2)(*key)
    nt = C.c_int32()
    th = lib().orc_vmf2_sample_angle(float(kappa), k, pid, wid, step, C.byref(nt))
    return th, nt.value


def vmf3_sample(kappa, mu, xi, xi2):
    mu = _f64(mu)
    nu = np.zeros(3)
    lib().orc_vmf3_sample(float(kappa), _d(mu), float(xi), float(xi2), _d(nu))
    return nu


def guided_draw(dim, mu, kappa, lam, c, key, pid, wid, step):
    mu, kappa, lam = _f64(mu).ravel(), _f64(kappa), _f64(lam)
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    nu = np.zeros(3)
    hit = lib().orc_guided_draw(dim, len(kappa), _d(mu), _d(kappa), _d(lam), float(c), k, pid, wid, step, _d(nu))
    return hit, nu[:dim]


def mixture_pdf(dim, mu, kappa, lam, nu):
    mu, kappa, lam, nu = _f64(mu).ravel(), _f64(kappa), _f64(lam), _f64(nu)
    return lib().orc_mixture_pdf(dim, len(kappa), _d(mu), _d(kappa), _d(lam), _d(nu))


# ---- field ------------------------------------------------------------------

@dataclass
class FieldParams:
    """Neural-field parameters in the exchange layout (all float64):
    grid (L, T, F), W1 (H, L*F), W2 (H, H), W3 (nout, H), b3 (nout)."""
    dim: int
    K: int
    L: int
    log2T: int
    F: int
    H: int
    base_res: int
    max_res: int
    lo: np.ndarray
    hi: np.ndarray
    grid: np.ndarray
    W1: np.ndarray
    W2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    grid_type: int = 0       # 0 hash grid, 1 dense grid

    @property
    def nout(self):
        return (self.dim + 2) * self.K + 1

    def arrays(self):
        return [self.grid, self.W1, self.W2, self.W3, self.b3]


class Field:
    def __init__(self, fp: FieldParams):
        self.fp = fp
        self._arrs = [_f64(a) for a in fp.arrays()]
        lo = list(fp.lo) + [0.0] * (3 - len(fp.lo))
        hi = list(fp.hi) + [1.0] * (3 - len(fp.hi))
        self.s = _Field(fp.dim, fp.K, fp.L, fp.log2T, fp.F, fp.H, fp.base_res, fp.max_res,
                        (C.c_double * 3)(*lo), (C.c_double * 3)(*hi),
                        *[_d(a) for a in self._arrs], int(fp.grid_type))
        if self._arrs[0].size != lib().orc_field_entries(self.ref()) * fp.F:
            raise ValueError("grid size does not match the encoding")

    def ref(self):
        return C.byref(self.s)

    def level_res(self, l):
        return lib().orc_level_res(self.ref(), l)

    def encode(self, pts):
        pts = _f64(pts)
        out = np.zeros((len(pts), self.fp.L * self.fp.F))
        for i, p in enumerate(pts):
            p3 = np.zeros(3)
            p3[:len(p)] = p
            lib().orc_field_encode(self.ref(), _d(p3), _d(out[i]))
        return out

    def forward(self, pts):
        pts = _f64(pts)
        out = np.zeros((len(pts), self.fp.nout))
        for i, p in enumerate(pts):
            p3 = np.zeros(3)
            p3[:len(p)] = p
            row = np.zeros(self.fp.nout)
            lib().orc_field_forward(self.ref(), _d(p3), _d(row))
            out[i] = row
        return out

    def theta(self, raw):
        raw = _f64(raw)
        K, d = self.fp.K, self.fp.dim
        mu = np.zeros(K * d)
        kap = np.zeros(K)
        lam = np.zeros(K)
        c = C.c_double()
        lib().orc_theta_map(self.ref(), _d(raw), _d(mu), _d(kap), _d(lam), C.byref(c))
        return mu.reshape(K, d), kap, lam, c.value

    def train_loss(self, recs, e_sel=0.2, c_mode=0, c_fixed=0.5, reflect=1, frozen_pg=None, grad=True):
        recs = _f64(recs)
        n = len(recs)
        out_pg = np.zeros(n)
        fz = _f64(frozen_pg) if frozen_pg is not None else None
        g = [np.zeros_like(a) for a in self._arrs] if grad else None
        null = C.cast(None, _dp)
        loss = lib().orc_train_loss(self.ref(), _d(recs), n, e_sel, c_mode, c_fixed, reflect,
                                    _d(fz) if fz is not None else null, _d(out_pg),
                                    *([_d(a) for a in g] if grad else [null] * 5))
        return loss, g, out_pg


def adam(p, g, m, v, lr, b1, b2, eps, t):
    for a in (p, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(_d(p), _d(g), _d(m), _d(v), p.size, lr, b1, b2, eps, t)


# ---- walks ------------------------------------------------------------------

def make_params(eps=1e-3, maxsteps=128, guided=0, c_mode=0, c_fixed=0.5, reflect=1, seed=1,
                scene_id=0, nthreads=None, rr_depth=0, rr_survival=0.95):
    return Params(eps, maxsteps, guided, c_mode, c_fixed, reflect, seed, scene_id,
                  nthreads or os.cpu_count() or 1, rr_depth, rr_survival)


def walk(scene: Scene, prm: Params, pid, wid, x0, field: Optional[Field] = None, records=False):
    """One walk.  With ``records``: its training records, and ``w`` / ``S``
    (each record's step weight and source term) and ``last`` (the walk's
    final value), the inputs of the suffix pass."""
    x = np.zeros(3)
    x[:scene.dim] = x0
    st, tr, nr = C.c_int32(), C.c_int32(), C.c_int32()
    recs = np.zeros((prm.maxsteps, REC)) if records else None
    terms = np.zeros(2 * prm.maxsteps + 1) if records else None
    v = lib().orc_walk_terms(scene._h, C.cast(C.byref(field.s), C.c_void_p) if field else None, C.byref(prm),
                             pid, wid, _d(x), C.byref(st), C.byref(tr),
                             _d(recs) if records else C.cast(None, _dp), prm.maxsteps, C.byref(nr),
                             _d(terms) if records else C.cast(None, _dp))
    out = dict(value=v, steps=st.value, truncated=tr.value)
    if records:
        n = nr.value
        out["records"] = recs[:n].copy()
        out["w"] = terms[0:2 * n:2].copy()
        out["S"] = terms[1:2 * n:2].copy()
        out["last"] = float(terms[2 * n])
    return out


def solve(scene: Scene, prm: Params, points, walk_begin, nwalks, field: Optional[Field] = None,
          records=False):
    """Returns dict(sum, sum2, steps, truncated[, records list]) over the walks."""
    pts = np.zeros((len(points), 3))
    pts[:, :scene.dim] = points
    pts = _f64(pts[:, :scene.dim])
    n = len(pts)
    s1, s2 = np.zeros(n), np.zeros(n)
    st, tr = C.c_int64(0), C.c_int64(0)
    recs = np.zeros((n, prm.maxsteps, REC)) if records else None
    nrec = np.zeros(n, np.int32)
    lib().orc_solve(scene._h, C.cast(C.byref(field.s), C.c_void_p) if field else None, C.byref(prm),
                    _d(pts), n, walk_begin, nwalks, _d(s1), _d(s2), C.byref(st), C.byref(tr),
                    _d(recs) if records else C.cast(None, _dp), nrec.ctypes.data_as(_ip))
    out = dict(sum=s1, sum2=s2, steps=st.value, truncated=tr.value)
    if records:
        out["records"] = np.concatenate([recs[i, :nrec[i]] for i in range(n)], 0)
    return out


def mean_var(sum_, sum2, n):
    mean = sum_ / n
    var = (sum2 - n * mean * mean) / (n * (n - 1)) if n > 1 else np.zeros_like(mean)
    return mean, np.maximum(var, 0)
