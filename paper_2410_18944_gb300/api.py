"""Python binding of libwost with the C ABI's names (include/wost.h).

Only argument marshalling happens here: arrays are passed as host pointers
(numpy) or device pointers (torch CUDA tensors); every computation runs in the
CUDA library.  PyTorch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional

import numpy as np

from . import _lib as L
from ._lib import Exec, FieldDesc, SceneDesc, Stats, check


def _is_cuda_tensor(a):
    return hasattr(a, "is_cuda") and a.is_cuda


def _ptr(a, dtype):
    """(pointer, on_device, keepalive) for a numpy array or a torch tensor."""
    if _is_cuda_tensor(a):
        return C.c_void_p(a.data_ptr()), 1, a
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr.ctypes.data_as(C.c_void_p), 0, arr


def _fn(desc) -> L.Fn:
    f = L.Fn()
    f.kind = int(desc.kind)
    f.nparams = len(desc.params)
    for i, v in enumerate(desc.params[:40]):
        f.params[i] = float(v)
    return f


def exec_defaults(**kw) -> Exec:
    e = Exec()
    L.load().wost_exec_defaults(C.byref(e))
    for k, v in kw.items():
        if k == "stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream
        setattr(e, k, v)
    return e


class Scene:
    """wost_create_scene / wost_destroy_scene around a ``wost_inputs.Scene``
    (or any object with dim, verts, prims, bc, g, f, h, scene_id)."""

    def __init__(self, sc):
        lib = L.load()
        self.dim = sc.dim
        self.src = sc
        self._V = np.ascontiguousarray(sc.verts, np.float64)
        self._P = np.ascontiguousarray(sc.prims, np.int32)
        self._bc = np.ascontiguousarray(sc.bc, np.uint8)
        d = SceneDesc()
        d.dim = sc.dim
        d.nverts = len(self._V)
        d.verts = self._V.ctypes.data_as(C.POINTER(C.c_double))
        d.nprims = len(self._P)
        d.prims = self._P.ctypes.data_as(C.POINTER(C.c_int32))
        d.bc = self._bc.ctypes.data_as(C.POINTER(C.c_uint8))
        d.g = _fn(sc.g)
        d.f = _fn(sc.f)
        d.h = _fn(sc.h)
        d.scene_id = getattr(sc, "scene_id", 0)
        h = C.c_void_p()
        check(lib.wost_create_scene(C.byref(d), C.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            L.load().wost_destroy_scene(self._h)
            self._h = None

    __del__ = close

    def device(self):
        d = C.c_int32()
        check(L.load().wost_scene_device(self._h, C.byref(d)))
        return d.value

    def bbox(self):
        lo, hi = np.zeros(3), np.zeros(3)
        check(L.load().wost_scene_bbox(self._h, lo.ctypes.data_as(L._dp), hi.ctypes.data_as(L._dp)))
        return lo[:self.dim], hi[:self.dim]

    # ---- queries ----
    def query_closest(self, pts):
        p = np.ascontiguousarray(pts, np.float64)
        n = len(p)
        idx = np.zeros(n, np.int32)
        d = np.zeros(n, np.float32)
        check(L.load().wost_query_closest(self._h, p.ctypes.data_as(L._dp), n, idx.ctypes.data_as(L._i32p),
                                          d.ctypes.data_as(L._fp)))
        return idx, d

    def query_silhouette(self, pts):
        p = np.ascontiguousarray(pts, np.float64)
        n = len(p)
        idx = np.zeros(n, np.int64)
        d = np.zeros(n, np.float32)
        check(L.load().wost_query_silhouette(self._h, p.ctypes.data_as(L._dp), n, idx.ctypes.data_as(L._i64p),
                                             d.ctypes.data_as(L._fp)))
        return idx, d

    def query_ray(self, org, dirs, tmax, skip=None, exit_only=False):
        """wost_query_ray (first hit of either orientation) or, with
        ``exit_only``, wost_query_ray_exit (the cast of a walk step)."""
        o = np.ascontiguousarray(org, np.float64)
        v = np.ascontiguousarray(dirs, np.float64)
        n = len(o)
        t = np.ascontiguousarray(np.broadcast_to(np.asarray(tmax, np.float64), (n,)))
        s = None if skip is None else np.ascontiguousarray(np.broadcast_to(np.asarray(skip, np.int32), (n,)))
        idx = np.zeros(n, np.int32)
        th = np.zeros(n, np.float32)
        fn = L.load().wost_query_ray_exit if exit_only else L.load().wost_query_ray
        check(fn(self._h, o.ctypes.data_as(L._dp), v.ctypes.data_as(L._dp), t.ctypes.data_as(L._dp),
                 s.ctypes.data_as(L._i32p) if s is not None else None, n, idx.ctypes.data_as(L._i32p),
                 th.ctypes.data_as(L._fp)))
        return idx, th


class Field:
    """wost_create_field / parameters / decode / training records."""

    def __init__(self, dim, lo=None, hi=None, **kw):
        lib = L.load()
        d = FieldDesc()
        lib.wost_field_desc_defaults(C.byref(d), dim)
        if lo is not None:
            for k in range(dim):
                d.lo[k] = float(lo[k])
                d.hi[k] = float(hi[k])
        for k, v in kw.items():
            setattr(d, k, v)
        self.desc = d
        self.dim = dim
        self.K = d.K
        self.nout = (dim + 2) * d.K + 1
        self.T = 1 << d.log2_table
        h = C.c_void_p()
        check(lib.wost_create_field(C.byref(d), C.byref(h)))
        self._h = h
        n = C.c_int64()
        check(lib.wost_field_grid_entries(h, C.byref(n)))
        self.entries = n.value

    def close(self):
        if getattr(self, "_h", None):
            L.load().wost_destroy_field(self._h)
            self._h = None

    __del__ = close

    def shapes(self):
        d = self.desc
        nin = d.levels * d.features
        grid = (d.levels, self.T, d.features) if d.grid_type == 0 else (self.entries, d.features)
        return dict(grid=grid, W1=(d.hidden, nin), W2=(d.hidden, d.hidden),
                    W3=(self.nout, d.hidden), b3=(self.nout,))

    def set_params(self, grid, W1, W2, W3, b3):
        arrs = [np.ascontiguousarray(a, np.float32) for a in (grid, W1, W2, W3, b3)]
        for a, (k, s) in zip(arrs, self.shapes().items()):
            if a.shape != s:
                raise ValueError(f"{k}: shape {a.shape}, expected {s}")
        check(L.load().wost_field_set_params(self._h, *[a.ctypes.data_as(L._fp) for a in arrs]))

    def get_params(self):
        out = {k: np.zeros(s, np.float32) for k, s in self.shapes().items()}
        check(L.load().wost_field_get_params(self._h, *[out[k].ctypes.data_as(L._fp) for k in
                                                        ("grid", "W1", "W2", "W3", "b3")]))
        return out

    def decode(self, pts, exec_=None, out=None):
        """wost_field_decode: raw outputs (n, nout).  ``pts`` is a numpy array
        (host) or a CUDA float64 tensor (device; then the result is a CUDA
        float32 tensor, ``out`` optional)."""
        e = exec_ or exec_defaults()
        if _is_cuda_tensor(pts):
            import torch
            if out is None:
                out = torch.empty((pts.shape[0], self.nout), dtype=torch.float32, device=pts.device)
            e.points_on_device = 1
            e.out_on_device = 1
            check(L.load().wost_field_decode(self._h, C.c_void_p(pts.data_ptr()), pts.shape[0],
                                             C.c_void_p(out.data_ptr()), C.byref(e)))
            return out
        p = np.ascontiguousarray(pts, np.float64)
        out = np.zeros((len(p), self.nout), np.float32)
        check(L.load().wost_field_decode(self._h, p.ctypes.data_as(C.c_void_p), len(p),
                                         out.ctypes.data_as(C.c_void_p), C.byref(e)))
        return out

    def set_records(self, recs, c_mode=0, c_fixed=0.5, reflect=1):
        r = np.ascontiguousarray(recs, np.float32)
        e = exec_defaults(c_mode=c_mode, c_fixed=c_fixed, reflect=reflect)
        check(L.load().wost_train_records(self._h, r.ctypes.data_as(C.c_void_p), len(r), C.byref(e)))

    def get_records(self, cap=None):
        n = C.c_int64()
        check(L.load().wost_get_records(self._h, None, 0, C.byref(n)))
        m = n.value if cap is None else min(cap, n.value)
        out = np.zeros((m, 12), np.float32)
        check(L.load().wost_get_records(self._h, out.ctypes.data_as(L._fp), m, C.byref(n)))
        return out

    def train_grad(self, samples=0):
        """wost_train_grad on the record buffer (all records, or the strided
        subset of about ``samples`` records, exec train_samples)."""
        g = {k: np.zeros(s, np.float32) for k, s in self.shapes().items()}
        loss = C.c_float()
        e = exec_defaults(train_samples=int(samples))
        check(L.load().wost_train_grad(self._h, C.byref(e), C.byref(loss),
                                       *[g[k].ctypes.data_as(L._fp) for k in ("grid", "W1", "W2", "W3", "b3")]))
        return loss.value, g

    def train_step(self, scene: Optional[Scene] = None, exec_=None):
        loss = C.c_float()
        e = exec_ or exec_defaults()
        check(L.load().wost_train_step(scene._h if scene else None, self._h, C.byref(e), C.byref(loss)))
        return loss.value


def solve(scene: Scene, points, nwalks, eps=1e-3, maxsteps=128, guided=False, field: Optional[Field] = None,
          with_var=True, **exec_kw):
    """wost_solve.  ``points`` is a numpy array (host) or a torch CUDA tensor
    (device, float64, shape (n, dim)); outputs follow the points' location.
    Returns (mean, var, stats dict)."""
    lib = L.load()
    e = exec_defaults(**exec_kw)
    n = len(points)
    pp, on_dev, keep = _ptr(points, np.float64)
    e.points_on_device = on_dev
    e.out_on_device = on_dev
    if on_dev:
        import torch
        mean = torch.empty(n, dtype=torch.float64, device=points.device)
        var = torch.empty(n, dtype=torch.float64, device=points.device) if with_var else None
        mp, vp = C.c_void_p(mean.data_ptr()), (C.c_void_p(var.data_ptr()) if with_var else None)
    else:
        mean = np.zeros(n)
        var = np.zeros(n) if with_var else None
        mp = mean.ctypes.data_as(C.c_void_p)
        vp = var.ctypes.data_as(C.c_void_p) if with_var else None
    st = Stats()
    check(lib.wost_solve(scene._h, field._h if field is not None else None, pp, n, int(nwalks), float(eps),
                         int(maxsteps), 1 if guided else 0, mp, vp, C.byref(st), C.byref(e)))
    return mean, var, st.as_dict()


def _job_array(jobs, with_var):
    """ctypes wost_job array for job dicts; returns (array, means, vars, keepalive)."""
    import torch
    arr = (L.Job * len(jobs))()
    means, vars_, keep = [], [], []
    for j, spec in enumerate(jobs):
        pts = spec["points"]
        if not _is_cuda_tensor(pts) or pts.dtype != torch.float64 or not pts.is_contiguous():
            raise ValueError("batch points must be contiguous float64 CUDA tensors")
        n = pts.shape[0]
        m = torch.empty(n, dtype=torch.float64, device=pts.device)
        v = torch.empty(n, dtype=torch.float64, device=pts.device) if with_var else None
        keep += [pts, spec["scene"], spec.get("field")]
        means.append(m)
        vars_.append(v)
        J = arr[j]
        J.scene = spec["scene"]._h
        J.field = spec["field"]._h if spec.get("field") is not None else None
        J.points = pts.data_ptr()
        J.npoints = n
        J.nwalks = int(spec["nwalks"])
        J.eps = float(spec.get("eps", 1e-3))
        J.maxsteps = int(spec.get("maxsteps", 128))
        J.seed = int(spec.get("seed", 1))
        J.out_mean = m.data_ptr()
        J.out_var = v.data_ptr() if v is not None else None
    return arr, means, vars_, keep


class Batch:
    """wost_batch_create / wost_batch_run / wost_batch_destroy: many scenes in
    one persistent launch, replayed from a captured CUDA graph.

    ``jobs`` is a sequence of dicts with keys scene (Scene), points (torch
    CUDA float64 tensor (n, dim)), nwalks, and optionally eps (1e-3),
    maxsteps (128), seed (1), field (Field, guided batches).  The plan owns
    the output tensors ``mean[j]`` / ``var[j]`` and keeps the points alive."""

    def __init__(self, jobs, guided=False, with_var=True, **exec_kw):
        self._h = None
        lib = L.load()
        self._jobs, self.mean, self.var, self._keep = _job_array(jobs, with_var)
        e = exec_defaults(**exec_kw)
        h = C.c_void_p()
        check(lib.wost_batch_create(len(jobs), self._jobs, 1 if guided else 0, C.byref(e), C.byref(h)))
        self._h = h

    def run(self, stream=None):
        """Replays the plan; returns the summed stats dict."""
        st = Stats()
        check(L.load().wost_batch_run(self._h, stream, C.byref(st)))
        return st.as_dict()

    def info(self):
        bi = L.BatchInfo()
        check(L.load().wost_batch_info_get(self._h, C.byref(bi)))
        return bi.as_dict()

    def close(self):
        if self._h:
            L.load().wost_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve_batch(jobs, guided=False, with_var=True, **exec_kw):
    """wost_solve_batch (plan, run, release in one call): (means, vars, stats)."""
    arr, means, vars_, keep = _job_array(jobs, with_var)
    e = exec_defaults(**exec_kw)
    st = Stats()
    check(L.load().wost_solve_batch(len(jobs), arr, 1 if guided else 0, C.byref(e), C.byref(st)))
    del keep
    return means, vars_, st.as_dict()


def mixture_eval(dim, mu, kappa, lam, nu):
    mu = np.ascontiguousarray(mu, np.float32)
    kappa = np.ascontiguousarray(kappa, np.float32)
    lam = np.ascontiguousarray(lam, np.float32)
    nu = np.ascontiguousarray(nu, np.float32)
    n, K = kappa.shape
    out = np.zeros(n, np.float32)
    check(L.load().wost_mixture_eval(dim, K, mu.ctypes.data_as(L._fp), kappa.ctypes.data_as(L._fp),
                                     lam.ctypes.data_as(L._fp), nu.ctypes.data_as(L._fp), n,
                                     out.ctypes.data_as(L._fp)))
    return out


def mixture_sample(dim, mu, kappa, lam, counters, seed, scene_id=0):
    mu = np.ascontiguousarray(mu, np.float32)
    kappa = np.ascontiguousarray(kappa, np.float32)
    lam = np.ascontiguousarray(lam, np.float32)
    ctr = np.ascontiguousarray(counters, np.uint32)
    n, K = kappa.shape
    nu = np.zeros((n, dim), np.float32)
    pdf = np.zeros(n, np.float32)
    check(L.load().wost_mixture_sample(dim, K, mu.ctypes.data_as(L._fp), kappa.ctypes.data_as(L._fp),
                                       lam.ctypes.data_as(L._fp), ctr.ctypes.data_as(L._u32p), seed, scene_id, n,
                                       nu.ctypes.data_as(L._fp), pdf.ctypes.data_as(L._fp)))
    return nu, pdf


def diag_umma(a_mn, b_mn, A, B):
    A = np.ascontiguousarray(A, np.float32)
    B = np.ascontiguousarray(B, np.float32)
    N, K = B.shape
    D = np.zeros((128, N), np.float32)
    check(L.load().wost_diag_umma(a_mn, b_mn, N, K, A.ctypes.data_as(L._fp), B.ctypes.data_as(L._fp),
                                  D.ctypes.data_as(L._fp)))
    return D
