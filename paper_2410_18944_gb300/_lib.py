"""ctypes view of libwost (include/wost.h).  Argument marshalling only: every
step of the walk runs in the CUDA library.  There is no fallback -- if the
library has not been built, or cannot be loaded, this module raises."""
from __future__ import annotations

import ctypes as C
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libwost.so")
_lock = threading.Lock()
_lib = None

WOST_OK = 0
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "ILL_POSED", 3: "CUDA", 4: "TIMEOUT", 5: "OOM", 6: "UNSUPPORTED"}


class WostError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"wost status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Fn(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nparams", C.c_int32), ("params", C.c_double * 40)]


class SceneDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("nverts", C.c_int64), ("verts", C.POINTER(C.c_double)),
                ("nprims", C.c_int64), ("prims", C.POINTER(C.c_int32)), ("bc", C.POINTER(C.c_uint8)),
                ("g", Fn), ("f", Fn), ("h", Fn), ("scene_id", C.c_uint32)]


class FieldDesc(C.Structure):
    _fields_ = [("dim", C.c_int32), ("K", C.c_int32), ("levels", C.c_int32), ("log2_table", C.c_int32),
                ("features", C.c_int32), ("hidden", C.c_int32), ("base_res", C.c_int32), ("max_res", C.c_int32),
                ("lo", C.c_double * 3), ("hi", C.c_double * 3), ("seed", C.c_uint64),
                ("lr_grid", C.c_float), ("lr_mlp", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("adam_eps", C.c_float), ("e_sel", C.c_float), ("grid_type", C.c_int32)]


class Exec(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("stream", C.c_void_p), ("points_on_device", C.c_int32),
                ("out_on_device", C.c_int32), ("c_mode", C.c_int32), ("c_fixed", C.c_float),
                ("reflect", C.c_int32), ("train", C.c_int32), ("train_until_wpp", C.c_int32),
                ("max_train_records", C.c_int64), ("walk_begin", C.c_int32), ("ctas_per_sm", C.c_int32),
                ("guided_kernel", C.c_int32), ("wavefront_slots", C.c_int32),
                ("train_samples", C.c_int64), ("rr_depth", C.c_int32), ("rr_survival", C.c_float),
                ("wait_ns", C.c_int64), ("batch_wpp", C.c_int32),
                ("walker_warps", C.c_int32)]


class Stats(C.Structure):
    _fields_ = [("walk_steps", C.c_int64), ("walks", C.c_int64), ("truncated", C.c_int64),
                ("records", C.c_int64), ("records_dropped", C.c_int64), ("train_steps", C.c_int32),
                ("last_loss", C.c_float), ("ms_walk", C.c_double), ("ms_train", C.c_double),
                ("kernel_launches", C.c_int64), ("walk_launches", C.c_int64), ("node_visits", C.c_int64),
                ("prim_visits", C.c_int64), ("alg_bytes", C.c_double), ("dir_prim_visits", C.c_int64),
                ("sil_prim_visits", C.c_int64), ("neu_prim_visits", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Job(C.Structure):
    _fields_ = [("scene", C.c_void_p), ("field", C.c_void_p), ("points", C.c_void_p), ("npoints", C.c_int64),
                ("nwalks", C.c_int32), ("eps", C.c_double), ("maxsteps", C.c_int32), ("seed", C.c_uint64),
                ("out_mean", C.c_void_p), ("out_var", C.c_void_p)]


class BatchInfo(C.Structure):
    _fields_ = [("ctas_per_sm", C.c_int32), ("flush_polls", C.c_int32), ("candidates", C.c_int32),
                ("best_ms", C.c_double), ("worst_ms", C.c_double), ("walk_launches", C.c_int32),
                ("train_steps", C.c_int32), ("graph_nodes", C.c_int64),
                ("walker_warps", C.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp = C.c_void_p
_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_u32p = C.POINTER(C.c_uint32)

# name -> (restype, argtypes)
SIGNATURES = {
    "wost_last_error": (C.c_char_p, []),
    "wost_exec_defaults": (None, [C.POINTER(Exec)]),
    "wost_field_desc_defaults": (None, [C.POINTER(FieldDesc), C.c_int32]),
    "wost_create_scene": (C.c_int, [C.POINTER(SceneDesc), C.POINTER(_vp)]),
    "wost_destroy_scene": (C.c_int, [_vp]),
    "wost_scene_bbox": (C.c_int, [_vp, _dp, _dp]),
    "wost_scene_device": (C.c_int, [_vp, _i32p]),
    "wost_diag_scene_rebind": (C.c_int, [_vp, C.c_int32]),
    "wost_solve": (C.c_int, [_vp, _vp, _vp, C.c_int64, C.c_int32, C.c_double, C.c_int32, C.c_int32,
                             _vp, _vp, C.POINTER(Stats), C.POINTER(Exec)]),
    "wost_create_field": (C.c_int, [C.POINTER(FieldDesc), C.POINTER(_vp)]),
    "wost_destroy_field": (C.c_int, [_vp]),
    "wost_field_set_params": (C.c_int, [_vp, _fp, _fp, _fp, _fp, _fp]),
    "wost_field_get_params": (C.c_int, [_vp, _fp, _fp, _fp, _fp, _fp]),
    "wost_field_decode": (C.c_int, [_vp, _vp, C.c_int64, _vp, C.POINTER(Exec)]),
    "wost_field_grid_entries": (C.c_int, [_vp, _i64p]),
    "wost_train_step": (C.c_int, [_vp, _vp, C.POINTER(Exec), _fp]),
    "wost_train_records": (C.c_int, [_vp, _vp, C.c_int64, C.POINTER(Exec)]),
    "wost_get_records": (C.c_int, [_vp, _fp, C.c_int64, _i64p]),
    "wost_train_grad": (C.c_int, [_vp, C.POINTER(Exec), _fp, _fp, _fp, _fp, _fp, _fp]),
    "wost_train_loss": (C.c_int, [_vp, C.POINTER(Exec), _vp]),
    "wost_query_closest": (C.c_int, [_vp, _dp, C.c_int64, _i32p, _fp]),
    "wost_query_silhouette": (C.c_int, [_vp, _dp, C.c_int64, _i64p, _fp]),
    "wost_query_ray": (C.c_int, [_vp, _dp, _dp, _dp, _i32p, C.c_int64, _i32p, _fp]),
    "wost_query_ray_exit": (C.c_int, [_vp, _dp, _dp, _dp, _i32p, C.c_int64, _i32p, _fp]),
    "wost_mixture_eval": (C.c_int, [C.c_int32, C.c_int32, _fp, _fp, _fp, _fp, C.c_int64, _fp]),
    "wost_mixture_sample": (C.c_int, [C.c_int32, C.c_int32, _fp, _fp, _fp, _u32p, C.c_uint64, C.c_uint32,
                                      C.c_int64, _fp, _fp]),
    "wost_diag_umma": (C.c_int, [C.c_int32, C.c_int32, C.c_int32, C.c_int32, _fp, _fp, _fp]),
    "wost_diag_wait": (C.c_int, [C.c_int64, C.c_int32]),
    "wost_batch_create": (C.c_int, [C.c_int32, C.POINTER(Job), C.c_int32, C.POINTER(Exec), C.POINTER(_vp)]),
    "wost_batch_run": (C.c_int, [_vp, _vp, C.POINTER(Stats)]),
    "wost_batch_info_get": (C.c_int, [_vp, C.POINTER(BatchInfo)]),
    "wost_batch_destroy": (C.c_int, [_vp]),
    "wost_solve_batch": (C.c_int, [C.c_int32, C.POINTER(Job), C.c_int32, C.POINTER(Exec), C.POINTER(Stats)]),
    "wost_solve_plain_static": (C.c_int, [_vp, _vp, C.c_int64, C.c_int32, C.c_double, C.c_int32, C.c_uint64, _vp,
                                          _vp, _vp, _i64p]),
}


def load():
    """Load the built library; raises if it is missing (no CPU fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libwost is not built ({LIB_PATH} missing); run __graft_entry__.build() "
                                   "or python -m paper_2410_18944_gb300.build")
            lib = C.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def check(status):
    if status != WOST_OK:
        msg = load().wost_last_error()
        raise WostError(status, msg.decode() if msg else "")
