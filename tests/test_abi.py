"""The C-ABI library loads on a machine without a GPU and exports every
symbol declared in include/*.h (no compute calls)."""
import glob
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        names += re.findall(r"^(?:wost_status|const char \*|void)\s*\**\s*(wost_\w+)\s*\(", txt, re.M)
    return sorted(set(names))


def test_library_builds_and_exports_header_symbols():
    from paper_2410_18944_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # every binding signature names a declared symbol
    assert set(_lib.SIGNATURES) <= set(names)


def test_defaults_are_host_only():
    from paper_2410_18944_gb300 import api
    e = api.exec_defaults()
    assert e.seed == 1 and e.reflect == 1 and e.train_until_wpp == 256
    f = api.L.FieldDesc()
    api.L.load().wost_field_desc_defaults(api.C.byref(f), 3)
    assert (f.K, f.levels, f.features, f.hidden, f.log2_table, f.max_res) == (8, 16, 2, 64, 19, 512)


def test_invalid_arguments_are_rejected_without_gpu():
    import ctypes as C
    from paper_2410_18944_gb300 import _lib
    lib = _lib.load()
    h = C.c_void_p()
    assert lib.wost_create_scene(None, C.byref(h)) == 1
    d = _lib.SceneDesc()
    d.dim = 4
    assert lib.wost_create_scene(C.byref(d), C.byref(h)) == 1
    assert b"dim" in lib.wost_last_error()


def test_field_and_mixture_limits_are_checked_without_gpu():
    # argument checks come before any CUDA call: lobe counts 1..16, the
    # fixed network shape, the table size and the box
    import ctypes as C
    from paper_2410_18944_gb300 import _lib
    lib = _lib.load()
    UNSUPPORTED, INVALID = 6, 1
    h = C.c_void_p()
    for field, value, want in (("K", 0, UNSUPPORTED), ("K", 17, UNSUPPORTED), ("levels", 8, UNSUPPORTED),
                               ("hidden", 32, UNSUPPORTED), ("log2_table", 30, INVALID), ("grid_type", 2, INVALID)):
        d = _lib.FieldDesc()
        lib.wost_field_desc_defaults(C.byref(d), 2)
        setattr(d, field, value)
        assert lib.wost_create_field(C.byref(d), C.byref(h)) == want, (field, value)
    d = _lib.FieldDesc()
    lib.wost_field_desc_defaults(C.byref(d), 3)
    d.hi[1] = d.lo[1]
    assert lib.wost_create_field(C.byref(d), C.byref(h)) == INVALID
    assert b"box" in lib.wost_last_error()
    one = (C.c_float * 64)()
    for K in (0, 17):
        assert lib.wost_mixture_eval(2, K, one, one, one, one, 1, one) == INVALID
    assert lib.wost_solve(None, None, None, 0, 1, 1e-3, 16, 0, None, None, None, None) == INVALID
