"""wost_solve_plain_static: the plain walk-on-stars solve for callers that
cannot allocate device memory while solving (for example when another
component owns the device memory pool, or in a loop that must not pay the
synchronisation of cudaFree).  It keeps its scratch in a fixed array inside
the library; these tests call it through the C ABI and compare it with
wost_solve on the same inputs and seeds, on two calls in a row (the second
call must not see the first one's sums)."""
import ctypes as C

import numpy as np
import pytest

import wost_inputs as wi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2410_18944_gb300 import build, _lib
    build.build()
    return _lib


def _static_solve(_lib, scene, pts_dev, nwalks, eps, maxsteps, seed):
    n = pts_dev.shape[0]
    mean = torch.empty(n, dtype=torch.float64, device=pts_dev.device)
    var = torch.empty(n, dtype=torch.float64, device=pts_dev.device)
    steps = C.c_int64()
    stream = torch.cuda.current_stream().cuda_stream
    _lib.check(_lib.load().wost_solve_plain_static(scene._h, C.c_void_p(pts_dev.data_ptr()), n, nwalks, eps,
                                                   maxsteps, seed, C.c_void_p(stream), C.c_void_p(mean.data_ptr()),
                                                   C.c_void_p(var.data_ptr()), C.byref(steps)))
    return mean.cpu().numpy(), var.cpu().numpy(), steps.value


def test_static_solve_matches_wost_solve_twice(lib):
    from paper_2410_18944_gb300 import api
    sc, pts = wi.config_star_guided(res=96, nseg=1024)
    S = api.Scene(sc)
    pd = torch.tensor(pts, dtype=torch.float64, device="cuda")
    for call, (nwalks, seed) in enumerate([(64, 5), (32, 11)]):
        m_s, v_s, steps_s = _static_solve(lib, S, pd, nwalks, 1e-3, 128, seed)
        m_r, v_r, st = api.solve(S, pd, nwalks, eps=1e-3, maxsteps=128, seed=seed)
        m_r, v_r = m_r.cpu().numpy(), v_r.cpu().numpy()
        # same Philox streams and arithmetic: equal up to the order of the
        # FP64 atomic additions
        assert steps_s == st["walk_steps"], call
        assert np.allclose(m_s, m_r, rtol=1e-9, atol=1e-12), call
        assert np.allclose(v_s, v_r, rtol=1e-6, atol=1e-12), call


def test_static_solve_rejects_too_many_points(lib):
    from paper_2410_18944_gb300 import api
    S = api.Scene(wi.ngon(16))
    n = 262144 + 1
    pd = torch.zeros((n, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(lib.WostError) as e:
        _static_solve(lib, S, pd, 1, 1e-3, 8, 1)
    assert "WOST_STATIC_MAX_POINTS" in str(e.value)
