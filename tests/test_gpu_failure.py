"""Failure detection on the GPU without a fault.

* A device wait that runs out of its bound returns MAM_ERR_TIMEOUT instead
  of hanging: the self-test waits, through the column kernels' bounded
  mbarrier wait, on a phase that expects two arrivals and gets none.  The
  CUDA context stays usable afterwards.
* A problem whose first device allocation exceeds the GPU's memory fails
  with MAM_ERR_OOM, returns no handle and leaves the device memory as it
  was.
"""
import ctypes as C
import time

import numpy as np
import pytest

from workloads import config1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2309_05315_gb300.build import build
    build()
    from paper_2309_05315_gb300 import _capi
    return _capi.lib()


def test_bounded_wait_runs_out_and_context_survives(lib):
    from paper_2309_05315_gb300 import Mam
    t0 = time.perf_counter()
    st = lib.mam_selftest_wait_timeout(50000)  # 50 ms bound
    dt = time.perf_counter() - t0
    assert st == 5, lib.mam_last_error(None)   # MAM_ERR_TIMEOUT
    assert dt < 10.0
    assert b"ran out" in lib.mam_last_error(None)
    with Mam(config1(), diag="never") as g:       # the context is still usable
        g.step(5)
        assert np.all(np.isfinite(g.barycenter()))


def test_first_allocation_too_large_reports_oom(lib):
    import torch
    from paper_2309_05315_gb300 import _capi
    free0, total = torch.cuda.mem_get_info()
    R = 12288
    S = int(total // (4 * R)) + 1000        # theta alone exceeds the device memory
    q = np.full(S, 1.0 / S)
    zeta = np.zeros((S, 2))
    xi = np.zeros((R, 2))
    Sa = np.array([S], dtype=np.int32)
    alpha = np.array([1.0])
    d = _capi.MamDesc()
    d.M, d.R, d.dim = 1, R, 2
    d.S = Sa.ctypes.data_as(C.POINTER(C.c_int32))
    d.q = q.ctypes.data_as(C.POINTER(C.c_double))
    d.zeta = zeta.ctypes.data_as(C.POINTER(C.c_double))
    d.alpha = alpha.ctypes.data_as(C.POINTER(C.c_double))
    d.xi = xi.ctypes.data_as(C.POINTER(C.c_double))
    d.cost = None
    d.rho, d.gamma = 100.0, float("inf")
    h = C.c_void_p()
    st = lib.mam_create(C.byref(d), C.byref(h))
    assert st == 3, lib.mam_last_error(None)  # MAM_ERR_OOM
    assert not h.value
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert abs(free1 - free0) < (64 << 20)
