"""The allocation-free column update (mam_column_update_noalloc) agrees with
the regular entry points.

Some callers cannot call cudaMalloc (their device memory belongs to another
framework's pool, or their loop cannot afford cudaMalloc's synchronisation);
for them the library offers a column update whose scratch lives in a static
device array.  Here the same Algorithm 1 step is run twice in a row, once
through mam_create/mam_step and once through the allocation-free entry point
on caller-owned torch buffers, and plans and row sums are compared with the
tolerance of the other parity tests.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import config1

pytestmark = pytest.mark.gpu

TOL = 1e-5


def host_costs(prob, keep):
    """alpha_m ||xi_r - zeta_s||^2 in FP64, rounded once to FP32."""
    out = []
    for m in range(prob.M):
        z = np.asarray(prob.zeta[m])[keep[m]]
        diff = z[:, None, :] - prob.xi[None, :, :]
        out.append((prob.alpha[m] * np.einsum("srd,srd->sr", diff, diff)).astype(np.float32))
    return out


def test_noalloc_matches_regular_path_twice():
    torch = pytest.importorskip("torch")
    from paper_2309_05315_gb300 import Mam, _capi
    from paper_2309_05315_gb300.build import build
    build()
    L = _capi.lib()
    prob = config1()
    keep = [np.nonzero(q > 0)[0] for q in prob.q]
    S = [len(k) for k in keep]
    off = np.concatenate([[0], np.cumsum(S)])
    R = prob.R
    a = (1.0 / np.array(S)) / (1.0 / np.array(S)).sum()
    cost = torch.tensor(np.concatenate(host_costs(prob, keep)), device="cuda")
    q = torch.tensor(np.concatenate([prob.q[m][keep[m]] for m in range(prob.M)]),
                     dtype=torch.float32, device="cuda")
    with Mam(prob, cost_dtype="f32", diag="never") as ref:
        theta = torch.tensor(ref.theta(), device="cuda").contiguous()
        pm = ref.marginals()
        for call in range(2):
            p = (a[:, None] * pm).sum(axis=0)
            rows = torch.zeros((prob.M, R), dtype=torch.float64, device="cuda")
            for m in range(prob.M):
                d = torch.tensor((p - pm[m]) / S[m], dtype=torch.float32, device="cuda")
                th_m = theta[off[m]:off[m + 1]]
                st = L.mam_column_update_noalloc(
                    C.c_void_p(th_m.data_ptr()), C.c_void_p(cost[off[m]:off[m + 1]].data_ptr()),
                    C.c_void_p(q[off[m]:off[m + 1]].data_ptr()), C.c_void_p(d.data_ptr()),
                    R, R, S[m], float(prob.rho), float(prob.q[m].sum()),
                    C.c_void_p(rows[m].data_ptr()), None)
                _capi.check(st)
            torch.cuda.synchronize()
            ref.step(1)
            th_ref = ref.theta().astype(np.float64)
            pm_ref = ref.marginals()
            mass = sum(float(v.sum()) for v in prob.q)
            err_th = np.abs(theta.cpu().numpy().astype(np.float64) - th_ref).sum() / mass
            err_rows = np.abs(rows.cpu().numpy() - pm_ref).sum() / mass
            assert err_th <= TOL, (call, err_th)
            assert err_rows <= TOL, (call, err_rows)
            pm = rows.cpu().numpy()   # the allocation-free chain continues on its own


def test_noalloc_rejects_oversized_R():
    from paper_2309_05315_gb300 import _capi
    L = _capi.lib()
    dummy = C.c_void_p(1)
    st = L.mam_column_update_noalloc(dummy, dummy, dummy, dummy, 20000, 20000, 1, 1.0, 1.0,
                                     dummy, None)
    assert st == 1
    assert b"12288" in L.mam_last_error(None)
