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

from oracle.mam_oracle import project_simplex
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


def noalloc_call(L, theta, cost, q, d, R, ld, S, rho, mass_bound, rows):
    return L.mam_column_update_noalloc(
        C.c_void_p(theta.data_ptr()), C.c_void_p(cost.data_ptr()), C.c_void_p(q.data_ptr()),
        C.c_void_p(d.data_ptr()), R, ld, S, float(rho), float(mass_bound),
        C.c_void_p(rows.data_ptr()), None)


def test_noalloc_largest_R_matches_fp64_projection():
    """R = 12288, the largest column the static accumulator holds (48 KB of
    dynamic shared memory per CTA): plans and row sums of two calls in a row
    against FP64 projections of the same FP32 inputs."""
    torch = pytest.importorskip("torch")
    from paper_2309_05315_gb300 import _capi
    from paper_2309_05315_gb300.build import build
    build()
    L = _capi.lib()
    K1, K2 = 96, 128
    R, S, ld, rho = K1 * K2, 7, K1 * K2 + 8, 40.0
    i, j = np.meshgrid(np.arange(K1), np.arange(K2), indexing="ij")
    xi = np.stack([i.ravel() / (K1 - 1), j.ravel() / (K2 - 1)], 1)
    rng = np.random.default_rng(12)
    zeta = rng.uniform(size=(S, 2))
    qh = rng.uniform(0.5, 1.5, size=S).astype(np.float32)
    qh /= qh.sum()
    c = np.full((S, ld), np.inf, dtype=np.float32)
    c[:, :R] = ((zeta[:, None, :] - xi[None, :, :]) ** 2).sum(-1)
    th = np.zeros((S, ld), dtype=np.float32)
    th[:, :R] = rng.normal(scale=1e-4, size=(S, R))
    dh = rng.normal(scale=1e-5, size=R).astype(np.float32)
    theta = torch.tensor(th, device="cuda")
    cost = torch.tensor(c, device="cuda")
    q = torch.tensor(qh, device="cuda")
    d = torch.tensor(dh, device="cuda")
    rows = torch.zeros(R, dtype=torch.float64, device="cuda")
    ref = th[:, :R].astype(np.float64)
    for call in range(2):
        _capi.check(noalloc_call(L, theta, cost, q, d, R, ld, S, rho, 1.0, rows))
        torch.cuda.synchronize()
        w = ref + 2.0 * dh[None, :].astype(np.float64) - c[:, :R].astype(np.float64) / rho
        x, _ = project_simplex(w, qh.astype(np.float64))
        ref = x - dh[None, :].astype(np.float64)
        got = theta.cpu().numpy()[:, :R].astype(np.float64)
        for s in range(S):
            assert np.abs(got[s] - ref[s]).sum() <= TOL * qh[s], (call, s)
        np.testing.assert_array_equal(theta.cpu().numpy()[:, R:], 0.0)   # padding untouched
        err_rows = np.abs(rows.cpu().numpy() - ref.sum(axis=0)).sum() / qh.sum()
        assert err_rows <= TOL, (call, err_rows)


def test_noalloc_reports_device_failures_as_nan_rows():
    """An overflowing accumulator (mass_bound a sixth of the mass that lands
    on one row) and an empty active set (a weight below the FP32 resolution
    of w) both make every row sum NaN; a correct call afterwards is clean."""
    torch = pytest.importorskip("torch")
    from paper_2309_05315_gb300 import _capi
    L = _capi.lib()
    R, S = 64, 4
    c = np.full((S, R), 50.0, dtype=np.float32)
    c[:, 0] = 0.0                            # every column wants row 0
    cost = torch.tensor(c, device="cuda")
    d = torch.zeros(R, dtype=torch.float32, device="cuda")
    rows = torch.zeros(R, dtype=torch.float64, device="cuda")
    q = torch.full((S,), 0.25, dtype=torch.float32, device="cuda")
    theta = torch.zeros((S, R), dtype=torch.float32, device="cuda")
    _capi.check(noalloc_call(L, theta, cost, q, d, R, R, S, 1.0, 1.0 / 6.0, rows))
    torch.cuda.synchronize()
    assert torch.isnan(rows).all()
    theta.zero_()
    _capi.check(noalloc_call(L, theta, cost, q, d, R, R, S, 1.0, 1.0, rows))
    torch.cuda.synchronize()
    assert not torch.isnan(rows).any()
    assert float(rows[0]) == pytest.approx(1.0, abs=1e-6)
    theta.fill_(1.0)
    q_tiny = torch.tensor([1e-12, 0.25, 0.25, 0.25], dtype=torch.float32, device="cuda")
    _capi.check(noalloc_call(L, theta, cost, q_tiny, d, R, R, S, 1.0, 1.0, rows))
    torch.cuda.synchronize()
    assert torch.isnan(rows).all()


def test_noalloc_rejects_oversized_R():
    from paper_2309_05315_gb300 import _capi
    L = _capi.lib()
    dummy = C.c_void_p(1)
    st = L.mam_column_update_noalloc(dummy, dummy, dummy, dummy, 20000, 20000, 1, 1.0, 1.0,
                                     dummy, None)
    assert st == 1
    assert b"12288" in L.mam_last_error(None)
