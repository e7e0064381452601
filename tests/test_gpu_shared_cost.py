"""GPU parity of the shared cost layout (MAM_COST_SHARED) against the FP64
oracle (Algorithm 1).

Measures on one pixel grid have the same support points before pruning, so
one matrix C_rs = ||xi_r - zeta_s||^2 serves them all and c^(m) = alpha_m C
(eq. HugeLP); the kernels read the column of C that a plan column's support
point selects and apply alpha_m in the factor of c.  Checked: the three
kernel kinds (warp per column, CTA per column, cluster per column) on the
blob workload, BF16 costs against the oracle on the same rounding (C rounded,
then scaled by alpha_m), gamma finite, Remark 2 bundles, capped columns with
eta, the fused diagnostics, a batch of stroke problems sharing one matrix,
and the support step of Algorithm 2 (which rebuilds C for the new support).
"""
import math

import numpy as np
import pytest

from oracle.mam_oracle import MamOracle, prepare
from workloads import config1, config3, tiny_problem

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-5


@pytest.fixture(scope="module")
def Mam():
    from paper_2309_05315_gb300.build import build
    build()
    from paper_2309_05315_gb300 import Mam as _Mam
    return _Mam


def flat(th):
    return np.concatenate([t.ravel() for t in th])


def trajectory(Mam, prob, iters, config=None, cost_dtype="f32", gamma=math.inf,
               n_bundles=1, seed=0, capped=False, eta=0.0):
    oracle_cost = "f64" if cost_dtype == "f32" else cost_dtype
    prep = prepare(prob, oracle_cost, eta=eta, round_before_alpha=cost_dtype != "f32")
    orc = MamOracle(prep, prob.rho, gamma=gamma, n_bundles=n_bundles, seed=seed,
                    capped=capped)
    Q = sum(float(q.sum()) for q in prep.q)
    Qa = sum(prep.a[m] * float(prep.q[m].sum()) for m in range(prep.M))
    with Mam(prob, cost_dtype=cost_dtype, diag="never", gamma=gamma, n_bundles=n_bundles,
             seed=seed, capped=capped, eta=eta, cost_layout="shared") as gpu:
        if config:
            gpu.set_config(**config)
        for k in range(iters):
            orc.step(diagnostics=False)
            gpu.step(1)
            e_th = np.abs(gpu.theta().astype(np.float64).ravel() - flat(orc.theta)).sum() / Q
            e_p = np.abs(gpu.barycenter() - orc.barycenter()).sum() / Qa
            assert e_th <= ITER_TOL, (k, e_th)
            assert e_p <= ITER_TOL, (k, e_p)


@pytest.mark.parametrize("config", [
    None,                                                   # warp per column (R = 256)
    dict(kind=0, threads=64, vec=1, stages=2),              # CTA per column
    dict(kind=2, vec=4, threads=64, stages=1),              # cluster per column
])
def test_shared_cost_kernel_kinds(Mam, config):
    trajectory(Mam, config1(), 40, config=config)


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_shared_cost_reduced_precision(Mam, dtype):
    trajectory(Mam, config1(), 40, cost_dtype=dtype)


@pytest.mark.parametrize("kw", [
    dict(gamma=0.02),
    dict(gamma=0.05, n_bundles=3, seed=4),
    dict(capped=True, eta=0.05),
])
def test_shared_cost_unbalanced_variants(Mam, kw):
    prob = tiny_problem(701, M=4, K=6, rho=8.0, masses=[0.6, 1.0, 1.3, 0.9])
    trajectory(Mam, prob, 30, **kw)


def test_shared_cost_diagnostics(Mam):
    prob = tiny_problem(702, M=3, K=6, rho=8.0, masses=[0.7, 1.0, 1.3])
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho, gamma=0.01)
    orc.run(29)
    ref = orc.step(diagnostics=True)
    with Mam(prob, diag="last", gamma=0.01, cost_layout="shared") as gpu:
        gpu.step(30)
        o = gpu.objective()
    for k in ("w_hat", "lower_bound", "f_unbal"):
        assert abs(o[k] - ref[k]) <= 1e-4 * abs(ref[k]), k


def test_shared_cost_stroke_batch(Mam):
    """16 stroke problems (R = 784) in one batch sharing one 784 x 784 BF16
    matrix; the first problem against the oracle for 30 iterations."""
    probs = config3(16)
    with Mam(problems=probs, cost_dtype="bf16", diag="never", cost_layout="shared") as b:
        b.step(30)
        pb = b.barycenter()
    for i in (0, 7, 15):
        prep = prepare(probs[i], "bf16", round_before_alpha=True)
        orc = MamOracle(prep, probs[i].rho)
        orc.run(30)
        Qa = sum(prep.a[m] * float(prep.q[m].sum()) for m in range(prep.M))
        assert np.abs(pb[i] - orc.barycenter()).sum() / Qa <= ITER_TOL, i


def test_shared_cost_support_step(Mam):
    """Algorithm 2's support step rebuilds C for the new support."""
    prob = tiny_problem(703, M=3, K=6, rho=8.0)
    orc = MamOracle(prepare(prob), prob.rho)
    Q = sum(float(q.sum()) for q in orc.prep.q)
    with Mam(prob, diag="never", cost_layout="shared") as gpu:
        for _ in range(2):
            orc.run(15)
            gpu.step(15)
            xi_g = gpu.update_support()
            plans = orc.next_pihat()
            den = sum(orc.prep.alpha[m] * plans[m].sum(axis=0) for m in range(orc.prep.M))
            xi_o = orc.update_support()
            # rows weighted by their mass (a row whose only mass sits at the
            # threshold may differ between FP32 and FP64 and carries none)
            dist = np.linalg.norm(xi_g - xi_o, axis=1)
            assert float(np.dot(den, dist) / den.sum()) <= 1e-5
        orc.run(10)
        gpu.step(10)
        e_th = np.abs(gpu.theta().astype(np.float64).ravel() - flat(orc.theta)).sum() / Q
        assert e_th <= 1e-4
