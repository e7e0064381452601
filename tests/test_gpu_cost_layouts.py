"""GPU parity of the shared and generated cost layouts against the FP64
oracle (Algorithm 1).

Shared (MAM_COST_SHARED): measures on one pixel grid have the same support
points before pruning, so one matrix C_rs = ||xi_r - zeta_s||^2 serves them
all and c^(m) = alpha_m C (eq. HugeLP); the kernels read the column of C that
a plan column's support point selects and apply alpha_m in the factor of c.
Generated (MAM_COST_GENERATED): no cost is stored; the kernels compute
||xi_r - zeta_s||^2 in FP32 from FP32 copies of the points (an FP32
difference of coordinates in [0, 1] and two fused multiply-adds: well within
the iterate tolerance, as the oracle's FP64 cost is the reference).
Checked: the kernel kinds on the blob workload, BF16/FP16 shared costs
against the oracle on the same rounding (C rounded, then scaled by alpha_m),
gamma finite, Remark 2 bundles, capped columns with eta, the fused
diagnostics, a batch of stroke problems sharing one matrix, long columns on
the free-support grid (generated), and the support step of Algorithm 2
(which rebuilds C, or the FP32 points, for the new support).
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
               n_bundles=1, seed=0, capped=False, eta=0.0, layout="shared", every=1):
    oracle_cost = "f64" if cost_dtype == "f32" else cost_dtype
    prep = prepare(prob, oracle_cost, eta=eta, round_before_alpha=cost_dtype != "f32")
    orc = MamOracle(prep, prob.rho, gamma=gamma, n_bundles=n_bundles, seed=seed,
                    capped=capped)
    Q = sum(float(q.sum()) for q in prep.q)
    Qa = sum(prep.a[m] * float(prep.q[m].sum()) for m in range(prep.M))
    with Mam(prob, cost_dtype=cost_dtype, diag="never", gamma=gamma, n_bundles=n_bundles,
             seed=seed, capped=capped, eta=eta, cost_layout=layout) as gpu:
        if config:
            gpu.set_config(**config)
        for k in range(iters):
            orc.step(diagnostics=False)
            gpu.step(1)
            if (k + 1) % every and k + 1 != iters:
                continue
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


def test_generated_cost_blobs(Mam):
    with Mam(config1(), diag="never", cost_layout="generated") as g:
        assert g.config()["kind"] == 2
    trajectory(Mam, config1(), 40, layout="generated")
    trajectory(Mam, config1(), 20, layout="generated",
               config=dict(kind=2, vec=8, threads=64, stages=1))


@pytest.mark.parametrize("layout", ["shared", "generated"])
@pytest.mark.parametrize("kw", [
    dict(gamma=0.02),
    dict(gamma=0.05, n_bundles=3, seed=4),
    dict(capped=True, eta=0.05),
])
def test_cost_layouts_unbalanced_variants(Mam, kw, layout):
    prob = tiny_problem(701, M=4, K=6, rho=8.0, masses=[0.6, 1.0, 1.3, 0.9])
    trajectory(Mam, prob, 30, layout=layout, **kw)


@pytest.mark.parametrize("layout", ["shared", "generated"])
@pytest.mark.parametrize("n_bundles", [1, 3])
def test_cost_layouts_diagnostics(Mam, layout, n_bundles):
    """W-hat and the lower bound, fused (deterministic) or from the
    lower-bound kernel (randomized index sets, every iteration diagnostic)."""
    prob = tiny_problem(702, M=3, K=6, rho=8.0, masses=[0.7, 1.0, 1.3])
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho, gamma=0.01, n_bundles=n_bundles, seed=3)
    orc.run(29)
    ref = orc.step(diagnostics=True)
    diag = "every" if n_bundles > 1 else "last"
    with Mam(prob, diag=diag, gamma=0.01, n_bundles=n_bundles, seed=3,
             cost_layout=layout) as gpu:
        gpu.step(30)
        o = gpu.objective()
    for k in ("w_hat", "lower_bound", "f_unbal"):
        assert abs(o[k] - ref[k]) <= 1e-4 * abs(ref[k]), k


def test_generated_cost_long_columns(Mam):
    """Two measures on the free-support grid of ten 60x60 images
    (R = 349281): no 4 GB cost buffer, c computed in the cluster kernel."""
    from workloads import Problem, free_support_grid
    xi = free_support_grid(10, 60)
    rng = np.random.default_rng(17)
    zeta = [rng.uniform(size=(6, 2)) for _ in range(2)]
    q = [v / v.sum() for v in (rng.uniform(0.5, 1.5, size=6) for _ in range(2))]
    prob = Problem("long", xi=xi, zeta=zeta, q=q, alpha=np.full(2, 0.5), rho=50.0)
    trajectory(Mam, prob, 12, layout="generated", every=4)


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


@pytest.mark.parametrize("layout", ["shared", "generated"])
def test_cost_layouts_support_step(Mam, layout):
    """Algorithm 2's support step rebuilds C (or the FP32 points) for the new
    support."""
    prob = tiny_problem(703, M=3, K=6, rho=8.0)
    orc = MamOracle(prepare(prob), prob.rho)
    Q = sum(float(q.sum()) for q in orc.prep.q)
    with Mam(prob, diag="never", cost_layout=layout) as gpu:
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
