"""GPU parity of the long-column kernel (kind 2: one column per thread-block
cluster, the CTAs exchanging their partial sums through distributed shared
memory) against the FP64 oracle (Algorithm 1).

* Forced on short columns in every cluster size and several CTA widths, so
  that slices are ragged, some CTAs hold no rows, and the cluster exchange
  carries every search pass; with gamma finite, Remark 2 bundles, capped
  columns, BF16 costs and the fused diagnostics.
* By default on the free-support grid of ten 60x60 images
  (R = 591^2 = 349281, Theorem 1), where one column needs 16 CTAs: a
  two-measure problem against the oracle's trajectory and its support step
  (Prop. 4), and the full nested-ellipse problem (3.56e9 plan entries) by
  sampled columns one step ahead, the row sums of the new plans and the
  barycenter.
"""
import math

import numpy as np
import pytest

from oracle.mam_oracle import MamOracle, prepare, project_simplex, sq_euclid_cost
from workloads import Problem, config1, config2_free_support, free_support_grid, tiny_problem

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


def trajectory(Mam, prob, iters, config=None, cost_dtype="f32", oracle_cost="f64",
               n_bundles=1, seed=0, gamma=math.inf, capped=False, eta=0.0, every=1):
    prep = prepare(prob, oracle_cost, eta=eta)
    orc = MamOracle(prep, prob.rho, gamma=gamma, n_bundles=n_bundles, seed=seed,
                    capped=capped)
    Q = sum(float(q.sum()) for q in prep.q)
    Qa = sum(prep.a[m] * float(prep.q[m].sum()) for m in range(prep.M))
    with Mam(prob, cost_dtype=cost_dtype, diag="never", n_bundles=n_bundles, seed=seed,
             gamma=gamma, capped=capped, eta=eta) as gpu:
        if config:
            gpu.set_config(**config)
        kind = gpu.config()["kind"]
        for k in range(iters):
            orc.step(diagnostics=False)
            gpu.step(1)
            if (k + 1) % every and k + 1 != iters:
                continue
            e_p = np.abs(gpu.barycenter() - orc.barycenter()).sum() / Qa
            e_th = np.abs(gpu.theta().astype(np.float64).ravel() - flat(orc.theta)).sum() / Q
            assert e_th <= ITER_TOL, (k, e_th)
            assert e_p <= ITER_TOL, (k, e_p)
    return kind


@pytest.mark.parametrize("cs, threads", [(2, 64), (4, 96), (8, 256), (16, 256), (16, 64)])
def test_cluster_kernel_on_short_columns(Mam, cs, threads):
    kind = trajectory(Mam, config1(), 25, config=dict(kind=2, vec=cs, threads=threads, stages=1))
    assert kind == 2


@pytest.mark.parametrize("kw", [
    dict(gamma=0.02, masses=[0.6, 1.0, 1.4]),
    dict(n_bundles=3, seed=21, gamma=0.05, masses=[0.6, 1.0, 1.4]),
    dict(capped=True, eta=0.05, masses=[0.6, 1.0, 1.4]),
    dict(cost_dtype="bf16", oracle_cost="bf16"),
])
def test_cluster_kernel_variants(Mam, kw):
    kw = dict(kw)
    masses = kw.pop("masses", None)
    prob = tiny_problem(601, M=3, K=11, rho=8.0, masses=masses)
    trajectory(Mam, prob, 30, config=dict(kind=2, vec=4, threads=64, stages=1), **kw)


def test_cluster_kernel_diagnostics(Mam):
    prob = tiny_problem(602, M=3, K=9, rho=8.0, masses=[0.7, 1.0, 1.3])
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho, gamma=0.01)
    orc.run(29)
    ref = orc.step(diagnostics=True)
    with Mam(prob, diag="last", gamma=0.01) as gpu:
        gpu.set_config(kind=2, vec=8, threads=64, stages=1)
        gpu.step(30)
        o = gpu.objective()
    for k in ("w_hat", "lower_bound", "f_unbal"):
        assert abs(o[k] - ref[k]) <= 1e-4 * abs(ref[k]), k
    assert abs(o["dist_pihat"] - ref["dist_pihat"]) <= 1e-3 * ref["dist_pihat"]


def long_problem(M=2, S=6, seed=7):
    """M measures of S random points each on the free-support grid of ten
    60x60 images (R = 349281)."""
    xi = free_support_grid(10, 60)
    rng = np.random.default_rng(seed)
    zeta = [rng.uniform(size=(S, 2)) for _ in range(M)]
    q = [rng.uniform(0.5, 1.5, size=S) for _ in range(M)]
    q = [v / v.sum() for v in q]
    return Problem("long", xi=xi, zeta=zeta, q=q, alpha=np.full(M, 1.0 / M), rho=50.0)


def test_long_columns_follow_the_oracle(Mam):
    prob = long_problem()
    with Mam(prob, diag="never") as g:
        cfg = g.config()
    assert cfg["kind"] == 2 and cfg["vec"] == 16
    trajectory(Mam, prob, 12, every=4)


def test_long_columns_support_step(Mam):
    """Prop. 4 on the long columns after 10 iterations."""
    prob = long_problem(seed=8)
    orc = MamOracle(prepare(prob), prob.rho)
    orc.run(10)
    plans = orc.next_pihat()
    den = sum(orc.prep.alpha[m] * plans[m].sum(axis=0) for m in range(orc.prep.M))
    xi_o = orc.update_support()
    with Mam(prob, diag="never") as gpu:
        gpu.step(10)
        xi_g = gpu.update_support()
    d = np.linalg.norm(xi_g - xi_o, axis=1)
    assert float(np.dot(den, d) / den.sum()) <= 1e-5


def test_free_support_grid_full_size_sampled_columns(Mam):
    """Ten nested-ellipse images on their free-support grid (R = 349281,
    10185 kept columns, 3.56e9 plan entries): after 20 iterations, sampled
    columns of one more step against FP64 projections of the same input
    state, the Step 3 row sums of one measure's new plans, and p (eq. pr)."""
    prob = config2_free_support()
    keep = [np.nonzero(q > 0)[0] for q in prob.q]
    S = np.array([len(k) for k in keep])
    offs = np.concatenate([[0], np.cumsum(S)])
    a = (1.0 / S) / (1.0 / S).sum()
    rng = np.random.default_rng(4)
    sample = [(int(m), int(rng.integers(0, S[m]))) for m in rng.integers(0, prob.M, 120)]
    with Mam(prob, diag="never") as gpu:
        assert gpu.config()["kind"] == 2
        gpu.step(20)
        pm0 = gpu.marginals()
        p0 = gpu.barycenter()
        before = {c: gpu.theta_columns(offs[c[0]] + c[1], 1)[0] for c in sample}
        gpu.step(1)
        after = {c: gpu.theta_columns(offs[c[0]] + c[1], 1)[0] for c in sample}
        pm1 = gpu.marginals()
        p1 = gpu.barycenter()
        m_chk = 3
        rows = np.zeros(prob.R)
        for c0 in range(0, S[m_chk], 64):
            n = min(64, S[m_chk] - c0)
            rows += gpu.theta_columns(offs[m_chk] + c0, n).astype(np.float64).sum(axis=0)
    for (m, s) in sample:
        qs = float(prob.q[m][keep[m][s]])
        z = np.asarray(prob.zeta[m])[keep[m][s]][None, :]
        c = sq_euclid_cost(prob.xi, z, float(prob.alpha[m])).astype(np.float32)[0]
        d = (p0 - pm0[m]) / S[m]
        w = before[(m, s)].astype(np.float64) + 2.0 * d - c.astype(np.float64) / prob.rho
        x, _ = project_simplex(w, qs)
        err = np.abs(after[(m, s)].astype(np.float64) - (x[0] - d)).sum()
        assert err <= ITER_TOL * qs + 1e-9, (m, s, err, qs)
    Qm = float(np.sum(prob.q[m_chk]))
    assert np.abs(rows - pm1[m_chk]).sum() <= ITER_TOL * Qm
    # eq. (pr), to the fixed-point resolution of the averages (each of the M
    # products a_m p^(m) is floored to 2^-58 Q_max: far below 1e-15 per row)
    p_ref = (a[:, None] * pm1).sum(axis=0)
    assert np.abs(p1 - p_ref).max() <= 1e-15 + 1e-12 * np.abs(p_ref).max()
