"""Pins of the oracle's full unbalanced extension (capped columns).

The extension (the paper's section "Algorithm's Extension: the Full
Unbalanced Setting") shifts the distance matrix to alpha_m (d - eta) and
replaces the projection onto Delta_R(q_s) in Step 2 with the one onto
Delta_<=(q_s) = {u >= 0 : sum u <= q_s}.  Pinned here against:
* brute-force enumeration of every support and the KKT system of the
  projection onto Delta_<=(tau), plus its closed-form special cases;
* the HiGHS optimum of the inequality-constrained LP (g = indicator of L);
* the balanced LP when eta exceeds every distance and the masses are equal
  (then every unit of mass is worth transporting);
* nonexpansiveness of the iteration map (it is a DR step, eq. DR).
"""
import itertools
import math

import numpy as np
import pytest

from oracle.lp import solve_barycenter_lp
from oracle.mam_oracle import MamOracle, prepare, project_capped_simplex, project_simplex
from workloads import tiny_problem


def brute_force_capped(w, tau):
    """Nearest feasible point among the candidates x_A = w_A - lam, x_rest = 0,
    for every support A and lam in {0, (sum_A w - tau)/|A|}; the projection
    has this form for its own support, so it is the nearest feasible one."""
    R = len(w)
    best, best_d = np.zeros(R), float(np.dot(w, w))
    for k in range(1, R + 1):
        for A in itertools.combinations(range(R), k):
            A = list(A)
            for lam in (0.0, (w[A].sum() - tau) / k):
                if lam < 0:
                    continue
                x = np.zeros(R)
                x[A] = w[A] - lam
                if np.all(x >= 0) and x.sum() <= tau * (1 + 1e-12) + 1e-15:
                    dd = float(np.dot(x - w, x - w))
                    if dd < best_d - 1e-15:
                        best, best_d = x, dd
    return best


@pytest.mark.parametrize("seed", range(30))
def test_capped_projection_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    R = int(rng.integers(1, 7))
    w = rng.normal(size=R) * rng.choice([0.1, 1.0, 3.0])
    tau = float(rng.choice([0.0, rng.uniform(0.01, 0.5), rng.uniform(0.5, 4.0)]))
    x, _ = project_capped_simplex(w[None, :], tau)
    np.testing.assert_allclose(x[0], brute_force_capped(w, tau), atol=1e-12)


@pytest.mark.parametrize("seed", range(20))
def test_capped_projection_kkt(seed):
    rng = np.random.default_rng(100 + seed)
    R = int(rng.integers(2, 40))
    W = rng.normal(size=(5, R))
    tau = rng.uniform(0.0, 3.0, size=5)
    X, lam = project_capped_simplex(W, tau)
    for i in range(5):
        x, l, t = X[i], lam[i], tau[i]
        assert np.all(x >= 0)
        assert x.sum() <= t * (1 + 1e-12) + 1e-15
        assert l >= 0
        assert abs(l * (t - x.sum())) <= 1e-12 * (1 + abs(l))  # complementary slackness
        np.testing.assert_allclose(x, np.maximum(W[i] - l, 0.0), atol=1e-12)


def test_capped_projection_special_cases():
    # all entries nonpositive: the projection is 0 (the clipped vector)
    x, lam = project_capped_simplex(np.array([[-1.0, -0.5, 0.0]]), 1.0)
    np.testing.assert_array_equal(x[0], 0.0)
    assert lam[0] == 0.0
    # clipped mass within tau: the clipped vector itself
    x, lam = project_capped_simplex(np.array([[0.2, -0.5, 0.3]]), 1.0)
    np.testing.assert_array_equal(x[0], [0.2, 0.0, 0.3])
    # clipped mass above tau: the simplex projection
    w = np.array([[2.0, 1.0, -1.0, 0.5]])
    x, lam = project_capped_simplex(w, 1.0)
    xs, ls = project_simplex(w, 1.0)
    np.testing.assert_array_equal(x, xs)
    np.testing.assert_array_equal(lam, ls)
    # tau = 0: {0}
    x, _ = project_capped_simplex(np.array([[3.0, 1.0]]), 0.0)
    np.testing.assert_array_equal(x[0], 0.0)


def run_capped(prob, eta, iters, gamma=math.inf):
    prep = prepare(prob, eta=eta)
    orc = MamOracle(prep, prob.rho, gamma=gamma, capped=True)
    out = None
    for k in range(iters):
        out = orc.step(diagnostics=(k % 500 == 499 or k == iters - 1))
    return prep, orc, out


@pytest.mark.parametrize("seed", [0, 1])
def test_capped_converges_to_lp_optimum(seed):
    """Unequal masses, eta between the grid's squared distances: some pairs
    are worth transporting and some are not."""
    prob = tiny_problem(seed, M=3, K=3, rho=5.0, masses=[0.5, 1.0, 1.5])
    eta = 0.3
    prep = prepare(prob, eta=eta)
    lp = solve_barycenter_lp(prep, capped=True)
    scale = sum(float(np.abs(c).max()) * float(q.sum()) for c, q in zip(prep.c, prep.q))
    orc = MamOracle(prep, prob.rho, capped=True)
    for k in range(20000):
        out = orc.step(diagnostics=(k % 500 == 499))
        if out.get("lower_bound") is not None:
            assert out["lower_bound"] <= lp["opt"] + 1e-12 * scale
    out = orc.step(diagnostics=True)
    assert abs(out["w_hat"] - lp["opt"]) <= 1e-8 * scale
    assert abs(out["lower_bound"] - lp["opt"]) <= 1e-8 * scale
    assert out["dist_pihat"] < 1e-8
    # capped columns: the transported mass is at most every measure's mass;
    # the LP may have several optimal barycenters, but here they all carry
    # the same mass
    p = orc.barycenter()
    assert p.sum() <= min(float(q.sum()) for q in prep.q) * (1 + 1e-9)
    assert abs(p.sum() - lp["p"].sum()) <= 1e-6


def test_large_eta_equal_masses_is_the_balanced_problem():
    """eta above every distance makes every cost negative; with equal masses
    the capped optimum then transports all mass, so it is the balanced
    optimum minus sum_m alpha_m eta Q_m."""
    prob = tiny_problem(5, M=3, K=3, rho=5.0)
    eta = 3.0  # squared distances on the unit square are at most 2
    prep_c = prepare(prob, eta=eta)
    prep_b = prepare(prob)
    lp_c = solve_barycenter_lp(prep_c, capped=True)
    lp_b = solve_barycenter_lp(prep_b)
    shift = sum(float(prep_b.alpha[m]) * eta * float(prep_b.q[m].sum()) for m in range(prep_b.M))
    assert abs(lp_c["opt"] - (lp_b["opt"] - shift)) <= 1e-9 * shift
    _, orc, out = run_capped(prob, eta, 20000)
    assert abs(out["w_hat"] - lp_c["opt"]) <= 1e-8 * shift
    np.testing.assert_allclose(orc.barycenter().sum(), 1.0, rtol=1e-9)


@pytest.mark.parametrize("gamma", [math.inf, 0.05])
def test_capped_iteration_is_nonexpansive(gamma):
    prob = tiny_problem(7, M=3, K=3, rho=4.0, masses=[0.7, 1.0, 1.3])
    prep = prepare(prob, eta=0.4)
    rng = np.random.default_rng(0)
    for _ in range(10):
        a = MamOracle(prep, prob.rho, gamma=gamma, capped=True)
        b = MamOracle(prep, prob.rho, gamma=gamma, capped=True)
        ta = [rng.normal(scale=0.3, size=t.shape) for t in a.theta]
        tb = [rng.normal(scale=0.3, size=t.shape) for t in b.theta]
        for orc, th in ((a, ta), (b, tb)):
            orc.theta = [t.copy() for t in th]
            orc.pm = [t.sum(axis=0) for t in orc.theta]
        before = math.sqrt(sum(float(np.sum((x - y) ** 2)) for x, y in zip(ta, tb)))
        a.step(diagnostics=False)
        b.step(diagnostics=False)
        after = math.sqrt(sum(float(np.sum((x - y) ** 2)) for x, y in zip(a.theta, b.theta)))
        assert after <= before * (1 + 1e-12)
