"""Pins of the oracle's Algorithm 1 (MAM) against things it does not compute.

* the optimum of eq. (HugeLP) from the HiGHS LP solver;
* the exact Douglas-Rachford fixed point built from the LP's primal and dual
  solutions (Prop. 2 + Prop. 3 + complementary slackness);
* a generic eq. (DR) step written with least-squares Proj_L, a scalar
  minimisation for the prox of gamma*dist_L (eq. Unbalanced-prox) and
  brute-force simplex projections (the proof of the convergence theorem:
  Algorithm 1 is eq. (DR));
* closed forms: one measure, identical measures, the 1-D two-measure
  barycenter (Theorem 1 a), Prop. 1 (large gamma = balanced);
* invariants of DR: pi-hat feasible, mass of p, p >= 0, monotone and
  nonexpansive fixed-point map, LB <= optimum;
* Remark 2 draws: SplitMix64 reference outputs and bundle frequencies.
"""
import math
import os

import numpy as np
import pytest
from scipy import optimize

from oracle.lp import solve_barycenter_lp
from oracle.mam_oracle import (MamOracle, bundle_sequence, bundles, prepare,
                               proj_balanced, splitmix64)
from tests.test_oracle_balanced import constraint_matrix, flat, unflat
from tests.test_oracle_projection import brute_force_projection
from workloads import Problem, grid_points, problem_from_images, tiny_problem


def set_theta(orc, theta):
    orc.theta = [t.copy() for t in theta]
    orc.pm = [t.sum(axis=0) for t in orc.theta]


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_converges_to_lp_optimum(seed):
    prob = tiny_problem(seed, M=3, K=3, rho=5.0)
    prep = prepare(prob)
    lp = solve_barycenter_lp(prep)
    orc = MamOracle(prep, prob.rho)
    for k in range(20000):
        out = orc.step(diagnostics=(k % 500 == 499))
        if out.get("lower_bound") is not None:
            assert out["lower_bound"] <= lp["opt"] * (1 + 1e-12) + 1e-15
    out = orc.step(diagnostics=True)
    assert abs(out["w_hat"] - lp["opt"]) <= 1e-8 * lp["opt"]
    assert abs(out["lower_bound"] - lp["opt"]) <= 1e-8 * lp["opt"]
    assert out["dist_pihat"] < 1e-8
    # the barycenter's transport cost equals the optimum: p is a WB
    p = orc.barycenter()
    np.testing.assert_allclose(p.sum(), 1.0, rtol=1e-12)


@pytest.mark.parametrize("seed", [3, 4])
def test_exact_dr_fixed_point(seed):
    prob = tiny_problem(seed, M=3, K=3, rho=2.5)
    prep = prepare(prob)
    lp = solve_barycenter_lp(prep)
    rho = prob.rho
    # Sum of the coupling duals vanishes (dual constraint of the free p).
    np.testing.assert_allclose(sum(lp["v"]), 0, atol=1e-9)
    theta_star = [lp["pi"][m] - lp["v"][m][None, :] / rho for m in range(prep.M)]
    orc = MamOracle(prep, rho)
    set_theta(orc, theta_star)
    orc.step(diagnostics=False)
    scale = max(np.abs(flat(theta_star)).max(), 1e-300)
    np.testing.assert_allclose(flat(orc.theta), flat(theta_star), atol=1e-11 * scale)
    np.testing.assert_allclose(orc.barycenter(), lp["p"], atol=1e-11)


def generic_dr_step(prep, theta, rho, gamma):
    """One step of eq. (DR) with generic building blocks (no Prop. 2/3)."""
    S = [int(s) for s in prep.S]
    R = prep.R
    x = flat(theta)
    B = constraint_matrix(S, R)
    PL = x - B.T @ np.linalg.lstsq(B @ B.T, B @ x, rcond=None)[0]
    if math.isinf(gamma):
        pi = PL
    else:
        # prox of gamma*dist_L lies on the segment [theta, Proj_L theta]
        def obj(s):
            z = x + s * (PL - x)
            zp = z - B.T @ np.linalg.lstsq(B @ B.T, B @ z, rcond=None)[0]
            return gamma * np.linalg.norm(z - zp) + 0.5 * rho * np.sum((z - x) ** 2)
        res = optimize.minimize_scalar(obj, bounds=(0.0, 1.0), method="bounded",
                                       options={"xatol": 1e-14})
        pi = x + res.x * (PL - x)
    y = unflat(2 * pi - x, S, R)
    pihat = []
    for m in range(prep.M):
        cols = [brute_force_projection(y[m][s] - prep.c[m][s] / rho, prep.q[m][s])
                for s in range(S[m])]
        pihat.append(np.array(cols))
    return unflat(x + flat(pihat) - pi, S, R)


@pytest.mark.parametrize("gamma", [math.inf, 0.02, 0.2])
def test_algorithm1_is_dr(gamma):
    masses = None if math.isinf(gamma) else [1.0, 1.7, 0.6]
    prob = tiny_problem(21, M=3, K=2, rho=3.0, gamma=gamma, masses=masses)
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho, gamma=gamma)
    rng = np.random.default_rng(5)
    set_theta(orc, [rng.normal(scale=0.2, size=t.shape) for t in orc.theta])
    for _ in range(3):
        ref = generic_dr_step(prep, orc.theta, prob.rho, gamma)
        out = orc.step(diagnostics=False)
        tol = 1e-7 if not math.isinf(gamma) else 1e-11
        np.testing.assert_allclose(flat(orc.theta), flat(ref), atol=tol)
    if not math.isinf(gamma):
        assert out["t"] < 1.0        # the unbalanced branch was exercised


def test_single_measure_is_nearest_point_pushforward():
    rng = np.random.default_rng(9)
    xi = grid_points(4)
    zeta = rng.uniform(size=(7, 2))
    q = rng.uniform(0.1, 1, size=7)
    q /= q.sum()
    prob = Problem("m1", xi=xi, zeta=[zeta], q=[q], alpha=np.array([1.0]))
    prep = prepare(prob)
    d2 = ((zeta[:, None, :] - xi[None]) ** 2).sum(-1).min(axis=1)
    w_star = float(np.dot(q, d2))
    orc = MamOracle(prep, rho=20.0)
    orc.run(3000)
    out = orc.step()
    assert abs(out["w_hat"] - w_star) <= 1e-9
    assert abs(out["lower_bound"] - w_star) <= 1e-9


def test_identical_measures_have_zero_cost():
    rng = np.random.default_rng(3)
    img = rng.uniform(size=(4, 4))
    img[img < 0.3] = 0
    prob = problem_from_images("same", [img, img, img], rho=10.0)
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho)
    orc.run(4000)
    out = orc.step()
    assert out["w_hat"] < 1e-9
    np.testing.assert_allclose(orc.barycenter(), prob.q[0], atol=1e-7)


def w2_squared_1d(x1, q1, x2, q2):
    """Exact W_2^2 between 1-D discrete measures (quantile functions)."""
    o1, o2 = np.argsort(x1), np.argsort(x2)
    x1, q1, x2, q2 = x1[o1], q1[o1], x2[o2], q2[o2]
    c1, c2 = np.cumsum(q1), np.cumsum(q2)
    grid = np.unique(np.concatenate([[0.0], c1, c2]))
    grid = grid[grid <= 1.0 + 1e-15]
    tot = 0.0
    for a, b in zip(grid[:-1], grid[1:]):
        u = 0.5 * (a + b)
        i = min(np.searchsorted(c1, u), len(x1) - 1)
        j = min(np.searchsorted(c2, u), len(x2) - 1)
        tot += (b - a) * (x1[i] - x2[j]) ** 2
    return tot


def test_two_measures_on_a_line():
    """Theorem 1 a): on the half-step grid the fixed-support optimum equals
    the free-support one, alpha1*alpha2*W_2^2(nu1, nu2) (McCann midpoint)."""
    K = 6
    z = np.linspace(0, 1, K)[:, None]
    xi = np.linspace(0, 1, 2 * K - 1)[:, None]
    q1 = np.array([0.3, 0.0, 0.2, 0.0, 0.5, 0.0])
    q2 = np.array([0.0, 0.1, 0.0, 0.6, 0.0, 0.3])
    prob = Problem("line", xi=xi, zeta=[z, z], q=[q1, q2], alpha=np.array([0.5, 0.5]))
    prep = prepare(prob)
    lp = solve_barycenter_lp(prep)
    exact = 0.25 * w2_squared_1d(z[:, 0], q1, z[:, 0], q2)
    assert abs(lp["opt"] - exact) < 1e-12
    orc = MamOracle(prep, rho=50.0)
    orc.run(20000)
    out = orc.step()
    assert abs(out["w_hat"] - exact) <= 1e-8 * exact


def test_prop1_large_gamma_equals_balanced():
    prob = tiny_problem(6, M=3, K=3, rho=4.0)
    prep = prepare(prob)
    cnorm = math.sqrt(sum(float(np.sum(c ** 2)) for c in prep.c))
    a = MamOracle(prep, prob.rho)
    b = MamOracle(prep, prob.rho, gamma=10 * cnorm)
    for _ in range(300):
        a.step(diagnostics=False)
        out = b.step(diagnostics=False)
        assert out["t"] == 1.0
    for m in range(prep.M):
        assert np.array_equal(a.theta[m], b.theta[m])


@pytest.mark.parametrize("gamma", [math.inf, 0.05])
def test_dr_invariants(gamma):
    masses = None if math.isinf(gamma) else [0.7, 1.0, 1.6]
    prob = tiny_problem(8, M=3, K=4, rho=20.0, gamma=gamma, masses=masses)
    prep = prepare(prob)
    lp_opt = solve_barycenter_lp(prep)["opt"] if math.isinf(gamma) else None
    orc = MamOracle(prep, prob.rho, gamma=gamma)
    Qa = sum(prep.a[m] * prep.q[m].sum() for m in range(prep.M))
    prev_res = math.inf
    for k in range(300):
        p_before, _, t = orc.average()
        d = [t * (p_before - orc.pm[m]) / prep.S[m] for m in range(prep.M)]
        out = orc.step()
        for m in range(prep.M):
            pihat = orc.theta[m] + d[m][None, :]
            assert np.all(pihat >= -1e-15)
            np.testing.assert_allclose(pihat.sum(axis=1), prep.q[m], rtol=1e-11)
        p = orc.barycenter()
        assert abs(p.sum() - Qa) < 1e-12
        if math.isinf(gamma):
            assert np.all(p >= -1e-14)
            assert out["lower_bound"] <= lp_opt * (1 + 1e-12)
            assert out["fp_resid"] <= prev_res * (1 + 1e-9) + 1e-15
            prev_res = out["fp_resid"]
        # v = rho*d sums to zero over measures
        np.testing.assert_allclose(sum(d), 0.0, atol=1e-14)


@pytest.mark.parametrize("gamma", [math.inf, 0.05])
def test_nonexpansive(gamma):
    masses = None if math.isinf(gamma) else [0.7, 1.0, 1.6]
    prob = tiny_problem(12, M=3, K=3, rho=7.0, gamma=gamma, masses=masses)
    prep = prepare(prob)
    rng = np.random.default_rng(1)
    for _ in range(20):
        A = MamOracle(prep, prob.rho, gamma=gamma)
        B = MamOracle(prep, prob.rho, gamma=gamma)
        ta = [rng.normal(scale=0.1, size=t.shape) for t in A.theta]
        tb = [rng.normal(scale=0.1, size=t.shape) for t in A.theta]
        set_theta(A, ta)
        set_theta(B, tb)
        A.step(False)
        B.step(False)
        assert (np.linalg.norm(flat(A.theta) - flat(B.theta))
                <= np.linalg.norm(flat(ta) - flat(tb)) * (1 + 1e-12))


def test_splitmix64_reference_outputs():
    """Published SplitMix64 outputs (tests/golden/splitmix64.txt): the oracle's
    splitmix64(x) is the finaliser applied to the state x - increment."""
    g = 0x9E3779B97F4A7C15
    path = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 3
    for state, out in rows:
        assert splitmix64((int(state, 16) - g) % (1 << 64)) == int(out, 16)


def test_bundle_draw_frequencies():
    alpha = np.array([0.1, 0.2, 0.3, 0.15, 0.25])
    nb = 3
    B = bundles(5, nb)
    assert B == [[0], [1, 2], [3, 4]]
    seq = bundle_sequence(alpha, nb, seed=42, n_iters=60000)
    freq = np.bincount(seq, minlength=nb) / len(seq)
    beta = np.array([alpha[A].sum() for A in B])
    np.testing.assert_allclose(freq, beta / beta.sum(), atol=0.01)
    assert seq[:50] == bundle_sequence(alpha, nb, 42, 50)
    assert bundle_sequence(alpha, nb, 42, 10, start=7) == seq[7:17]


def test_randomized_mam_converges_and_freezes_other_measures():
    prob = tiny_problem(14, M=4, K=3, rho=5.0, n_bundles=2)
    prep = prepare(prob)
    lp = solve_barycenter_lp(prep)
    orc = MamOracle(prep, prob.rho, n_bundles=2, seed=3)
    for _ in range(200):
        before = [t.copy() for t in orc.theta]
        out = orc.step(diagnostics=False)
        Mk = out["index_set"]
        for m in range(prep.M):
            if m not in Mk:
                assert np.array_equal(orc.theta[m], before[m])
    orc.run(30000)
    out = orc.step()
    assert abs(out["w_hat"] - lp["opt"]) <= 1e-7 * lp["opt"]
