"""Pins of the oracle's free-support step (Prop. 4, Algorithm 2).

* Prop. 4's closed form against a numerical minimisation of
  Psi(xi) = sum_m alpha_m sum_{r,s} ||xi_r - zeta_s||^2 pi_{rs} / 2 and against
  the stationarity condition of Psi;
* rows without mass keep their point;
* translating every point moves the updated support by the same vector;
* Algorithm 2 with exact inner solves (HiGHS) never increases the barycenter
  objective, and the support step from MAM's converged (LP-optimal) plans
  lowers the cost of those plans.
"""
import copy

import numpy as np
import pytest
from scipy import optimize

from oracle.lp import solve_barycenter_lp
from oracle.mam_oracle import MamOracle, free_support, prepare, support_from_plans
from workloads import tiny_problem


def psi(xi_flat, R, dim, zeta, alpha, plans):
    xi = xi_flat.reshape(R, dim)
    tot = 0.0
    for m, pl in enumerate(plans):
        diff = xi[None, :, :] - zeta[m][:, None, :]          # (S, R, dim)
        tot += alpha[m] * 0.5 * float(np.sum(pl * np.sum(diff * diff, axis=2)))
    return tot


@pytest.mark.parametrize("seed", range(5))
def test_prop4_minimises_psi(seed):
    rng = np.random.default_rng(seed)
    R, dim, M = 5, int(rng.integers(1, 4)), 3
    S = rng.integers(2, 6, size=M)
    zeta = [rng.normal(size=(s, dim)) for s in S]
    alpha = rng.uniform(0.2, 1.0, size=M)
    plans = [rng.uniform(0, 1, size=(s, R)) * (rng.uniform(size=(s, R)) < 0.7) for s in S]
    xi0 = rng.normal(size=(R, dim))
    xi = support_from_plans(xi0, zeta, alpha, plans)
    res = optimize.minimize(psi, xi0.ravel(), args=(R, dim, zeta, alpha, plans),
                            method="BFGS", options={"gtol": 1e-12})
    den = sum(alpha[m] * plans[m].sum(axis=0) for m in range(M))
    for r in range(R):
        if den[r] > 0:
            np.testing.assert_allclose(xi[r], res.x.reshape(R, dim)[r], atol=1e-6)
    # stationarity: sum_m alpha_m sum_s (xi_r - zeta_s) pi_rs = 0
    grad = sum(alpha[m] * (plans[m].sum(axis=0)[:, None] * xi - plans[m].T @ zeta[m])
               for m in range(M))
    np.testing.assert_allclose(grad, 0.0, atol=1e-12)


def test_rows_without_mass_keep_their_point():
    xi0 = np.array([[0.0, 0.0], [1.0, 1.0], [2.0, 5.0]])
    zeta = [np.array([[3.0, 4.0], [5.0, 6.0]])]
    plans = [np.array([[0.5, 0.0, 0.0], [0.5, 0.0, 0.0]])]  # only row 0 carries mass
    xi = support_from_plans(xi0, zeta, np.array([1.0]), plans)
    np.testing.assert_allclose(xi[0], [4.0, 5.0])
    np.testing.assert_array_equal(xi[1:], xi0[1:])


def test_translation_moves_the_support_by_the_same_vector():
    prob = tiny_problem(21, M=3, K=4, rho=6.0)
    v = np.array([0.3, -1.7])
    moved = copy.deepcopy(prob)
    moved.xi = prob.xi + v
    moved.zeta = [np.asarray(z) + v for z in prob.zeta]
    a = MamOracle(prepare(prob), prob.rho)
    b = MamOracle(prepare(moved), moved.rho)
    a.run(40)
    b.run(40)
    np.testing.assert_allclose(b.update_support(), a.update_support() + v, atol=1e-12)


def with_support(prob, xi):
    out = copy.deepcopy(prob)
    out.xi = np.asarray(xi)
    return out


def test_algorithm2_exact_inner_solves_do_not_increase_the_objective():
    prob = tiny_problem(23, M=3, K=3, rho=5.0)
    cur = prob
    lp = solve_barycenter_lp(prepare(cur))
    for _ in range(4):
        prep = prepare(cur)
        xi = support_from_plans(prep.xi, prep.zeta, prep.alpha, lp["pi"])
        cur = with_support(cur, xi)
        lp_new = solve_barycenter_lp(prepare(cur))
        assert lp_new["opt"] <= lp["opt"] * (1 + 1e-9) + 1e-12
        lp = lp_new


def plan_cost(prep, plans):
    return sum(float(np.sum(prep.c[m] * plans[m])) for m in range(prep.M))


def test_support_step_from_converged_mam_plans():
    """MAM run to convergence: its plans are optimal for the old support (the
    LP optimum), the support step cannot raise the cost of those same plans
    (Prop. 4 minimises it over xi), and re-solving at the new support is no
    worse again.  (The LP's optimal plan need not be unique, so its own
    support step may land elsewhere.)"""
    prob = tiny_problem(25, M=3, K=3, rho=5.0)
    prep = prepare(prob)
    lp = solve_barycenter_lp(prep)
    orc = MamOracle(prep, prob.rho)
    orc.run(20000)
    plans = orc.next_pihat()
    assert abs(plan_cost(prep, plans) - lp["opt"]) <= 1e-8 * lp["opt"]
    xi_new = orc.update_support()
    prep_new = prepare(with_support(prob, xi_new))
    assert plan_cost(prep_new, plans) <= lp["opt"] * (1 + 1e-12)
    opt_new = solve_barycenter_lp(prep_new)["opt"]
    assert opt_new <= plan_cost(prep_new, plans) * (1 + 1e-9)
    # the oracle's costs now belong to the new support
    np.testing.assert_allclose(orc.prep.c[0], prep_new.c[0], rtol=1e-12, atol=1e-15)


def test_free_support_rounds_lower_the_lp_optimum():
    """Algorithm 2 with MAM run close to convergence in every round: the
    barycenter LP optimum at the final support is below the one at the
    initial grid (each round is a block coordinate step)."""
    prob = tiny_problem(27, M=3, K=3, rho=5.0)
    opt0 = solve_barycenter_lp(prepare(prob))["opt"]
    orc = free_support(prob, outer=3, inner=4000)
    opt3 = solve_barycenter_lp(prepare(with_support(prob, orc.prep.xi)))["opt"]
    assert opt3 <= opt0 * (1 + 1e-9)
    assert opt3 < opt0 * 0.999  # the grid was not already optimal
