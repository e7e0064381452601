"""Pins of the oracle's reverse sweep through unrolled MAM iterations.

The gradient of L = ||p^K - target||^2 w.r.t. the weights q, the measures'
support points zeta and the barycenter points xi is checked against central
finite differences of the forward oracle.  Away from changes of the active
sets the K-step map is piecewise affine in (q, c) and c is quadratic in the
coordinates, so central differences agree to rounding level.
"""
import copy

import numpy as np
import pytest

from oracle.mam_oracle import MamOracle, prepare, unrolled_loss, unrolled_loss_and_grad
from workloads import tiny_problem


def perturbed(prob, which, direction, h):
    p = copy.deepcopy(prob)
    if which == "q":
        p.q = [p.q[m] + h * direction[m] for m in range(p.M)]
    elif which == "zeta":
        p.zeta = [p.zeta[m] + h * direction[m] for m in range(p.M)]
    else:
        p.xi = p.xi + h * direction
    return p


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("which", ["q", "zeta", "xi"])
def test_gradient_matches_central_differences(seed, which):
    prob = tiny_problem(30 + seed, M=3, K=3, rho=4.0, density=0.8)
    K = 12
    rng = np.random.default_rng(seed)
    target = rng.uniform(size=prob.R)
    target /= target.sum()
    loss, gq, gz, gxi = unrolled_loss_and_grad(prob, K, prob.rho, target)
    if which == "q":
        d = [np.where(q > 0, rng.normal(size=q.shape) * q, 0.0) for q in prob.q]
        analytic = sum(float(np.dot(gq[m], d[m])) for m in range(prob.M))
    elif which == "zeta":
        d = [rng.normal(size=z.shape) for z in prob.zeta]
        analytic = sum(float(np.sum(gz[m] * d[m])) for m in range(prob.M))
    else:
        d = rng.normal(size=prob.xi.shape)
        analytic = float(np.sum(gxi * d))
    h = 1e-6
    fd = (unrolled_loss(perturbed(prob, which, d, h), K, prob.rho, target)
          - unrolled_loss(perturbed(prob, which, d, -h), K, prob.rho, target)) / (2 * h)
    assert abs(fd - analytic) <= 1e-6 * max(abs(fd), 1e-3 * loss), (fd, analytic)


def test_pruned_columns_get_zero_gradient():
    prob = tiny_problem(40, M=3, K=3, rho=4.0, density=0.6)
    target = np.full(prob.R, 1.0 / prob.R)
    _, gq, gz, _ = unrolled_loss_and_grad(prob, 5, prob.rho, target)
    for m in range(prob.M):
        z = prob.q[m] == 0
        assert z.any()
        assert np.all(gq[m][z] == 0) and np.all(gz[m][z] == 0)


def test_zero_iterations_gradient_is_closed_form():
    """K = 0: p^0 = sum_m a_m (Q_m / R) 1, so dL/dq_s = a_m * sum(g) / R."""
    prob = tiny_problem(41, M=2, K=3, rho=4.0)
    rng = np.random.default_rng(0)
    target = rng.uniform(size=prob.R)
    loss, gq, _, gxi = unrolled_loss_and_grad(prob, 0, prob.rho, target)
    S = np.array([(q > 0).sum() for q in prob.q])
    a = (1 / S) / (1 / S).sum()
    p0 = sum(a[m] * prob.q[m].sum() / prob.R for m in range(prob.M))
    g = 2 * (p0 - target)
    for m in range(prob.M):
        expect = np.where(prob.q[m] > 0, a[m] * g.sum() / prob.R, 0.0)
        np.testing.assert_allclose(gq[m], expect, rtol=1e-12)
    assert np.all(gxi == 0)


@pytest.mark.parametrize("which", ["q", "zeta", "xi"])
def test_dot_product_with_a_random_cotangent(which):
    """<J v, w> = <v, J^T w> for a random cotangent w of p^K (not only the
    loss residual) and a random direction v.  With target = p^K - w / 2 at
    the base point, the gradient of ||p^K - target||^2 is J^T w, and central
    differences of the same loss give <J v, w>."""
    prob = tiny_problem(50, M=3, K=3, rho=4.0, density=0.8)
    K = 10
    rng = np.random.default_rng(7)
    orc = MamOracle(prepare(prob, "f64"), prob.rho)
    orc.run(K)
    pK = orc.barycenter()
    w = rng.normal(size=prob.R)
    target = pK - 0.5 * w
    _, gq, gz, gxi = unrolled_loss_and_grad(prob, K, prob.rho, target)
    if which == "q":
        v = [np.where(q > 0, rng.normal(size=q.shape) * q, 0.0) for q in prob.q]
        adj = sum(float(np.dot(gq[m], v[m])) for m in range(prob.M))
    elif which == "zeta":
        v = [rng.normal(size=z.shape) for z in prob.zeta]
        adj = sum(float(np.sum(gz[m] * v[m])) for m in range(prob.M))
    else:
        v = rng.normal(size=prob.xi.shape)
        adj = float(np.sum(gxi * v))
    h = 1e-6
    tangent = (unrolled_loss(perturbed(prob, which, v, h), K, prob.rho, target)
               - unrolled_loss(perturbed(prob, which, v, -h), K, prob.rho, target)) / (2 * h)
    assert abs(tangent - adj) <= 1e-6 * max(abs(adj), 1e-6), (tangent, adj)
