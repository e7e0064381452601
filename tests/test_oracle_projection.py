"""Pins of the oracle's simplex projection (Prop. 3, Remark 1, eq. Delta).

The projection onto Delta_R(tau) is fixed by its KKT system; these tests
check the sort-based routine against brute-force enumeration of every
support, the KKT conditions, closed-form special cases and the scaling
identity of Remark 1.
"""
import itertools

import numpy as np
import pytest

from oracle.mam_oracle import project_simplex


def brute_force_projection(w, tau):
    """Enumerate every nonempty support A; the projection is the unique x
    with x_A = w_A - lam > 0, x_{not A} = 0, sum x = tau, w_{not A} <= lam."""
    R = len(w)
    if tau == 0:
        return np.zeros(R)
    hits = []
    for k in range(1, R + 1):
        for A in itertools.combinations(range(R), k):
            A = list(A)
            lam = (w[A].sum() - tau) / k
            x = np.zeros(R)
            x[A] = w[A] - lam
            rest = [r for r in range(R) if r not in A]
            if np.all(x[A] > 0) and np.all(w[rest] <= lam + 1e-15):
                hits.append(x)
    assert len(hits) >= 1
    for h in hits[1:]:
        np.testing.assert_allclose(h, hits[0], atol=1e-12)
    return hits[0]


@pytest.mark.parametrize("seed", range(40))
def test_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    R = int(rng.integers(1, 9))
    w = rng.normal(size=R) * rng.choice([1e-3, 1.0, 10.0])
    tau = float(rng.choice([0.0, 1e-3, 0.5, 1.0, 7.0]))
    x, _ = project_simplex(w, tau)
    np.testing.assert_allclose(x[0], brute_force_projection(w, tau), atol=1e-12)


@pytest.mark.parametrize("seed", range(10))
def test_kkt_conditions(seed):
    rng = np.random.default_rng(100 + seed)
    n, R = 50, 300
    W = rng.normal(size=(n, R)) * rng.uniform(1e-3, 10, size=(n, 1))
    tau = rng.uniform(0.01, 3.0, size=n)
    X, lam = project_simplex(W, tau)
    assert np.all(X >= 0)
    np.testing.assert_allclose(X.sum(axis=1), tau, rtol=1e-12)
    act = X > 0
    np.testing.assert_allclose((W - X)[act], np.broadcast_to(lam[:, None], W.shape)[act],
                               rtol=1e-10, atol=1e-12)
    assert np.all(W[~act] <= np.broadcast_to(lam[:, None], W.shape)[~act] + 1e-12)


def test_special_cases():
    # all-equal entries: x = tau / R
    x, _ = project_simplex(np.full(7, 3.3), 2.0)
    np.testing.assert_allclose(x[0], np.full(7, 2.0 / 7), rtol=1e-14)
    # tau = 0: {0} (Remark 1)
    x, lam = project_simplex(np.array([5.0, -1.0, 2.0]), 0.0)
    assert np.all(x == 0) and lam[0] == 0
    # dominant entry: e_r * tau
    w = np.array([0.0, 10.0, 0.1, -3.0])
    x, _ = project_simplex(w, 1.5)
    np.testing.assert_allclose(x[0], [0, 1.5, 0, 0], atol=1e-15)
    # w already in the simplex: unchanged
    w = np.array([0.2, 0.3, 0.5, 0.0])
    x, _ = project_simplex(w, 1.0)
    np.testing.assert_allclose(x[0], w, atol=1e-15)
    # a shift of w by a constant does not move the projection
    rng = np.random.default_rng(7)
    w = rng.normal(size=20)
    x1, l1 = project_simplex(w, 0.7)
    x2, l2 = project_simplex(w + 12.5, 0.7)
    np.testing.assert_allclose(x1, x2, atol=1e-12)
    np.testing.assert_allclose(l2 - l1, 12.5, rtol=1e-12)


@pytest.mark.parametrize("tau", [1e-4, 0.3, 1.0, 25.0])
def test_remark1_scaling(tau):
    """Proj_{Delta(tau)}(w) = tau * Proj_{Delta(1)}(w / tau) (Remark 1)."""
    rng = np.random.default_rng(int(tau * 1e4) % 1000)
    W = rng.normal(size=(30, 64))
    X, _ = project_simplex(W, tau)
    Y, _ = project_simplex(W / tau, 1.0)
    np.testing.assert_allclose(X, tau * Y, rtol=1e-10, atol=1e-14)


def test_is_nearest_point():
    """The projection beats every other feasible point in a random cloud."""
    rng = np.random.default_rng(11)
    w = rng.normal(size=6)
    x, _ = project_simplex(w, 1.0)
    d0 = np.sum((x[0] - w) ** 2)
    Y = rng.dirichlet(np.ones(6), size=20000)
    assert np.all(np.sum((Y - w) ** 2, axis=1) >= d0 - 1e-12)


def test_hand_worked_examples():
    """tests/golden/simplex_projection_examples.txt: projections worked by hand
    from the KKT conditions."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "simplex_projection_examples.txt")
    n = 0
    for ln in open(path):
        if not ln.strip() or ln.startswith("#"):
            continue
        tau, w, x = (part.split() for part in ln.split("|"))
        got, _ = project_simplex(np.array([[float(v) for v in w]]), np.array([float(tau[0])]))
        np.testing.assert_allclose(got[0], [float(v) for v in x], atol=1e-15)
        n += 1
    assert n == 5
