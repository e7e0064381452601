"""Pins of the oracle's projection onto the balanced subspace L (Prop. 2).

Proj_L is checked against the generic least-squares projection built from
the constraint rows of eq. (L) (consecutive row-marginal differences), so a
wrong averaging weight a_m, a missing 1/S_m or a sign error fails here.
"""
import numpy as np
import pytest

from oracle.mam_oracle import averaging_weights, dist_balanced, proj_balanced


def constraint_matrix(S, R):
    """Rows of eq. (L): sum_s pi^(m)_{rs} - sum_s pi^(m+1)_{rs} = 0."""
    M = len(S)
    n = sum(S) * R
    offs = np.cumsum([0] + [s * R for s in S])
    rows = []
    for m in range(M - 1):
        for r in range(R):
            row = np.zeros(n)
            for s in range(S[m]):
                row[offs[m] + s * R + r] += 1.0
            for s in range(S[m + 1]):
                row[offs[m + 1] + s * R + r] -= 1.0
            rows.append(row)
    return np.array(rows).reshape(-1, n)


def flat(th):
    return np.concatenate([t.ravel() for t in th])


def unflat(x, S, R):
    out, o = [], 0
    for s in S:
        out.append(x[o:o + s * R].reshape(s, R))
        o += s * R
    return out


@pytest.mark.parametrize("seed", range(8))
def test_prop2_equals_least_squares(seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(1, 5))
    R = int(rng.integers(1, 7))
    S = [int(s) for s in rng.integers(1, 6, size=M)]
    th = [rng.normal(size=(s, R)) for s in S]
    pi, p = proj_balanced(th)
    x = flat(th)
    if M > 1:
        B = constraint_matrix(S, R)
        corr = B.T @ np.linalg.lstsq(B @ B.T, B @ x, rcond=None)[0]
        y = x - corr
    else:
        y = x
    np.testing.assert_allclose(flat(pi), y, atol=1e-12)
    # all row marginals of the projection equal p
    for m in range(M):
        np.testing.assert_allclose(pi[m].sum(axis=0), p, atol=1e-12)


@pytest.mark.parametrize("seed", range(5))
def test_projection_properties(seed):
    rng = np.random.default_rng(50 + seed)
    M, R = 4, 5
    S = [3, 1, 4, 2]
    th = [rng.normal(size=(s, R)) for s in S]
    pi, _ = proj_balanced(th)
    pi2, _ = proj_balanced(pi)
    np.testing.assert_allclose(flat(pi2), flat(pi), atol=1e-13)   # idempotent
    # theta - Proj_L(theta) is orthogonal to L
    resid = flat(th) - flat(pi)
    for _ in range(5):
        y, _ = proj_balanced([rng.normal(size=(s, R)) for s in S])
        assert abs(np.dot(resid, flat(y))) < 1e-11
    # dist_L formula of the text after Algorithm 1
    pm = [t.sum(axis=0) for t in th]
    assert abs(dist_balanced(pm, S) - np.linalg.norm(resid)) < 1e-12


def test_averaging_weights():
    a = averaging_weights([2, 4, 4])
    np.testing.assert_allclose(a, [0.5, 0.25, 0.25])
    assert abs(a.sum() - 1) < 1e-15
