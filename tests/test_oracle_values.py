"""Pins of the oracle's value functions against definitions it does not use.

* ``round_to_bf16`` / ``round_to_f16``: hand-derived IEEE 754 bit patterns
  (``tests/golden/cost_rounding.txt``): ties to even on both sides, overflow
  to infinity, subnormals, signed zero, negative values, and the FP64 ->
  FP32 -> 16-bit double rounding that a reduced-precision cost store
  performs.  Rounding ties away from zero, truncating, or skipping the FP32
  step each fail at least one line.
* ``dist_balanced``: a two-measure example worked out by hand (below), and
  the definition dist_L(pi) = min over theta in L of ||theta - pi||
  (section "Discrete unbalanced Wasserstein Barycenter") evaluated with a
  generic least-squares projection onto the constraint rows of eq. (L).
* The unbalanced objective F(pi-hat) = W-hat + gamma dist_L(pi-hat)
  (eq. UWB) that ``MamOracle.diagnostics`` reports: on real iterates,
  against W-hat and dist_L recomputed from pi-hat by the definitions; and at
  convergence, against the minimum of eq. (UWB) found by a general
  constrained solver (SLSQP) on a tiny instance.
"""
import math
import os

import numpy as np
import pytest
from scipy import optimize

from oracle.mam_oracle import (MamOracle, dist_balanced, prepare, round_to_bf16,
                               round_to_f16)
from tests.test_oracle_balanced import constraint_matrix, flat, unflat
from workloads import tiny_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "cost_rounding.txt")


def golden_cases():
    out = []
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fmt, x, bits = line.split()[:3]
            out.append((fmt, math.inf if x == "inf" else float.fromhex(x), int(bits, 16)))
    return out


def bf16_bits(v):
    """16-bit pattern of a float64 value that a bfloat16 represents exactly."""
    b = int(np.asarray(v, dtype=np.float32).reshape(1).view(np.uint32)[0])
    assert b & 0xFFFF == 0, hex(b)          # exactly representable in bfloat16
    assert float(np.float32(v)) == v or math.isnan(v)
    return b >> 16


def f16_bits(v):
    h = np.asarray(v, dtype=np.float16)
    assert float(h) == v or math.isnan(v)  # exactly representable in binary16
    return int(h.reshape(1).view(np.uint16)[0])


def test_golden_file_covers_both_formats():
    kinds = [c[0] for c in golden_cases()]
    assert kinds.count("bf16") >= 15 and kinds.count("f16") >= 15


@pytest.mark.parametrize("fmt,x,bits", golden_cases())
def test_rounding_matches_hand_derived_bits(fmt, x, bits):
    if fmt == "bf16":
        assert bf16_bits(round_to_bf16(np.array([x]))[0]) == bits
    else:
        assert f16_bits(round_to_f16(np.array([x]))[0]) == bits


def test_rounding_of_arrays_matches_elementwise():
    cases = golden_cases()
    for fmt, fn, conv in (("bf16", round_to_bf16, bf16_bits), ("f16", round_to_f16, f16_bits)):
        xs = np.array([c[1] for c in cases if c[0] == fmt])
        want = [c[2] for c in cases if c[0] == fmt]
        got = [conv(v) for v in fn(xs)]
        assert got == want


def test_dist_balanced_hand_worked():
    # Two measures, R = 3, S = (2, 3):  a = (1/2, 1/3) / (5/6) = (3/5, 2/5).
    # p^(1) = (0.6, 0.4, 0.0), p^(2) = (0.1, 0.4, 0.5)
    # p = 3/5 p^(1) + 2/5 p^(2) = (0.36 + 0.04, 0.24 + 0.16, 0.0 + 0.2)
    #   = (0.40, 0.40, 0.20)
    # p - p^(1) = (-0.2, 0, 0.2):  ||.||^2 = 0.08,  / S_1 = 0.04
    # p - p^(2) = ( 0.3, 0, -0.3): ||.||^2 = 0.18,  / S_2 = 0.06
    # dist^2 = 0.10.  (Equal weights give 0.1042, dropping 1/S_m gives 0.26,
    # weighting by a_m instead of 1/S_m gives 0.12.)
    pm = [np.array([0.6, 0.4, 0.0]), np.array([0.1, 0.4, 0.5])]
    assert dist_balanced(pm, [2, 3]) == pytest.approx(math.sqrt(0.10), rel=1e-14)


def generic_dist_to_L(pi, S, R):
    """min_{theta in L} ||theta - pi|| by least squares on the rows of eq. (L)."""
    x = flat(pi)
    B = constraint_matrix(S, R)
    y = B.T @ np.linalg.lstsq(B @ B.T, B @ x, rcond=None)[0]   # pi - Proj_L(pi)
    return float(np.linalg.norm(y))


@pytest.mark.parametrize("seed", range(6))
def test_dist_balanced_is_the_distance_to_L(seed):
    rng = np.random.default_rng(seed)
    M = int(rng.integers(2, 5))
    R = int(rng.integers(1, 6))
    S = [int(v) for v in rng.integers(1, 5, size=M)]
    pi = [rng.normal(size=(s, R)) for s in S]
    want = generic_dist_to_L(pi, S, R)
    got = dist_balanced([t.sum(axis=0) for t in pi], S)
    assert got == pytest.approx(want, rel=1e-12, abs=1e-14)


@pytest.mark.parametrize("gamma", [0.01, 0.2])
def test_reported_objective_matches_the_definitions(gamma):
    """W-hat = sum_m <c^(m), pi-hat^(m)>, dist_L(pi-hat) and F = W-hat +
    gamma dist_L (eq. UWB) recomputed from the pi-hat of a real step."""
    prob = tiny_problem(41, M=3, K=3, rho=6.0, masses=[0.7, 1.0, 1.6])
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho, gamma=gamma)
    orc.run(7)
    p, _, t = orc.average()
    d = [t * (p - orc.pm[m]) / prep.S[m] for m in range(prep.M)]
    out = orc.step(diagnostics=True)
    pihat = [orc.theta[m] + d[m][None, :] for m in range(prep.M)]   # theta' = pi-hat - d
    assert min(float(x.min()) for x in pihat) >= -1e-15
    w_hat = sum(float(np.sum(prep.c[m] * pihat[m])) for m in range(prep.M))
    dist = generic_dist_to_L(pihat, [int(s) for s in prep.S], prep.R)
    assert out["w_hat"] == pytest.approx(w_hat, rel=1e-12)
    assert out["dist_pihat"] == pytest.approx(dist, rel=1e-9, abs=1e-15)
    assert out["f_unbal"] == pytest.approx(w_hat + gamma * dist, rel=1e-12)
    assert out["t"] < 1.0     # the unbalanced branch of t^k ran


@pytest.mark.slow
def test_unbalanced_objective_at_convergence_is_the_uwb_minimum():
    """Unequal masses, gamma = 0.05: F(pi-hat^k) after a long MAM run equals
    the minimum of eq. (UWB) over pi^(m) in Pi^(m) found by SLSQP, whose
    objective takes dist_L from the least-squares projection."""
    gamma = 0.05
    prob = tiny_problem(43, M=2, K=2, rho=4.0, masses=[0.8, 1.3], density=1.0)
    prep = prepare(prob)
    S = [int(s) for s in prep.S]
    R = prep.R
    orc = MamOracle(prep, prob.rho, gamma=gamma)
    orc.run(20000)
    out = orc.step(diagnostics=True)

    c = flat(prep.c)
    B = constraint_matrix(S, R)
    BBt = B @ B.T

    def F(x):
        y = B.T @ np.linalg.lstsq(BBt, B @ x, rcond=None)[0]
        return float(c @ x) + gamma * float(np.linalg.norm(y))

    cons = []
    offs = np.cumsum([0] + [s * R for s in S])
    for m in range(len(S)):
        for s in range(S[m]):
            sel = np.zeros(len(c))
            sel[offs[m] + s * R: offs[m] + (s + 1) * R] = 1.0
            cons.append({"type": "eq", "fun": (lambda x, sel=sel, v=prep.q[m][s]: sel @ x - v)})
    x0 = flat([np.repeat((q / R)[:, None], R, axis=1) for q in prep.q])
    best = math.inf
    for start in (x0, flat([np.maximum(t + 1e-3, 0) for t in orc.theta])):
        res = optimize.minimize(F, start, method="SLSQP", bounds=[(0, None)] * len(c),
                                constraints=cons, options={"ftol": 1e-15, "maxiter": 2000})
        best = min(best, res.fun)
    assert out["f_unbal"] == pytest.approx(best, rel=2e-6)
    assert out["f_unbal"] >= best * (1 - 1e-9)   # pi-hat is feasible: never below the minimum
