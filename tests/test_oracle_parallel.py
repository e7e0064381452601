"""The process-pool oracle follows MamOracle bit for bit.

ParallelMamOracle runs ``column_step`` of each measure in worker processes
and Step 1 in the coordinator with MamOracle's own code, so its iterates,
marginals, thresholds and diagnostics must equal the sequential oracle's
exactly, for the deterministic and randomized index sets, balanced and
unbalanced, plain and capped columns.
"""
import math

import numpy as np
import pytest

from oracle.mam_oracle import MamOracle, prepare
from oracle.parallel import ParallelMamOracle, measure_groups
from workloads import tiny_problem


def test_reduced_precision_costs_built_in_the_workers():
    prob = tiny_problem(62, M=4, K=4, rho=5.0)
    seq = MamOracle(prepare(prob, "bf16"), prob.rho)
    with ParallelMamOracle(prob, cost_dtype="bf16", workers=2) as par:
        for _ in range(5):
            a, b = seq.step(diagnostics=True), par.step(diagnostics=True)
            assert a["w_hat"] == b["w_hat"] and a["lower_bound"] == b["lower_bound"]
        assert np.array_equal(seq.barycenter(), par.barycenter())


def test_measure_groups_are_contiguous_and_balanced():
    S = [5, 1, 1, 9, 2, 2, 2, 8]
    for n in range(1, 10):
        g = measure_groups(S, n)
        assert [m for grp in g for m in grp] == list(range(len(S)))
        assert len(g) == min(n, len(S)) and all(grp for grp in g)
    g = measure_groups([10] * 8, 4)
    assert [len(x) for x in g] == [2, 2, 2, 2]


@pytest.mark.parametrize("kw", [
    dict(),
    dict(gamma=0.03, masses=[0.6, 1.0, 1.3, 1.6, 0.9]),
    dict(n_bundles=3, seed=11, masses=[0.6, 1.0, 1.3, 1.6, 0.9], gamma=0.05),
    dict(capped=True, eta=0.05, masses=[0.6, 1.0, 1.3, 1.6, 0.9]),
])
def test_parallel_oracle_is_bitwise_the_sequential_one(kw):
    kw = dict(kw)
    masses = kw.pop("masses", None)
    eta = kw.pop("eta", 0.0)
    prob = tiny_problem(61, M=5, K=5, rho=7.0, masses=masses)
    seq = MamOracle(prepare(prob, eta=eta), prob.rho, **kw)
    with ParallelMamOracle(prob, prob.rho, eta=eta, workers=3, **kw) as par:
        assert par.workers == 3
        for k in range(12):
            diag = k % 4 == 3
            a = seq.step(diagnostics=diag)
            b = par.step(diagnostics=diag)
            for key in ("t", "dist_theta", "w_hat", "dist_pihat", "f_unbal", "lower_bound",
                        "fp_resid", "dp_norm"):
                if key in a:
                    assert a[key] == b[key] or (math.isnan(a[key]) and math.isnan(b[key])), key
            assert a["index_set"] == b["index_set"]
            for m in range(prob.M):
                assert np.array_equal(seq.pm[m], par.pm[m])
                assert np.array_equal(seq.lam[m], par.lam[m])
        for x, y in zip(seq.theta, par.theta):
            assert np.array_equal(x, y)
        assert np.array_equal(seq.barycenter(), par.barycenter())
