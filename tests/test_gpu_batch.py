"""GPU tests of the batched form and of the launch-shape autotuner.

* A problem solved inside a batch gives bit for bit the plans and barycenter
  of the same problem solved alone with the same kernel configuration: every
  column is projected from its own data, the row sums are 64-bit fixed-point
  integers (order-independent) and p = sum_m a_m p^(m) (eq. pr) is an integer
  sum over the problem's own measures.  Balanced problems (t^k = 1), so the
  FP32 distance sums that only feed t^k and the diagnostics play no part.
* The 256-problem stroke batch (28x28 images, M ~ U{4..16}, R = 784, BF16
  cost) at full size: problems checked bitwise against their unbatched runs,
  sampled problems against the FP64 oracle (Algorithm 1 on the same rounded
  costs) on the barycenter of each of the first 50 iterations and on the
  plans after them.
* mam_autotune returns a valid configuration, leaves the iteration state as
  it found it, and the tuned run still follows the oracle.
"""
import numpy as np
import pytest

from oracle.mam_oracle import MamOracle, prepare
from workloads import config3, tiny_problem

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-5


@pytest.fixture(scope="module")
def Mam():
    from paper_2309_05315_gb300.build import build
    build()
    from paper_2309_05315_gb300 import Mam as _Mam
    return _Mam


def column_ranges(sizes_per_problem):
    off = np.concatenate([[0], np.cumsum([sum(s) for s in sizes_per_problem])])
    return [(int(off[i]), int(off[i + 1])) for i in range(len(sizes_per_problem))]


def masses(prep):
    Q = sum(float(q.sum()) for q in prep.q)
    Qa = sum(prep.a[m] * float(prep.q[m].sum()) for m in range(prep.M))
    return Q, Qa


@pytest.mark.parametrize("cfg", [
    dict(kind=1, threads=128, vec=1, stages=8, ctas_per_sm=2, bisect_depth=4),
    dict(kind=0, threads=32, vec=1, stages=2, ctas_per_sm=0, bisect_depth=6),
])
def test_batched_bitwise_equals_unbatched(Mam, cfg):
    probs = [tiny_problem(300 + i, M=2 + i % 4, K=6, rho=6.0) for i in range(7)]
    iters = 30
    with Mam(problems=probs, diag="never") as batch:
        batch.set_config(**cfg)
        batch.step(iters)
        th_b = batch.theta()
        p_b = batch.barycenter()
        S_b = batch.pruned_sizes()
    sizes, k = [], 0
    for p in probs:
        sizes.append(S_b[k:k + p.M])
        k += p.M
    for i, (c0, c1) in enumerate(column_ranges(sizes)):
        with Mam(probs[i], diag="never") as one:
            one.set_config(**cfg)
            one.step(iters)
            assert np.array_equal(one.theta(), th_b[c0:c1]), i
            assert np.array_equal(one.barycenter(), p_b[i]), i


@pytest.fixture(scope="module")
def stroke_batch():
    return config3(256)


def test_config3_full_batch(Mam, stroke_batch):
    probs = stroke_batch
    iters = 50
    sampled = (0, 97, 255)
    bitwise = (5, 128)
    with Mam(problems=probs, cost_dtype="bf16", diag="never") as batch:
        cfg = batch.config()
        S_b = batch.pruned_sizes()
        p_traj = []
        for _ in range(iters):
            batch.step(1)
            p_traj.append(batch.barycenter())
        th_b = batch.theta()
    sizes, k = [], 0
    for p in probs:
        sizes.append(S_b[k:k + p.M])
        k += p.M
    ranges = column_ranges(sizes)
    for i in bitwise:
        with Mam(probs[i], cost_dtype="bf16", diag="never") as one:
            one.set_config(**cfg)
            one.step(iters)
            c0, c1 = ranges[i]
            assert np.array_equal(one.theta(), th_b[c0:c1]), i
            assert np.array_equal(one.barycenter(), p_traj[-1][i]), i
    for i in sampled:
        prep = prepare(probs[i], "bf16")
        orc = MamOracle(prep, probs[i].rho)
        Q, Qa = masses(prep)
        for k in range(iters):
            orc.step(diagnostics=False)
            e_p = np.abs(p_traj[k][i] - orc.barycenter()).sum() / Qa
            assert e_p <= ITER_TOL, (i, k, e_p)
        c0, c1 = ranges[i]
        ref = np.concatenate([t.ravel() for t in orc.theta])
        e_th = np.abs(th_b[c0:c1].astype(np.float64).ravel() - ref).sum() / Q
        assert e_th <= ITER_TOL, (i, e_th)
        # per column: no column off by more than the tolerance applied to its own
        # entries, |theta_s|_1 <= q_s + |d^(m)|_1 (d of the next step)
        p, _, t = orc.average()
        offs = np.concatenate([[0], np.cumsum(prep.S)])
        for m in range(prep.M):
            g = th_b[c0 + offs[m]:c0 + offs[m + 1]].astype(np.float64)
            err = np.abs(g - orc.theta[m]).sum(axis=1)
            scale = prep.q[m] + t * np.abs(p - orc.pm[m]).sum() / prep.S[m]
            assert np.all(err <= ITER_TOL * scale), (i, m, float((err / scale).max()))


def test_autotune_restores_state_and_keeps_parity(Mam):
    probs = [tiny_problem(400 + i, M=3 + i % 2, K=7, rho=6.0) for i in range(4)]
    with Mam(problems=probs, diag="never") as batch:
        batch.step(12)
        th0, p0, blob = batch.theta(), batch.barycenter(), batch.get_state()
        best = batch.autotune(3)
        assert batch.config() == best
        batch.set_config(**best)             # passes the library's own checks
        assert best["bisect_depth"] in (0, 2, 4, 6, 8, 12, 16, 24)
        assert np.array_equal(batch.theta(), th0)
        assert np.array_equal(batch.barycenter(), p0)
        assert batch.get_state() == blob
        batch.step(18)
        pb = batch.barycenter()
    for i, prob in enumerate(probs):
        prep = prepare(prob)
        orc = MamOracle(prep, prob.rho)
        orc.run(30)
        _, Qa = masses(prep)
        assert np.abs(pb[i] - orc.barycenter()).sum() / Qa <= ITER_TOL, i
