"""GPU: the sparse plan layout (mam_desc.plan_layout = MAM_PLAN_SPARSE).

Every column step of Algorithm 1 sets theta' = pihat - d, with pihat (the
projection onto Delta_R(q_s), Prop. 3) zero off its active set and d one
vector per measure.  The sparse layout stores exactly that: the (row, value)
pairs of each column's pihat and each measure's last d.  The FP32 numbers it
reconstructs, fl(pihat + fl(0 - d)), are the dense layout's fl(pihat - d), so
with the same launch shape the two layouts give bit-identical plans,
thresholds, marginals, barycenters and diagnostics.  These tests compare the
two layouts bit for bit on the workloads and modes of the parity suite, the
sparse layout against the FP64 oracle directly, its checkpoints, its
capacity error and its rejections.
"""
import numpy as np
import pytest

from oracle.mam_oracle import MamOracle, prepare
from workloads import config1, config2, config4, config5, grid_points, tiny_problem
from workloads import Problem

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-5


@pytest.fixture(scope="module")
def Mam():
    from paper_2309_05315_gb300.build import build
    build()
    from paper_2309_05315_gb300 import Mam as _Mam
    return _Mam


def _slots(gpu, sparse_slots=0):
    return sparse_slots if sparse_slots else min(gpu.ld, 1024)


def thresholds(gpu, sparse_slots=None):
    """The stored thresholds lambda_s [T] of a mam_get_state blob: a 64-byte
    header, then the plan pieces (dense: theta [T][ld] FP32; sparse: counts
    [T] int32, pairs [T][slots] (int32, FP32), d_last [Mtot][ld] FP32), then
    the thresholds."""
    blob = gpu.get_state()
    T, ld, Mt = gpu.T, gpu.ld, gpu.n_measures
    if sparse_slots is None:
        off = 64 + 4 * T * ld
    else:
        off = 64 + 4 * T + 8 * T * sparse_slots + 4 * Mt * ld
    return np.frombuffer(blob, dtype=np.float32, count=T, offset=off).copy()


def pair_of_handles(Mam, prob=None, problems=None, sparse_slots=0, config=None, **kw):
    """A sparse handle and a dense handle of the same problem on the same
    one-CTA-per-column launch shape (the sparse handle's, or `config`)."""
    args = dict(problems=problems) if problems is not None else dict(problem=prob)
    sp = Mam(**args, plan_layout="sparse", sparse_slots=sparse_slots, **kw)
    de = Mam(**args, **kw)
    if config:
        sp.set_config(**config)
    cfg = sp.config()
    assert cfg["kind"] == 0 and cfg["stages"] == 1
    de.set_config(**cfg)
    return sp, de


def assert_same_iterate(sp, de, slots, full_theta=True, diag=False):
    if full_theta:
        np.testing.assert_array_equal(sp.theta(), de.theta())
    np.testing.assert_array_equal(sp.barycenter(), de.barycenter())
    np.testing.assert_array_equal(sp.marginals(), de.marginals())
    np.testing.assert_array_equal(thresholds(sp, slots), thresholds(de))
    if diag:
        assert sp.objectives() == de.objectives()


def run_bitwise(Mam, prob=None, problems=None, schedule=(1, 1, 3, 10, 12), sparse_slots=0,
                config=None, diag=False, **kw):
    sp, de = pair_of_handles(Mam, prob, problems, sparse_slots, config,
                             diag="every" if diag else "never", **kw)
    with sp, de:
        slots = _slots(sp, sparse_slots)
        assert_same_iterate(sp, de, slots)  # theta^0 (and primed thresholds)
        for n in schedule:
            sp.step(n)
            de.step(n)
            assert_same_iterate(sp, de, slots, diag=diag)


def test_blobs_balanced_bitwise(Mam):
    run_bitwise(Mam, config1())


def test_blobs_unbalanced_bitwise(Mam):
    run_bitwise(Mam, config1(), gamma=0.05)


def test_bundles_with_priming_bitwise(Mam):
    """Bundles of Remark 2, thresholds primed at creation.  R = 1600, so that
    both layouts prime on the same one-CTA-per-column launch shape (the
    dense layout's default for columns of up to 1024 rows is the warp kernel,
    whose reductions add in another order)."""
    prob = config4(grid=40, M=6)
    run_bitwise(Mam, prob, schedule=(1, 2, 5, 10, 20), n_bundles=3, seed=1234, gamma=0.02)


def test_capped_bitwise(Mam):
    run_bitwise(Mam, config1(), gamma=0.02, capped=True, eta=0.05)


def test_theta0_zero_bitwise(Mam):
    run_bitwise(Mam, config1(), theta0="zero")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_reduced_precision_costs_bitwise(Mam, dtype):
    run_bitwise(Mam, config4(grid=16, M=4), cost_dtype=dtype)


def test_shared_cost_layout_bitwise(Mam):
    run_bitwise(Mam, config4(grid=16, M=4), cost_layout="shared")


def test_batched_bitwise(Mam):
    probs = [tiny_problem(200 + i, M=2 + i % 3, K=6, rho=6.0) for i in range(5)]
    run_bitwise(Mam, problems=probs, schedule=(1, 4, 25))


def test_diagnostics_bitwise(Mam):
    run_bitwise(Mam, config1(), schedule=(1, 2, 7), diag=True)


@pytest.mark.parametrize("cfg", [
    dict(threads=32, vec=2),
    dict(threads=64, vec=1, ctas_per_sm=2),
    dict(threads=32, vec=8, ctas_per_sm=1),
])
def test_launch_shapes_bitwise(Mam, cfg):
    run_bitwise(Mam, config1(), schedule=(1, 5, 14), config=cfg)


@pytest.mark.parametrize("R_side,M", [(3, 3), (7, 4), (11, 3)])
def test_ragged_rows_bitwise(Mam, R_side, M):
    run_bitwise(Mam, tiny_problem(R_side, M=M, K=R_side, rho=5.0), schedule=(1, 3, 16))


def test_general_cost_matrix_bitwise(Mam):
    rng = np.random.default_rng(4)
    prob = tiny_problem(7, M=3, K=5, rho=4.0, density=0.7)
    prob.cost = [np.abs(rng.normal(size=(len(q), prob.R))) for q in prob.q]
    run_bitwise(Mam, prob, schedule=(1, 3, 20))


def test_nested_ellipses_R3600_bitwise(Mam):
    """R = 3600 over 10185 columns (several CTA tiles of float4 groups per
    column), 25 iterations through the captured graphs."""
    run_bitwise(Mam, config2(), schedule=(1, 4, 20))


def test_unbalanced_mixtures_R10000_bitwise(Mam):
    """The 100 x 100 unbalanced mixtures with 4 bundles (Remark 2), BF16
    costs, on 8 measures: the plans compared on sampled column ranges, the
    thresholds, marginals and barycenter in full."""
    sp, de = pair_of_handles(Mam, config5(M=8), cost_dtype="bf16", diag="never")
    with sp, de:
        slots = _slots(sp)
        T = sp.T
        ranges = [(0, 64), (T // 3, 64), (T - 64, 64)]
        for n in (1, 2, 10):
            sp.step(n)
            de.step(n)
            assert_same_iterate(sp, de, slots, full_theta=False)
            for c0, nc in ranges:
                np.testing.assert_array_equal(sp.theta_columns(c0, nc),
                                              de.theta_columns(c0, nc))


def test_sparse_matches_oracle(Mam):
    """The sparse layout against the FP64 oracle (the same tolerance as the
    dense parity tests), first 40 iterations."""
    prob = config1()
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho)
    Q = sum(float(q.sum()) for q in prep.q)
    Qa = sum(prep.a[m] * float(prep.q[m].sum()) for m in range(prep.M))
    with Mam(prob, diag="never", plan_layout="sparse") as gpu:
        for k in range(40):
            orc.step(diagnostics=False)
            gpu.step(1)
            th = gpu.theta().astype(np.float64).ravel()
            ref = np.concatenate([t.ravel() for t in orc.theta])
            e_th = np.abs(th - ref).sum() / Q
            e_p = np.abs(gpu.barycenter() - orc.barycenter()).sum() / Qa
            assert e_th <= ITER_TOL, (k, e_th)
            assert e_p <= ITER_TOL, (k, e_p)


def test_theta_columns_sparse(Mam):
    """mam_get_theta_range on the sparse layout: any column range, including
    columns never visited (theta^0) with bundles."""
    prob = tiny_problem(10, M=6, K=7, rho=15.0, masses=[0.5, 1, 1.5, 0.8, 1.2, 2.0])
    with Mam(prob, plan_layout="sparse", n_bundles=3, seed=7, gamma=0.02, diag="never") as g:
        g.step(3)
        full = g.theta()
        for c0, nc in [(0, 1), (5, 17), (g.T - 3, 3), (0, g.T)]:
            np.testing.assert_array_equal(g.theta_columns(c0, nc), full[c0:c0 + nc])


def test_backward_bitwise(Mam):
    """Reverse mode (mam_forward_record / mam_backward): the recomputed
    iterates come from the same kernels, so the gradients agree bit for bit."""
    prob = config4(grid=16, M=4)
    out = []
    for layout in ("sparse", "dense"):
        with Mam(prob, diag="never", plan_layout=layout) as g:
            if layout == "sparse":
                cfg = g.config()
            else:
                g.set_config(**cfg)
            g.forward_record(30, 7)
            p = g.barycenter()
            out.append((p,) + g.backward(2.0 * (p - prob.target)))
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)


def test_state_roundtrip_and_layout_check(Mam):
    from paper_2309_05315_gb300._capi import MamError
    prob = config1()
    with Mam(prob, diag="never", plan_layout="sparse") as a, \
         Mam(prob, diag="never", plan_layout="sparse") as b, \
         Mam(prob, diag="never") as d:
        a.step(37)
        b.step(20)
        blob = b.get_state()
        b.step(5)          # diverge, then come back
        b.set_state(blob)
        b.step(17)
        np.testing.assert_array_equal(a.theta(), b.theta())
        np.testing.assert_array_equal(a.barycenter(), b.barycenter())
        with pytest.raises(MamError) as e:
            b.set_state(d.get_state())  # a dense state
        assert e.value.status == 1
        with pytest.raises(MamError) as e:
            d.set_state(blob)
        assert e.value.status == 1


def test_capacity_error(Mam):
    """A column whose active set exceeds sparse_slots fails the step with
    MAM_ERR_CAPACITY, and the handle refuses further work (MAM_ERR_STATE)."""
    from paper_2309_05315_gb300._capi import MamError
    with Mam(config1(), diag="never", plan_layout="sparse", sparse_slots=2) as g:
        with pytest.raises(MamError) as e:
            g.step(3)
            g.barycenter()  # (steps are asynchronous: the next synchronizing call reports)
        assert e.value.status == 9
        with pytest.raises(MamError) as e:
            g.step(1)
        assert e.value.status == 6


def test_slots_at_the_largest_active_set(Mam):
    """sparse_slots equal to the largest active set of the run (read after
    every step of a run with ample slots) is enough: same iterate, no error."""
    prob = config1()
    need = 0
    with Mam(prob, diag="never", plan_layout="sparse", sparse_slots=256) as g:
        for _ in range(12):
            g.step(1)
            cnt = np.frombuffer(g.get_state(), dtype=np.int32, count=g.T, offset=64)
            need = max(need, int(cnt.max()))
        ref = g.theta()
    assert 2 < need < 256
    k = need + (need % 2)
    with Mam(prob, diag="never", plan_layout="sparse", sparse_slots=k) as g:
        g.step(12)
        np.testing.assert_array_equal(g.theta(), ref)


def test_sparse_rejections(Mam):
    from paper_2309_05315_gb300._capi import MamError
    prob = config1()
    for kw in (dict(sparse_slots=3), dict(sparse_slots=-2), dict(sparse_slots=264),
               dict(cost_layout="generated")):
        with pytest.raises(MamError) as e:
            Mam(prob, plan_layout="sparse", **kw)
        assert e.value.status == 1, kw
    with pytest.raises(MamError) as e:
        Mam(prob, sparse_slots=16)  # slots without the sparse layout
    assert e.value.status == 1
    # R = 12321 > 12288 rows: more than one CTA holds
    xi = grid_points(111)
    big = Problem("R12321", xi=xi, zeta=[xi[:4].copy()], q=[np.full(4, 0.25)],
                  alpha=np.array([1.0]), rho=10.0)
    with pytest.raises(MamError) as e:
        Mam(big, plan_layout="sparse")
    assert e.value.status == 1
    with Mam(prob, plan_layout="sparse", diag="never") as g:
        for cfg in (dict(kind=1, threads=32, vec=2, stages=2), dict(stages=2),
                    dict(kind=2, threads=128, vec=2, stages=1)):
            with pytest.raises(MamError) as e:
                g.set_config(**cfg)
            assert e.value.status == 1, cfg
        with pytest.raises(MamError) as e:
            g.update_support()
        assert e.value.status == 7
        g.step(2)  # still usable after the refused calls
        tuned = g.autotune(2)
        assert tuned["kind"] == 0 and tuned["stages"] == 1
