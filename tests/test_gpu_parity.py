"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (fixed by how the method is used):
* iterates, first 50 iterations: ||theta_gpu - theta_ref||_1 / sum_m Q_m and
  ||p_gpu - p_ref||_1 / sum_m a_m Q_m below 1e-5;
* objective after the full run: |W_gpu - W_ref| / |W_ref| below 1e-4.
The DR map is nonexpansive, so FP32 rounding adds up across iterations
instead of growing geometrically; that is what makes an iterate tolerance
meaningful.
"""
import copy
import math

import numpy as np
import pytest

from oracle.mam_oracle import MamOracle, prepare, project_simplex
from workloads import Problem, config1, config2, grid_points, problem_from_images, tiny_problem

pytestmark = pytest.mark.gpu

ITER_TOL = 1e-5
OBJ_TOL = 1e-4


@pytest.fixture(scope="module")
def Mam():
    from paper_2309_05315_gb300.build import build
    build()
    from paper_2309_05315_gb300 import Mam as _Mam
    return _Mam


def masses(prep):
    Q = sum(float(q.sum()) for q in prep.q)
    Qa = sum(prep.a[m] * float(prep.q[m].sum()) for m in range(prep.M))
    return Q, Qa


def flat(th):
    return np.concatenate([t.ravel() for t in th])


def compare_trajectory(Mam, prob, iters, cost_dtype="f32", oracle_cost="f64",
                       n_bundles=1, seed=0, gamma=None, theta0="spread",
                       config=None, tol=ITER_TOL, capped=False, eta=0.0):
    g = math.inf if gamma is None else gamma
    prep = prepare(prob, oracle_cost, eta=eta)
    orc = MamOracle(prep, prob.rho, gamma=g, n_bundles=n_bundles, seed=seed,
                    theta0=theta0, capped=capped)
    Q, Qa = masses(prep)
    worst = 0.0
    with Mam(prob, cost_dtype=cost_dtype, diag="never", n_bundles=n_bundles,
             seed=seed, gamma=g, theta0=theta0, capped=capped, eta=eta) as gpu:
        if config:
            gpu.set_config(**config)
        assert gpu.T == sum(int(s) for s in prep.S)
        np.testing.assert_array_equal(gpu.pruned_sizes(), prep.S)
        for k in range(iters):
            orc.step(diagnostics=False)
            gpu.step(1)
            th = gpu.theta().astype(np.float64)
            e_th = np.abs(th.ravel() - flat(orc.theta)).sum() / Q
            e_p = np.abs(gpu.barycenter() - orc.barycenter()).sum() / Qa
            worst = max(worst, e_th, e_p)
            assert e_th <= tol, (k, e_th)
            assert e_p <= tol, (k, e_p)
    return worst


def test_config1_first_50_iterations(Mam):
    compare_trajectory(Mam, config1(), 50)


def test_config1_objective_after_500(Mam):
    prob = config1()
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho)
    orc.run(499)
    ref = orc.step(diagnostics=True)
    with Mam(prob, cost_dtype="f32", diag="last") as gpu:
        gpu.step(500)
        o = gpu.objective()
    assert o["iter"] == 500
    assert abs(o["w_hat"] - ref["w_hat"]) <= OBJ_TOL * abs(ref["w_hat"])
    assert abs(o["lower_bound"] - ref["lower_bound"]) <= OBJ_TOL * abs(ref["lower_bound"])
    assert abs(o["dist_pihat"] - ref["dist_pihat"]) <= 1e-3 * ref["dist_pihat"] + 1e-9
    assert abs(o["fp_resid"] - ref["fp_resid"]) <= 1e-2 * ref["fp_resid"] + 1e-9
    assert abs(o["dp_norm"] - ref["dp_norm"]) <= 1e-2 * ref["dp_norm"] + 1e-9
    assert o["t"] == 1.0


@pytest.mark.parametrize("R_side,M", [(3, 3), (5, 2), (7, 4), (11, 3)])
def test_ragged_rows(Mam, R_side, M):
    """R = 9, 25, 49, 121: columns not a multiple of the float4/8-element
    padding, tiny supports, several CTAs per measure."""
    prob = tiny_problem(100 + R_side, M=M, K=R_side, rho=5.0, density=0.6)
    compare_trajectory(Mam, prob, 30)


def test_ragged_R_not_grid(Mam):
    """R = 37 points and 1-point and 2-point measures (S_m after pruning)."""
    rng = np.random.default_rng(5)
    xi = rng.uniform(size=(37, 2))
    zeta = [rng.uniform(size=(4, 2)) for _ in range(3)]
    q = [np.array([0.0, 1.0, 0.0, 0.0]), np.array([0.5, 0.0, 0.5, 0.0]),
         np.array([0.25, 0.25, 0.25, 0.25])]
    prob = Problem("ragged", xi=xi, zeta=zeta, q=q, alpha=np.full(3, 1 / 3), rho=10.0)
    compare_trajectory(Mam, prob, 40)


def test_single_row_and_single_measure(Mam):
    xi = np.array([[0.3, 0.3]])
    prob = Problem("R1", xi=xi, zeta=[np.random.default_rng(0).uniform(size=(5, 2))],
                   q=[np.full(5, 0.2)], alpha=np.array([1.0]), rho=3.0)
    compare_trajectory(Mam, prob, 10)


def test_dimension_one_and_three(Mam):
    rng = np.random.default_rng(9)
    for dim in (1, 3):
        xi = rng.uniform(size=(40, dim))
        zeta = [rng.uniform(size=(9, dim)) for _ in range(2)]
        q = [rng.uniform(0.1, 1, size=9) for _ in range(2)]
        q = [v / v.sum() for v in q]
        prob = Problem(f"dim{dim}", xi=xi, zeta=zeta, q=q, alpha=np.array([0.4, 0.6]),
                       rho=20.0)
        compare_trajectory(Mam, prob, 25)


def test_general_cost_matrix(Mam):
    rng = np.random.default_rng(4)
    prob = tiny_problem(7, M=3, K=5, rho=4.0, density=0.7)
    prob.cost = [np.abs(rng.normal(size=(len(q), prob.R))) for q in prob.q]
    compare_trajectory(Mam, prob, 30)


def test_repeated_points_with_unequal_alpha(Mam):
    """Measures on one pixel grid with alpha = (0.25, 0.5, 0.25): creation
    builds each (point, alpha_m) class of cost columns once and copies it to
    the other columns of the class, so the first and third measures share
    cost columns while the second keeps its own."""
    prob = tiny_problem(41, M=3, K=10, rho=20.0, density=0.9, alpha=[0.25, 0.5, 0.25])
    compare_trajectory(Mam, prob, 25)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_tabulated_cost_equals_direct_formula(Mam, dtype):
    """Pixel-grid points take few values per coordinate, so creation builds
    the squared-Euclidean costs from per-coordinate tables of squares.  The
    same problem given as a general cost matrix (the same FP64 operations,
    d = z - x, d * d, the squares added in coordinate order, on the host) must
    give bit-identical iterates."""
    prob = tiny_problem(31, M=4, K=12, rho=20.0, density=0.8)
    alt = copy.copy(prob)
    xi = np.asarray(prob.xi, dtype=np.float64)
    alt.cost = [(z[:, None, 0] - xi[None, :, 0]) ** 2 + (z[:, None, 1] - xi[None, :, 1]) ** 2
                for z in (np.asarray(v, dtype=np.float64) for v in prob.zeta)]
    with Mam(prob, cost_dtype=dtype, diag="never") as a, \
         Mam(alt, cost_dtype=dtype, diag="never") as b:
        for n in (1, 4, 15):
            a.step(n)
            b.step(n)
            assert np.array_equal(a.theta(), b.theta())
            assert np.array_equal(a.barycenter(), b.barycenter())


def test_theta0_zero(Mam):
    compare_trajectory(Mam, tiny_problem(8, M=3, K=6, rho=10.0), 30, theta0="zero")


@pytest.mark.parametrize("dtype", ["bf16", "f16"])
def test_reduced_precision_costs(Mam, dtype):
    """The oracle rounds its costs the same way (FP64 -> FP32 -> dtype)."""
    compare_trajectory(Mam, config1(), 50, cost_dtype=dtype, oracle_cost=dtype)


@pytest.mark.parametrize("gamma", [0.003, 0.05])
def test_unbalanced(Mam, gamma):
    prob = tiny_problem(9, M=4, K=8, rho=20.0, masses=[0.6, 1.0, 1.5, 2.0])
    prob.gamma = gamma
    compare_trajectory(Mam, prob, 40, gamma=gamma)


def test_randomized_bundles(Mam):
    prob = tiny_problem(10, M=6, K=7, rho=15.0, masses=[0.5, 1, 1.5, 0.8, 1.2, 2.0])
    compare_trajectory(Mam, prob, 40, n_bundles=3, seed=1234, gamma=0.02)


def _state_parts(gpu):
    """theta [T][ld], the stored thresholds [T] and the iteration counter of a
    mam_get_state blob (a 64-byte header, then theta and the thresholds)."""
    blob = gpu.get_state()
    T, ld = gpu.T, gpu.ld
    it = int(np.frombuffer(blob, dtype=np.int64, count=1, offset=16)[0])
    th = np.frombuffer(blob, dtype=np.float32, count=T * ld, offset=64).reshape(T, ld)
    lam = np.frombuffer(blob, dtype=np.float32, count=T, offset=64 + 4 * T * ld)
    return th, lam, it


def test_thresholds_primed_for_bundles(Mam):
    """With randomized index sets (Remark 2) creation primes the stored
    thresholds: every kept column holds a finite threshold, while the iterate
    is exactly theta^0 (the plans, the Step 0 marginals and p of the same
    problem created without bundles, iteration 0).  With one index set the
    thresholds stay unknown (NaN)."""
    prob = tiny_problem(10, M=6, K=7, rho=15.0, masses=[0.5, 1, 1.5, 0.8, 1.2, 2.0])
    with Mam(prob, n_bundles=3, seed=1234, gamma=0.02, diag="never") as primed, \
         Mam(prob, n_bundles=1, gamma=0.02, diag="never") as plain:
        th_a, lam_a, it_a = _state_parts(primed)
        th_b, lam_b, it_b = _state_parts(plain)
        assert it_a == 0 and it_b == 0
        assert np.isfinite(lam_a).all()
        assert np.isnan(lam_b).all()
        np.testing.assert_array_equal(th_a, th_b)
        prep = prepare(prob)
        th0 = np.concatenate([np.repeat((q / prob.R).astype(np.float32)[:, None], prob.R, axis=1)
                              for q in prep.q])
        np.testing.assert_array_equal(th_a[:, :prob.R], th0)
        np.testing.assert_array_equal(primed.marginals(), plain.marginals())
        np.testing.assert_array_equal(primed.barycenter(), plain.barycenter())


@pytest.mark.parametrize("cfg", [
    dict(kind=0, threads=32, vec=2, stages=2),
    dict(kind=0, threads=64, vec=1, stages=3),
    dict(kind=0, threads=32, vec=8, stages=4, ctas_per_sm=1),
    dict(kind=0, threads=96, vec=1, stages=2, ctas_per_sm=2),
    dict(kind=1, threads=32, vec=2, stages=2, ctas_per_sm=4),
    dict(kind=1, threads=128, vec=2, stages=8, ctas_per_sm=1),
    dict(kind=1, threads=224, vec=4, stages=7, ctas_per_sm=1),
    dict(kind=1, threads=64, vec=8, stages=3, ctas_per_sm=2),
    dict(kind=1, threads=64, vec=2, stages=2, ctas_per_sm=8),
    dict(kind=1, threads=256, vec=2, stages=8, ctas_per_sm=1),
])
def test_kernel_configurations(Mam, cfg):
    compare_trajectory(Mam, config1(), 20, config=cfg)


@pytest.mark.parametrize("cfg", [
    dict(kind=1, threads=256, vec=7, stages=8, ctas_per_sm=2),
    dict(kind=1, threads=64, vec=8, stages=2, ctas_per_sm=4),
    dict(kind=0, threads=64, vec=4, stages=3),
])
def test_ring_slots_on_stroke_images(Mam, cfg):
    """R = 784 stroke images: as many warps as ring slots (every slot is
    re-claimed as soon as it is refilled) and BF16 costs."""
    from workloads import config3
    prob = config3(1, i0=3)[0]
    compare_trajectory(Mam, prob, 30, cost_dtype="bf16", oracle_cost="bf16", config=cfg)


@pytest.mark.parametrize("cfg", [
    None,  # the default: one CTA per column, 96 threads x 5 groups, one stage
    dict(kind=1, threads=384, vec=13, stages=12, ctas_per_sm=2),
    dict(kind=1, threads=128, vec=16, stages=4, ctas_per_sm=2),
    dict(kind=0, threads=128, vec=4, stages=2, ctas_per_sm=0),
])
def test_mixture_R1600_kernels(Mam, cfg):
    """The 40x40 Gaussian-mixture workload (R = 1600, 8 measures): the default
    CTA shape and the warp-per-column ring kernel at its two widest widths."""
    from workloads import config4
    compare_trajectory(Mam, config4(), 3, config=cfg)


def test_cold_start_bisection_depths(Mam):
    for kind, extra in ((1, {}), (0, dict(threads=64, vec=1, stages=2))):
        for depth in (0, 12, 30):
            compare_trajectory(Mam, config1(), 5, config=dict(kind=kind, bisect_depth=depth, **extra))


def test_config2_cta_kernel_iterates(Mam):
    """The one-CTA-per-column kernel on the R = 3600 workload."""
    compare_trajectory(Mam, config2(), 3, config=dict(kind=0, threads=160, vec=6, stages=2))


def test_diagnostics_match_oracle(Mam):
    prob = tiny_problem(11, M=3, K=6, rho=8.0, masses=[0.7, 1.0, 1.3])
    prob.gamma = 0.01
    prep = prepare(prob)
    orc = MamOracle(prep, prob.rho, gamma=0.01)
    orc.run(29)
    ref = orc.step(diagnostics=True)
    with Mam(prob, diag="last", gamma=0.01) as gpu:
        gpu.step(30)
        o = gpu.objective()
    for k in ("w_hat", "lower_bound", "f_unbal"):
        assert abs(o[k] - ref[k]) <= 1e-4 * abs(ref[k]), k
    assert abs(o["dist_pihat"] - ref["dist_pihat"]) <= 1e-3 * ref["dist_pihat"]
    assert abs(o["t"] - ref["t"]) <= 1e-4


@pytest.mark.parametrize("gamma, cfg", [
    (math.inf, None),                                   # ring kernel (R = 36)
    (math.inf, dict(kind=0, threads=32, vec=1, stages=1)),
    (0.02, None),
    (0.02, dict(kind=0, threads=64, vec=1, stages=2)),
])
def test_capped_columns(Mam, gamma, cfg):
    """Full unbalanced extension: unequal masses, cost alpha_m (d - eta) with
    eta between the grid's squared distances, projection onto
    Delta_<=(q_s)."""
    prob = tiny_problem(13, M=3, K=6, rho=8.0, masses=[0.6, 1.0, 1.4])
    worst = compare_trajectory(Mam, prob, 40, gamma=gamma, capped=True, eta=0.05,
                               config=cfg)
    assert worst >= 0.0


def test_capped_columns_mixture_cta_kernel(Mam):
    """R = 1600 mixture in the default one-CTA-per-column shape, capped."""
    from workloads import config4
    compare_trajectory(Mam, config4(), 3, capped=True, eta=0.01)


@pytest.mark.parametrize("n_bundles", [1, 3])
def test_capped_diagnostics_match_oracle(Mam, n_bundles):
    """W-hat and the lower bound with capped columns (each column's bound
    term is q_s min(0, min_r (c - rho d))), fused (deterministic) or
    recomputed by the lower-bound kernel (randomized index sets).  With
    randomized index sets every iteration is diagnostic, so that each
    column's W-hat term is the one of its last update, as in the oracle."""
    prob = tiny_problem(17, M=3, K=6, rho=8.0, masses=[0.8, 1.0, 1.2])
    eta = 0.05
    prep = prepare(prob, eta=eta)
    orc = MamOracle(prep, prob.rho, n_bundles=n_bundles, seed=5, capped=True)
    orc.run(29)
    ref = orc.step(diagnostics=True)
    diag = "every" if n_bundles > 1 else "last"
    with Mam(prob, diag=diag, n_bundles=n_bundles, seed=5, capped=True, eta=eta) as gpu:
        gpu.step(30)
        o = gpu.objective()
    scale = sum(float(np.abs(c).max()) * float(q.sum()) for c, q in zip(prep.c, prep.q))
    for k in ("w_hat", "lower_bound"):
        assert abs(o[k] - ref[k]) <= 1e-4 * scale, (k, o[k], ref[k])
    assert o["lower_bound"] <= o["w_hat"] + 1e-4 * scale


def support_error(orc, eta, xi_gpu):
    """Oracle support step; returns the mass-weighted mean distance between
    the two new supports (rows weighted by sum_m alpha_m sum_s pi-hat_rs: a
    row whose only mass is an entry at the threshold may differ between FP32
    and FP64, and carries no weight)."""
    plans = orc.next_pihat()
    den = sum(orc.prep.alpha[m] * plans[m].sum(axis=0) for m in range(orc.prep.M))
    xi_o = orc.update_support(eta)
    dist = np.linalg.norm(xi_gpu - xi_o, axis=1)
    return float(np.dot(den, dist) / den.sum())


@pytest.mark.parametrize("kw", [dict(), dict(gamma=0.02), dict(capped=True, eta=0.05)])
def test_support_step_matches_oracle(Mam, kw):
    """Algorithm 2: three rounds of 20 MAM iterations and a support step
    (Prop. 4), then 10 more iterations on the rebuilt costs."""
    gamma = kw.get("gamma", math.inf)
    capped, eta = kw.get("capped", False), kw.get("eta", 0.0)
    unequal = None if (math.isinf(gamma) and not capped) else [0.7, 1.0, 1.3]
    prob = tiny_problem(31, M=3, K=6, rho=8.0, masses=unequal)
    prep = prepare(prob, eta=eta)
    orc = MamOracle(prep, prob.rho, gamma=gamma, capped=capped)
    Q, _ = masses(prep)
    with Mam(prob, diag="never", gamma=gamma, capped=capped, eta=eta) as gpu:
        for _ in range(3):
            orc.run(20)
            gpu.step(20)
            xi_g = gpu.update_support()
            assert support_error(orc, eta, xi_g) <= 1e-5
        orc.run(10)
        gpu.step(10)
        e_th = np.abs(gpu.theta().astype(np.float64).ravel() - flat(orc.theta)).sum() / Q
        assert e_th <= 1e-4, e_th


def test_support_step_mixture_full_size(Mam):
    """R = 1600 mixture: 5 iterations, then the support step."""
    from workloads import config4
    prob = config4()
    orc = MamOracle(prepare(prob), prob.rho)
    with Mam(prob, diag="never") as gpu:
        orc.run(5)
        gpu.step(5)
        xi_g = gpu.update_support()
    assert support_error(orc, 0.0, xi_g) <= 1e-5


def test_free_support_rounds_match_oracle(Mam):
    """Algorithm 2 through mam_free_support: 3 rounds of 30 iterations and a
    support step, against the oracle's driver; then the barycenter."""
    from oracle.mam_oracle import free_support
    prob = tiny_problem(35, M=3, K=6, rho=8.0)
    orc = MamOracle(prepare(prob), prob.rho)
    for _ in range(3):  # the oracle's rounds, keeping the last round's row masses
        orc.run(30)
        plans = orc.next_pihat()
        weight = sum(orc.prep.alpha[m] * plans[m].sum(axis=0) for m in range(orc.prep.M))
        orc.update_support()
    ref = free_support(prob, outer=3, inner=30)   # the oracle's own driver agrees
    np.testing.assert_array_equal(ref.prep.xi, orc.prep.xi)
    with Mam(prob, diag="never") as gpu:
        xi0, it0 = gpu.free_support(0, 30)   # no round: the support as given
        np.testing.assert_array_equal(xi0, prob.xi)
        assert it0 == 0
        xi_g, iters = gpu.free_support(3, 30)
        p_g = gpu.barycenter()
    assert iters == 90
    d = np.linalg.norm(xi_g - orc.prep.xi, axis=1)
    assert float(np.dot(weight, d) / weight.sum()) <= 1e-5
    Qa = sum(orc.prep.a[m] * float(orc.prep.q[m].sum()) for m in range(orc.prep.M))
    assert np.abs(p_g - orc.barycenter()).sum() / Qa <= 1e-4


def test_support_step_rejections(Mam):
    from paper_2309_05315_gb300 import MamError
    prob = tiny_problem(33, M=3, K=4, rho=8.0)
    with Mam(prob, diag="never", n_bundles=3) as g:
        with pytest.raises(MamError) as e:
            g.update_support()
        assert e.value.status == 1
    gen = copy.deepcopy(prob)
    gen.cost = [np.ones((len(q), prob.R)) for q in prob.q]
    with Mam(gen, diag="never") as g:
        with pytest.raises(MamError) as e:
            g.update_support()
        assert e.value.status == 1
    with Mam(problems=[prob, prob], diag="never") as g:
        with pytest.raises(MamError) as e:
            g.update_support()
        assert e.value.status == 1


def test_bitwise_determinism_and_resume(Mam):
    prob = config1()
    with Mam(prob, diag="never") as a, Mam(prob, diag="never") as b:
        a.step(37)
        b.step(20)
        blob = b.get_state()
        b.step(5)          # diverge, then come back
        b.set_state(blob)
        b.step(17)
        assert np.array_equal(a.theta(), b.theta())
        assert np.array_equal(a.barycenter(), b.barycenter())


def test_graph_replay_equals_single_launches(Mam):
    prob = config1()
    with Mam(prob, diag="never") as a, Mam(prob, diag="never") as b:
        a.step(23)               # two captured 10-iteration graphs + 3 launches
        for _ in range(23):
            b.step(1)
        assert np.array_equal(a.theta(), b.theta())


def test_batched_matches_separate_problems(Mam):
    probs = [tiny_problem(200 + i, M=2 + i % 3, K=6, rho=6.0) for i in range(5)]
    with Mam(problems=probs, diag="last") as batch:
        batch.step(30)
        pb = batch.barycenter()
        objs = [batch.objective(i) for i in range(len(probs))]
        assert batch.objectives() == objs  # mam_objective_all agrees with mam_objective
    for i, prob in enumerate(probs):
        prep = prepare(prob)
        orc = MamOracle(prep, prob.rho)
        orc.run(29)
        ref = orc.step(diagnostics=True)
        Q, Qa = masses(prep)
        assert np.abs(pb[i] - orc.barycenter()).sum() / Qa <= ITER_TOL
        assert abs(objs[i]["w_hat"] - ref["w_hat"]) <= 1e-4 * ref["w_hat"]


@pytest.mark.parametrize("n, M, K", [(320, 3, 3), (160, 20, 8)])
def test_batched_averaging_block_shapes(Mam, n, M, K):
    """Batches shaped so that the averaging kernel runs with 1 measure slice
    (320 problems of 3 measures, R = 9) and with 4 slices (160 problems of 20
    measures, R = 64); sampled problems follow the oracle."""
    probs = [tiny_problem(5000 + i, M=M, K=K, rho=6.0) for i in range(n)]
    iters = 15
    with Mam(problems=probs, diag="never") as batch:
        batch.step(iters)
        pb = batch.barycenter()
    for i in (0, n // 2, n - 1):
        prep = prepare(probs[i])
        orc = MamOracle(prep, probs[i].rho)
        orc.run(iters)
        Q, Qa = masses(prep)
        assert np.abs(pb[i] - orc.barycenter()).sum() / Qa <= ITER_TOL


def test_solve_reaches_gap(Mam):
    prob = tiny_problem(12, M=3, K=4, rho=5.0)
    with Mam(prob) as gpu:
        it, gap = gpu.solve(20000, gap_tol=1e-4, check_every=50)
        o = gpu.objective()
    assert gap <= 1e-4 and it < 20000
    assert abs(o["w_hat"] - o["lower_bound"]) <= 1e-4 * abs(o["lower_bound"])


def test_config2_full_size_iterates(Mam):
    """The bench workload (60x60 nested ellipses, R=3600) in the bench's
    launch configuration: full iterates against the oracle for 5 steps."""
    prob = config2()
    compare_trajectory(Mam, prob, 5)


def test_config2_sampled_columns_after_warm_steps(Mam):
    """After 60 iterations, one more GPU step is checked column by column
    against an FP64 projection of the same input state."""
    prob = config2()
    prep = prepare(prob, "f32")
    with Mam(prob, diag="never") as gpu:
        gpu.step(60)
        th0 = gpu.theta().astype(np.float64)
        pm = gpu.marginals()
        p = gpu.barycenter()
        t = gpu.objective()["t_next"]
        gpu.step(1)
        th1 = gpu.theta().astype(np.float64)
    rng = np.random.default_rng(0)
    offs = np.concatenate([[0], np.cumsum(prep.S)])
    for col in rng.choice(int(offs[-1]), size=200, replace=False):
        m = int(np.searchsorted(offs, col, side="right") - 1)
        s = col - offs[m]
        d = t * (p - pm[m]) / prep.S[m]
        w = th0[col] + 2 * d - prep.c[m][s] / prob.rho
        x, _ = project_simplex(w, prep.q[m][s])
        ref = x[0] - d
        assert np.abs(th1[col] - ref).sum() <= 1e-5 * prep.q[m][s] + 1e-9, col


def test_maximum_R(Mam):
    """R = 12288 (the largest column a CTA holds) on a tiny problem."""
    K1, K2 = 96, 128
    i, j = np.meshgrid(np.arange(K1), np.arange(K2), indexing="ij")
    xi = np.stack([i.ravel() / (K1 - 1), j.ravel() / (K2 - 1)], 1)
    rng = np.random.default_rng(3)
    zeta = [rng.uniform(size=(6, 2)) for _ in range(2)]
    q = [np.full(6, 1 / 6), np.full(6, 1 / 6)]
    prob = Problem("maxR", xi=xi, zeta=zeta, q=q, alpha=np.array([0.5, 0.5]), rho=50.0)
    compare_trajectory(Mam, prob, 6)
