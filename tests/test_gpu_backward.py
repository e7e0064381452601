"""GPU reverse mode (mam_forward_record / mam_backward) against the FP64
oracle's reverse sweep.

The loss is L = ||p^K - target||^2 with p^K the barycenter after K
deterministic, balanced iterations.  The oracle's adjoint is pinned on its
own (dot-product test and central differences); here the FP32 GPU adjoint is
compared with it by relative L2 error, tolerance 1e-3, for the gradients
w.r.t. the weights q, the support points zeta and the barycenter points xi.
"""
import numpy as np
import pytest

from oracle.mam_oracle import prepare, unrolled_loss_and_grad
from workloads import config4

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def Mam():
    from paper_2309_05315_gb300.build import build
    build()
    from paper_2309_05315_gb300 import Mam as _Mam
    return _Mam


def rel_l2(a, b):
    a, b = np.ravel(a), np.ravel(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def gpu_grads(Mam, prob, K, ckpt, theta0="spread", want=("q", "zeta", "xi")):
    with Mam(prob, diag="never", theta0=theta0) as g:
        g.forward_record(K, ckpt)
        p = g.barycenter()
        gq, gz, gx = g.backward(2.0 * (p - prob.target), want=want)
    return p, gq, gz, gx


def oracle_grads(prob, K, theta0="spread"):
    loss, gq, gz, gx = unrolled_loss_and_grad(prob, K, prob.rho, prob.target, theta0=theta0)
    return loss, np.concatenate(gq), np.concatenate(gz), gx


@pytest.mark.parametrize("theta0", ["spread", "zero"])
def test_backward_matches_oracle(Mam, theta0):
    prob = config4(grid=16, M=4)
    K = 30
    p, gq, gz, gx = gpu_grads(Mam, prob, K, 7, theta0)
    loss, oq, oz, ox = oracle_grads(prob, K, theta0)
    gpu_loss = float(np.sum((p - prob.target) ** 2))
    assert abs(gpu_loss - loss) <= 1e-4 * loss
    assert rel_l2(gq, oq) <= GRAD_TOL, rel_l2(gq, oq)
    assert rel_l2(gz, oz) <= GRAD_TOL, rel_l2(gz, oz)
    assert rel_l2(gx, ox) <= GRAD_TOL, rel_l2(gx, ox)
    # zero weights are pruned: their gradient is zero (one-sided kink)
    qcat = np.concatenate(prob.q)
    assert np.all(gq[qcat == 0] == 0)


def test_backward_ragged_rows_and_tail(Mam):
    """R = 23 x 23 = 529 (not a multiple of the 256-thread sweep), K = 12 with
    a last segment shorter than the checkpoint interval."""
    prob = config4(grid=23, M=3)
    K = 12
    p, gq, gz, gx = gpu_grads(Mam, prob, K, 5)
    _, oq, oz, ox = oracle_grads(prob, K)
    for a, b in ((gq, oq), (gz, oz), (gx, ox)):
        assert rel_l2(a, b) <= GRAD_TOL, rel_l2(a, b)


def test_checkpoint_interval_does_not_change_gradients(Mam):
    """The recomputed forward is bit-identical whatever the interval, and the
    reverse sweep adds its row sums in a fixed order, so the gradients are
    bit-identical too."""
    prob = config4(grid=16, M=3)
    K = 15
    ref = gpu_grads(Mam, prob, K, 1)
    for ck in (4, 15, 0):
        out = gpu_grads(Mam, prob, K, ck)
        for a, b in zip(ref, out):
            np.testing.assert_array_equal(a, b)


def test_all_masks_mode_equals_checkpointing(Mam):
    """ckpt_every = 0 keeps every step's active sets from the forward pass
    (no recomputation); the gradients are bit for bit those of the
    checkpointed sweep, and the state afterwards is the one after K steps."""
    prob = config4(grid=24, M=4)
    K = 30
    ref = gpu_grads(Mam, prob, K, 7)
    out = gpu_grads(Mam, prob, K, 0)
    for a, b in zip(ref, out):
        np.testing.assert_array_equal(a, b)
    with Mam(prob, diag="never") as g:
        g.forward_record(K, 0)
        g.backward(np.ones(g.R))
        th = g.theta()
    with Mam(prob, diag="never") as g:
        g.step(K)
        np.testing.assert_array_equal(g.theta(), th)


def test_state_restored_after_backward(Mam):
    prob = config4(grid=16, M=3)
    with Mam(prob, diag="never") as g:
        g.forward_record(10, 3)
        th, p = g.theta(), g.barycenter()
        g.backward(np.ones(g.R))
        np.testing.assert_array_equal(g.theta(), th)
        np.testing.assert_array_equal(g.barycenter(), p)
        g.step(5)
        th15 = g.theta()
    with Mam(prob, diag="never") as g:
        g.step(15)
        np.testing.assert_array_equal(g.theta(), th15)


def test_sum_of_barycenter_closed_form(Mam):
    """sum_r p^K_r = sum_m a_m Q_m for every K (balanced), so grad_p = 1
    gives dL/dq_s = a_m on every kept column and zero coordinate gradients."""
    prob = config4(grid=16, M=4)
    prep = prepare(prob, "f64")
    with Mam(prob, diag="never") as g:
        g.forward_record(20, 6)
        gq, gz, gx = g.backward(np.ones(g.R))
    expect = np.concatenate([np.where(np.asarray(prob.q[m]) > 0, prep.a[m], 0.0)
                             for m in range(prep.M)])
    # the reverse sweep works in FP32 per plan entry: FP32 rounding of a_m
    np.testing.assert_allclose(gq, expect, rtol=1e-6, atol=1e-12)
    assert np.abs(gz).max() <= 1e-7 and np.abs(gx).max() <= 1e-7


def test_full_size_short_horizon(Mam):
    """The 8 x 40 x 40 mixture workload (R = 1600, about 1.1e4 kept columns)
    with the launch shapes of the full run, over K = 4 iterations (two
    segments of 3 and 1)."""
    prob = config4()
    K = 4
    p, gq, gz, gx = gpu_grads(Mam, prob, K, 3)
    _, oq, oz, ox = oracle_grads(prob, K)
    for a, b in ((gq, oq), (gz, oz), (gx, ox)):
        assert rel_l2(a, b) <= GRAD_TOL, rel_l2(a, b)


@pytest.mark.parametrize("grid", [48, 66])
def test_large_rows(Mam, grid):
    """R = 2304 (ring forward kernel limit passed: CTA kernel) and R = 4356."""
    prob = config4(grid=grid, M=2)
    K = 3
    p, gq, gz, gx = gpu_grads(Mam, prob, K, 2)
    _, oq, oz, ox = oracle_grads(prob, K)
    for a, b in ((gq, oq), (gz, oz), (gx, ox)):
        assert rel_l2(a, b) <= GRAD_TOL, rel_l2(a, b)


def test_full_size_long_horizon_invariants(Mam):
    """K = 200, checkpoint every 20: translation invariance of the cost
    (sum_s dL/dzeta_s + sum_r dL/dxi_r = 0, to the FP32 rounding of the
    per-entry products) and finiteness."""
    prob = config4()
    p, gq, gz, gx = gpu_grads(Mam, prob, 200, 20)
    assert np.all(np.isfinite(gq)) and np.all(np.isfinite(gz)) and np.all(np.isfinite(gx))
    tot = gz.sum(axis=0) + gx.sum(axis=0)
    scale = np.abs(gz).sum() + np.abs(gx).sum()
    assert np.abs(tot).max() <= 1e-6 * scale


def test_backward_rejections(Mam):
    from paper_2309_05315_gb300 import MamError
    prob = config4(grid=16, M=3)
    with Mam(prob, diag="never") as g:
        with pytest.raises(MamError) as e:
            g.backward(np.ones(g.R))
        assert e.value.status == 6
        with pytest.raises(MamError) as e:
            g.forward_record(0, 1)
        assert e.value.status == 1
    with Mam(prob, diag="never", n_bundles=3) as g:
        with pytest.raises(MamError) as e:
            g.forward_record(5, 1)
        assert e.value.status == 1
    with Mam(prob, diag="never", gamma=0.01) as g:
        with pytest.raises(MamError) as e:
            g.forward_record(5, 1)
        assert e.value.status == 1
    with Mam(prob, diag="never", capped=True, eta=0.01) as g:
        with pytest.raises(MamError) as e:
            g.forward_record(5, 1)
        assert e.value.status == 1


def test_torch_autograd_function(Mam):
    torch = pytest.importorskip("torch")
    from paper_2309_05315_gb300.torch_api import unrolled_barycenter
    prob = config4(grid=16, M=3)
    K = 10
    S = [len(q) for q in prob.q]
    dev = "cuda"
    q = torch.tensor(np.concatenate(prob.q), device=dev, requires_grad=True)
    zeta = torch.tensor(np.concatenate(prob.zeta), device=dev, requires_grad=True)
    xi = torch.tensor(prob.xi, device=dev, requires_grad=True)
    p = unrolled_barycenter(q, zeta, xi, S, prob.alpha, prob.rho, K, 4)
    tgt = torch.tensor(prob.target, device=dev)
    loss = ((p - tgt) ** 2).sum()
    loss.backward()
    _, oq, oz, ox = oracle_grads(prob, K)
    assert rel_l2(q.grad.cpu().numpy(), oq) <= GRAD_TOL
    assert rel_l2(zeta.grad.cpu().numpy(), oz) <= GRAD_TOL
    assert rel_l2(xi.grad.cpu().numpy(), ox) <= GRAD_TOL


def test_torch_solve(Mam):
    """torch_api.solve: tensors in, the barycenter tensor out, on torch's stream."""
    torch = pytest.importorskip("torch")
    from paper_2309_05315_gb300.torch_api import solve
    prob = config4(grid=16, M=3)
    S = [len(q) for q in prob.q]
    q = torch.tensor(np.concatenate(prob.q), device="cuda")
    zeta = torch.tensor(np.concatenate(prob.zeta), device="cuda")
    xi = torch.tensor(prob.xi, device="cuda")
    p, info = solve(q, zeta, xi, S, prob.alpha, prob.rho, max_iters=20000, gap_tol=1e-4)
    assert p.is_cuda and p.dtype == torch.float64 and p.shape == (prob.R,)
    assert info["gap"] <= 1e-4
    with Mam(prob, diag="never") as g:
        it, gap = g.solve(20000, 1e-4, 0.0, 10)
        np.testing.assert_array_equal(p.cpu().numpy(), g.barycenter())
        assert it == info["iterations"]
