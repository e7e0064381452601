"""torch binding of libmam (argument marshalling only): ``solve`` and the
unrolled barycenter as a ``torch.autograd.Function``.

``MamFunction.apply(q, zeta, xi, S, alpha, rho, K, ckpt_every, theta0)``
returns p^K, the barycenter estimate after K iterations of Algorithm 1 from
theta^0 (balanced, deterministic, t = 1), as a float64 tensor on the device
of ``q``.  Its backward pass is libmam's reverse sweep (mam_forward_record /
mam_backward): gradients w.r.t. the weights q (unpruned order, zero for zero
weights), the support points zeta and the barycenter points xi.  The inputs
are copied to the host for mam_create, which copies them again (the C ABI
takes host arrays there and for the gradients); torch supplies memory and
the stream: the library's work is ordered on torch's current stream of the
device, and p is copied device to device.  ``ckpt_every = 0`` lets the
library keep every step's active sets when they fit (no recomputation in the
backward pass).
"""
from __future__ import annotations

import math
from types import SimpleNamespace

import numpy as np
import torch

from .mam import Mam


def _problem(q, zeta, xi, S, alpha, rho):
    q = q.detach().to("cpu", torch.float64).numpy()
    zeta = zeta.detach().to("cpu", torch.float64).numpy()
    xi = xi.detach().to("cpu", torch.float64).numpy()
    off = np.concatenate([[0], np.cumsum(S)]).astype(int)
    return SimpleNamespace(
        q=[q[off[m]:off[m + 1]] for m in range(len(S))],
        zeta=[zeta[off[m]:off[m + 1]] for m in range(len(S))],
        xi=xi, alpha=np.asarray(alpha, dtype=np.float64), rho=float(rho),
        gamma=math.inf, n_bundles=1, cost=None)


class MamFunction(torch.autograd.Function):
    """p^K(q, zeta, xi) with libmam's checkpointed reverse sweep."""

    @staticmethod
    def forward(ctx, q, zeta, xi, S, alpha, rho=100.0, K=200, ckpt_every=20,
                theta0="spread"):
        prob = _problem(q, zeta, xi, S, alpha, rho)
        dev = q.device if q.is_cuda else torch.device("cuda")
        # the library orders its work on torch's current stream of that device
        stream = torch.cuda.current_stream(dev)
        mam = Mam(prob, cost_dtype="f32", theta0=theta0, diag="never", stream=stream)
        mam.forward_record(int(K), int(ckpt_every))
        p = mam.barycenter_into(torch.empty(mam.R, dtype=torch.float64, device=dev))
        p = p.to(q.device)
        ctx.mam = mam
        ctx.shapes = (q.shape, zeta.shape, xi.shape)
        ctx.devices = (q.device, zeta.device, xi.device)
        ctx.dtypes = (q.dtype, zeta.dtype, xi.dtype)
        return p

    @staticmethod
    def backward(ctx, grad_p):
        want = tuple(n for n, need in zip(("q", "zeta", "xi"), ctx.needs_input_grad[:3])
                     if need)
        gq, gz, gx = ctx.mam.backward(grad_p.detach().to("cpu", torch.float64).numpy(),
                                      want=want)
        ctx.mam.close()
        out = []
        for g, shp, dev, dt in zip((gq, gz, gx), ctx.shapes, ctx.devices, ctx.dtypes):
            out.append(None if g is None else
                       torch.from_numpy(np.asarray(g)).reshape(shp).to(dev, dt))
        return (*out, None, None, None, None, None, None)


def unrolled_barycenter(q, zeta, xi, S, alpha, rho=100.0, K=200, ckpt_every=20,
                        theta0="spread"):
    """Functional form of ``MamFunction.apply``."""
    return MamFunction.apply(q, zeta, xi, list(S), list(alpha), rho, K, ckpt_every,
                             theta0)


def solve(q, zeta, xi, S, alpha, rho=100.0, gamma=math.inf, max_iters=20000, gap_tol=1e-4,
          check_every=10, cost_dtype="f32", n_bundles=1, seed=0, capped=False, eta=0.0):
    """MAM to a relative gap of gap_tol (mam_solve) on torch's current CUDA
    stream; returns (p, info).  p is a float64 tensor [R] on the device of q
    (copied device to device from the library), info has the iterations run,
    the last gap and the diagnostics of mam_objective.  ``capped``/``eta``
    select the full unbalanced extension (columns projected onto
    Delta_<=(q_s), cost alpha_m (d - eta))."""
    prob = _problem(q, zeta, xi, S, alpha, rho)
    prob.gamma = float(gamma)
    prob.n_bundles = int(n_bundles)
    stream = torch.cuda.current_stream(q.device if q.is_cuda else None)
    with Mam(prob, cost_dtype=cost_dtype, diag="never", seed=seed, stream=stream,
             capped=capped, eta=eta) as g:
        iters, gap = g.solve(int(max_iters), float(gap_tol), 0.0, int(check_every))
        info = dict(g.objective(), iterations=iters, gap=gap)
        dev = q.device if q.is_cuda else torch.device("cuda")
        p = g.barycenter_into(torch.empty(g.R, dtype=torch.float64, device=dev))
    return p.to(q.device), info
