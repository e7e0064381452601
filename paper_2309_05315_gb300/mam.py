"""Python binding of libmam with the C ABI's names (argument marshalling only).

``Mam`` wraps one problem handle (or a batch of problems).  Every method is a
direct call of the C function of the same name in include/mam.h; numpy arrays
are passed as host pointers and, where the ABI accepts device pointers, torch
CUDA tensors as device pointers.  Nothing here computes any part of the
method.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Optional, Sequence

import numpy as np

from . import _capi
from ._capi import MamDesc, MamKernelConfig, MamObjective, MamShard, check


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


class _DescKeep:
    """Owns the contiguous arrays a mam_desc points into."""

    def __init__(self, problem, cost_dtype, theta0_mode, diag_mode, n_bundles,
                 seed, rho, gamma, stream, capped=False, eta=0.0, cost_layout="per_column",
                 plan_layout="dense", sparse_slots=0):
        M = len(problem.q)
        xi = np.ascontiguousarray(problem.xi, dtype=np.float64)
        if xi.ndim == 1:
            xi = xi[:, None]
        R, dim = xi.shape
        self.S = np.ascontiguousarray([len(q) for q in problem.q], dtype=np.int32)
        self.q = np.ascontiguousarray(np.concatenate(problem.q), dtype=np.float64)
        self.alpha = np.ascontiguousarray(problem.alpha, dtype=np.float64)
        self.xi = xi
        self.zeta = None
        if problem.zeta is not None:
            z = [np.asarray(v, dtype=np.float64).reshape(len(problem.q[m]), dim)
                 for m, v in enumerate(problem.zeta)]
            self.zeta = np.ascontiguousarray(np.concatenate(z))
        self.cost = None
        if getattr(problem, "cost", None) is not None:
            self.cost = np.ascontiguousarray(np.concatenate(
                [np.asarray(c, dtype=np.float64).reshape(len(problem.q[m]), R)
                 for m, c in enumerate(problem.cost)]))
        d = MamDesc()
        d.M, d.R, d.dim = M, R, dim
        d.S = self.S.ctypes.data_as(C.POINTER(C.c_int32))
        d.zeta = _dptr(self.zeta) if self.zeta is not None else None
        d.q = _dptr(self.q)
        d.alpha = _dptr(self.alpha)
        d.xi = _dptr(self.xi)
        d.cost = _dptr(self.cost) if self.cost is not None else None
        d.rho = float(problem.rho if rho is None else rho)
        g = getattr(problem, "gamma", math.inf) if gamma is None else gamma
        d.gamma = float(g)
        nb = getattr(problem, "n_bundles", 1) if n_bundles is None else n_bundles
        d.n_bundles = int(nb)
        d.seed = int(seed)
        d.cost_dtype = _capi.COST_DTYPES[cost_dtype]
        d.theta0_mode = {"spread": 0, "zero": 1}[theta0_mode]
        d.diag_mode = _capi.DIAG_MODES[diag_mode]
        d.stream = stream
        d.eta = float(eta)
        d.capped = 1 if capped else 0
        d.cost_layout = _capi.COST_LAYOUTS[cost_layout]
        d.plan_layout = _capi.PLAN_LAYOUTS[plan_layout]
        d.sparse_slots = int(sparse_slots)
        self.desc = d


class Mam:
    """One MAM problem (or a batch) living on the GPU.

    ``capped=True`` selects the full unbalanced extension: columns are
    projected onto Delta_<=(q_s) and the cost becomes alpha_m (d - eta).
    """

    def __init__(self, problem=None, *, problems: Optional[Sequence] = None,
                 cost_dtype: str = "f32", theta0: str = "spread",
                 diag: str = "last", n_bundles: Optional[int] = None,
                 seed: int = 0, rho: Optional[float] = None,
                 gamma: Optional[float] = None, stream=None,
                 capped: bool = False, eta: float = 0.0, shard=None,
                 cost_layout: str = "per_column", plan_layout: str = "dense",
                 sparse_slots: int = 0):
        """``cost_layout="shared"`` stores one cost matrix for measures on a
        common support (mam_desc.cost_layout).
        ``plan_layout="sparse"`` stores each column's pihat as (row, value)
        pairs, at most ``sparse_slots`` of them (mam_desc.plan_layout).
        ``shard=(m_begin, m_end, allreduce)`` creates this rank's part of a
        measure-sharded problem (mam_create_sharded); ``allreduce`` is a
        ctypes ``_capi.ALLREDUCE_FN`` (see ``paper_2309_05315_gb300.shard``),
        kept alive with the handle."""
        L = _capi.lib()
        if (problem is None) == (problems is None):
            raise ValueError("give exactly one of problem / problems")
        if shard is not None and problems is not None:
            raise ValueError("a sharded problem is a single problem")
        probs = [problem] if problems is None else list(problems)
        st = None
        if stream is not None:
            st = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        keeps = [_DescKeep(p, cost_dtype, theta0, diag, n_bundles, seed, rho, gamma, st,
                           capped, eta, cost_layout, plan_layout, sparse_slots)
                 for p in probs]
        self._h = C.c_void_p()
        self._shard = None
        if shard is not None:
            m0, m1, fn = shard
            self._shard_fn = fn   # the callback must outlive the handle
            self._shard = MamShard(int(m0), int(m1), fn, None)
            check(L.mam_create_sharded(C.byref(keeps[0].desc), C.byref(self._shard),
                                       C.byref(self._h)))
        elif problems is None:
            check(L.mam_create(C.byref(keeps[0].desc), C.byref(self._h)))
        else:
            arr = (MamDesc * len(keeps))(*[k.desc for k in keeps])
            check(L.mam_batch_create(len(keeps), arr, C.byref(self._h)))
        self.batched = problems is not None
        P, Mt, R, T, ld = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int64(), C.c_int32()
        check(L.mam_get_sizes(self._h, C.byref(P), C.byref(Mt), C.byref(R), C.byref(T),
                              C.byref(ld)), self._h)
        self.n_problems, self.n_measures = P.value, Mt.value
        self.R, self.T, self.ld = R.value, T.value, ld.value
        self.dim = keeps[0].xi.shape[1]
        self.S_unpruned = np.concatenate([k.S for k in keeps])
        self.n_unpruned = int(self.S_unpruned.sum())

    # -- lifetime
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _capi.lib().mam_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, status):
        check(status, self._h)

    # -- iteration
    def step(self, n_iters: int = 1):
        self._check(_capi.lib().mam_step(self._h, int(n_iters)))

    def solve(self, max_iters: int, gap_tol: float = 1e-4, w_ref: float = 0.0,
              check_every: int = 10):
        it, gap = C.c_int32(), C.c_double()
        self._check(_capi.lib().mam_solve(self._h, int(max_iters), float(gap_tol),
                                          float(w_ref), int(check_every),
                                          C.byref(it), C.byref(gap)))
        return it.value, gap.value

    def objective(self, index: int = 0) -> dict:
        o = MamObjective()
        self._check(_capi.lib().mam_objective(self._h, int(index), C.byref(o)))
        return o.as_dict()

    def objectives(self) -> list:
        """Diagnostics of every problem (one mam_objective_all call)."""
        arr = (MamObjective * self.n_problems)()
        self._check(_capi.lib().mam_objective_all(self._h, arr))
        return [o.as_dict() for o in arr]

    # -- outputs
    def barycenter(self) -> np.ndarray:
        out = np.empty((self.n_problems, self.R), dtype=np.float64)
        self._check(_capi.lib().mam_get_barycenter(self._h, out.ctypes.data, 0))
        return out if self.batched else out[0]

    def update_support(self) -> np.ndarray:
        """Free-support step (Algorithm 2, Prop. 4): moves the support to the
        weighted means of the next step's plans, rebuilds the costs and
        returns the new support [R, dim]."""
        out = np.empty((self.R, self.dim), dtype=np.float64)
        self._check(_capi.lib().mam_update_support(self._h, out.ctypes.data))
        return out

    def free_support(self, outer: int, inner_iters: int, gap_tol: float = 0.0,
                     check_every: int = 10):
        """Algorithm 2: ``outer`` rounds of Algorithm 1 (``inner_iters``
        iterations, or to ``gap_tol``) followed by the support step.
        Returns (support [R, dim], iterations run)."""
        out = np.empty((self.R, self.dim), dtype=np.float64)
        it = C.c_int32()
        self._check(_capi.lib().mam_free_support(self._h, int(outer), int(inner_iters),
                                                 float(gap_tol), int(check_every),
                                                 out.ctypes.data, C.byref(it)))
        return out, it.value

    def barycenter_into(self, tensor):
        """Copy p into a CUDA float64 tensor of n_problems*R elements."""
        assert tensor.is_cuda and tensor.dtype.is_floating_point and tensor.element_size() == 8
        assert tensor.is_contiguous() and tensor.numel() == self.n_problems * self.R
        self._check(_capi.lib().mam_get_barycenter(self._h, C.c_void_p(tensor.data_ptr()), 1))
        return tensor

    def marginals(self) -> np.ndarray:
        out = np.empty((self.n_measures, self.R), dtype=np.float64)
        self._check(_capi.lib().mam_get_marginals(self._h, out.ctypes.data, 0))
        return out

    def theta(self) -> np.ndarray:
        out = np.empty((self.T, self.R), dtype=np.float32)
        self._check(_capi.lib().mam_get_theta(self._h, out.ctypes.data))
        return out

    def theta_columns(self, col0: int, ncols: int) -> np.ndarray:
        """Columns col0 .. col0 + ncols - 1 of the plans, [ncols][R] FP32."""
        out = np.empty((int(ncols), self.R), dtype=np.float32)
        self._check(_capi.lib().mam_get_theta_range(self._h, int(col0), int(ncols),
                                                    out.ctypes.data))
        return out

    def work(self) -> dict:
        """Columns projected and plan entries updated by the column steps so
        far (the index sets actually drawn)."""
        c, e = C.c_int64(), C.c_int64()
        self._check(_capi.lib().mam_get_work(self._h, C.byref(c), C.byref(e)))
        return {"columns": c.value, "entries": e.value}

    def pruned_sizes(self) -> np.ndarray:
        out = np.empty(self.n_measures, dtype=np.int32)
        self._check(_capi.lib().mam_get_pruned_sizes(self._h, out.ctypes.data))
        return out

    # -- checkpoints
    def get_state(self) -> bytes:
        n = C.c_size_t()
        self._check(_capi.lib().mam_get_state(self._h, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        self._check(_capi.lib().mam_get_state(self._h, buf, C.byref(n)))
        return buf.raw

    def set_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        self._check(_capi.lib().mam_set_state(self._h, buf, len(blob)))

    # -- configuration
    def config(self) -> dict:
        c = MamKernelConfig()
        self._check(_capi.lib().mam_get_config(self._h, C.byref(c)))
        return c.as_dict()

    def set_config(self, **kw):
        c = MamKernelConfig()
        self._check(_capi.lib().mam_get_config(self._h, C.byref(c)))
        for k, v in kw.items():
            setattr(c, k, int(v))
        self._check(_capi.lib().mam_set_config(self._h, C.byref(c)))

    def autotune(self, iters: int = 5) -> dict:
        c = MamKernelConfig()
        self._check(_capi.lib().mam_autotune(self._h, int(iters), C.byref(c)))
        return c.as_dict()

    # -- measurement
    def profile_enable(self, enable: bool = True):
        self._check(_capi.lib().mam_profile_enable(self._h, int(bool(enable))))

    def profile_read(self):
        c, a, n = C.c_double(), C.c_double(), C.c_int64()
        self._check(_capi.lib().mam_profile_read(self._h, C.byref(c), C.byref(a), C.byref(n)))
        return {"column_ms": c.value, "average_ms": a.value, "iterations": n.value}

    # -- differentiation
    def forward_record(self, K: int, ckpt_every: int = 20):
        self._check(_capi.lib().mam_forward_record(self._h, int(K), int(ckpt_every)))

    def backward(self, grad_p, want=("q", "zeta", "xi")):
        g = np.ascontiguousarray(grad_p, dtype=np.float64).reshape(self.R)
        gq = np.zeros(self.n_unpruned) if "q" in want else None
        gz = np.zeros((self.n_unpruned, self.dim)) if "zeta" in want else None
        gx = np.zeros((self.R, self.dim)) if "xi" in want else None
        ptr = lambda a: a.ctypes.data if a is not None else None
        self._check(_capi.lib().mam_backward(self._h, g.ctypes.data, ptr(gq), ptr(gz), ptr(gx)))
        return gq, gz, gx
