"""Algorithm 1 with Step 2 spread over worker processes (FP64, CPU).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/`` and
``bench.py``'s CPU-baseline legs use it; the library never does.

Step 2 of Algorithm 1 is independent across measures (each column of each
plan is projected on its own), so the measures are split into contiguous
groups of about equal size sum_m S_m and each group lives in its own worker
process (started with ``spawn``).  Every iteration the coordinating process
does Step 1 (p = sum_m a_m p^(m), eq. pr; the distance and t^k) and the
index set of Remark 2 exactly as ``MamOracle`` does, sends each worker the
shifts d^(m) = t (p - p^(m)) / S_m of its measures, and the worker runs
``column_step`` (the same function ``MamOracle.step`` calls) and returns the
new row marginals p^(m) (Step 3).  The arithmetic is that of ``MamOracle``
operation for operation, so the iterates are bit for bit the same; only the
wall time changes.  This is the "all cores" setting of the CPU baseline.
"""
from __future__ import annotations

import math
import multiprocessing as mp
import os
from typing import List, Optional

import numpy as np

from .mam_oracle import MamOracle, column_step, lower_bound


def _serve(conn, rho, capped):
    """Worker loop: holds theta, c, q of its measures."""
    items = conn.recv()
    theta = {m: th for m, th, _, _ in items}
    cost = {m: c for m, _, c, _ in items}
    q = {m: v for m, _, _, v in items}
    while True:
        msg = conn.recv()
        if msg is None:
            break
        kind, payload = msg
        if kind == "step":
            out = {}
            for m, d in payload.items():
                old = theta[m]
                th, lam, w_hat, phat = column_step(old, d, cost[m], q[m], rho, capped)
                res = float(np.sum((th - old) ** 2))
                theta[m] = th
                out[m] = (th.sum(axis=0), lam, w_hat, phat, res)
            conn.send(out)
        elif kind == "theta":
            conn.send({m: theta[m] for m in payload})
        else:
            conn.send(None)
    conn.close()


def measure_groups(S, n):
    """Split measures 0..M-1 into at most n contiguous groups of about equal
    sum_m S_m (the plan entries of a group are R sum_m S_m)."""
    S = [int(s) for s in S]
    n = max(1, min(int(n), len(S)))
    total = float(sum(S))
    groups, cur, acc = [], [], 0.0
    for m, s in enumerate(S):
        cur.append(m)
        acc += s
        left_groups = n - len(groups) - 1
        left_meas = len(S) - m - 1
        if left_groups > 0 and (acc >= total * (len(groups) + 1) / n or left_meas == left_groups):
            groups.append(cur)
            cur = []
    if cur:
        groups.append(cur)
    return groups


class ParallelMamOracle(MamOracle):
    """``MamOracle`` whose Step 2 runs in worker processes.

    Same constructor arguments plus ``workers`` (default: one per core, at
    most one per measure).  ``theta`` is gathered from the workers on access.
    Call ``close()`` (or use it as a context manager) to stop the workers.
    """

    def __init__(self, prep, rho, gamma=math.inf, n_bundles=1, seed=0, theta0="spread",
                 capped=False, workers: Optional[int] = None):
        super().__init__(prep, rho, gamma=gamma, n_bundles=n_bundles, seed=seed,
                         theta0=theta0, capped=capped)
        n = workers if workers else (os.cpu_count() or 1)
        self.groups = measure_groups(prep.S, n)
        ctx = mp.get_context("spawn")
        self._conns, self._procs = [], []
        self._owner = {}
        theta0_plans = self.__dict__.pop("_theta_init")
        for gi, g in enumerate(self.groups):
            a, b = ctx.Pipe()
            proc = ctx.Process(target=_serve, args=(b, self.rho, self.capped), daemon=True)
            proc.start()
            a.send([(m, theta0_plans[m], prep.c[m], prep.q[m]) for m in g])
            self._conns.append(a)
            self._procs.append(proc)
            for m in g:
                self._owner[m] = gi

    @property
    def workers(self) -> int:
        return len(self._conns)

    @property
    def theta(self) -> List[np.ndarray]:
        if "_theta_init" in self.__dict__:      # during MamOracle.__init__
            return self.__dict__["_theta_init"]
        for c, g in zip(self._conns, self.groups):
            c.send(("theta", g))
        out = {}
        for c in self._conns:
            out.update(c.recv())
        return [out[m] for m in range(self.prep.M)]

    @theta.setter
    def theta(self, plans):
        # Only MamOracle.__init__ assigns theta (theta^0); the plans then move
        # to the workers.
        self.__dict__["_theta_init"] = plans

    def step(self, diagnostics: bool = True):
        prep = self.prep
        S = prep.S
        p_old = self.barycenter()
        p, D, t = self.average()                              # Step 1
        Mk = self.index_set()
        d_all = [t * (p - self.pm[m]) / S[m] for m in range(prep.M)]
        jobs = [dict() for _ in self._conns]
        for m in Mk:                                          # Step 2 (workers)
            jobs[self._owner[m]][m] = d_all[m]
        busy = [i for i, j in enumerate(jobs) if j]
        for i in busy:
            self._conns[i].send(("step", jobs[i]))
        res = 0.0
        results = {}
        for i in busy:
            results.update(self._conns[i].recv())
        for m in Mk:                                          # Step 3
            pm, lam, w_hat, phat, r = results[m]
            self.pm[m] = pm
            self.lam[m] = lam
            self.w_hat_m[m] = w_hat
            self.phat_m[m] = phat
            res += r
        self.k += 1
        out = {"t": t, "dist_theta": D, "index_set": Mk}
        if diagnostics:
            out.update(self.diagnostics(d_all))
            out["fp_resid"] = math.sqrt(res)
            out["dp_norm"] = float(np.linalg.norm(self.barycenter() - p_old))
        self.last = out
        return out

    def next_pihat(self):
        raise NotImplementedError("the free-support step runs on MamOracle")

    def close(self):
        for c in self._conns:
            try:
                c.send(None)
            except Exception:
                pass
        for proc in self._procs:
            proc.join(timeout=10)
            if proc.is_alive():
                proc.terminate()
        self._conns, self._procs = [], []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


__all__ = ["ParallelMamOracle", "measure_groups", "lower_bound"]
