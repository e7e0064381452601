"""Algorithm 1 with Step 2 spread over worker processes (FP64, CPU).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only ``tests/`` and
``bench.py``'s CPU-baseline legs use it; the library never does.

Step 2 of Algorithm 1 is independent across measures (each column of each
plan is projected on its own), so the measures are split into contiguous
groups of about equal size sum_m S_m and each group lives in its own worker
process (started with ``spawn``).  A worker builds its measures' data itself
with ``prepare`` (pruning, costs) and holds their plans.  Every iteration the
coordinating process does Step 1 (p = sum_m a_m p^(m), eq. pr; the distance
and t^k) and the index set of Remark 2 with ``MamOracle``'s own code, sends
each worker the shifts d^(m) = t (p - p^(m)) / S_m of its measures, and the
worker runs ``column_step`` (the function ``MamOracle.step`` calls) and
returns the new row marginals p^(m) (Step 3).  Every number is computed by
the same operations as in ``MamOracle``, so the iterates are bit for bit the
same; only the wall time changes.  This is the "all cores" setting of the
CPU baseline, and it keeps only R-vectors in the coordinating process.
"""
from __future__ import annotations

import copy
import math
import multiprocessing as mp
import os
from typing import List, Optional

import numpy as np

from .mam_oracle import MamOracle, averaging_weights, bundles, column_step, prepare


def _serve(conn):
    """Worker loop: builds and holds theta, c, q of its measures."""
    sub, ids, rho, cost_dtype, eta, theta0, capped = conn.recv()
    prep = prepare(sub, cost_dtype, eta=eta)
    R = prep.R
    if theta0 == "spread":
        theta = [np.repeat((q / R)[:, None], R, axis=1) for q in prep.q]
    else:
        theta = [np.zeros((len(q), R)) for q in prep.q]
    local = {m: i for i, m in enumerate(ids)}
    conn.send({m: theta[i].sum(axis=0) for m, i in local.items()})     # Step 0 marginals
    while True:
        msg = conn.recv()
        if msg is None:
            break
        kind, payload = msg
        if kind == "step":
            out = {}
            for m, d in payload.items():
                i = local[m]
                old = theta[i]
                th, lam, w_hat, phat = column_step(old, d, prep.c[i], prep.q[i], rho, capped)
                res = float(np.sum((th - old) ** 2))
                theta[i] = th
                out[m] = (th.sum(axis=0), lam, w_hat, phat, res)
            conn.send(out)
        elif kind == "lb":   # per-measure terms of lower_bound (same operations)
            out = {}
            for m, v in payload.items():
                i = local[m]
                col = (prep.c[i] - v[None, :]).min(axis=1)
                if capped:
                    col = np.minimum(col, 0.0)
                out[m] = float(np.dot(prep.q[i], col))
            conn.send(out)
        elif kind == "theta":
            conn.send({m: theta[local[m]] for m in payload})
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


class _Light:
    """What the coordinator keeps of the pruned problem: sizes, weights and
    averaging weights (no plans, no costs)."""

    def __init__(self, problem):
        self.q = []
        for m in range(problem.M):
            qm = np.asarray(problem.q[m], dtype=np.float64)
            self.q.append(qm[qm > 0])
        self.S = np.asarray([len(q) for q in self.q], dtype=np.int64)
        self.R = problem.R
        self.alpha = np.asarray(problem.alpha, dtype=np.float64)
        self.a = averaging_weights(self.S)

    @property
    def M(self):
        return len(self.q)


class ParallelMamOracle(MamOracle):
    """``MamOracle`` whose Step 2 runs in worker processes.

    Built from the problem itself (``prepare`` runs in the workers, with
    ``cost_dtype`` and ``eta`` as there); otherwise the arguments of
    ``MamOracle``, plus ``workers`` (default: one per core, at most one per
    measure).  ``theta`` is gathered from the workers on access.  Call
    ``close()`` (or use it as a context manager) to stop the workers.
    """

    def __init__(self, problem, rho: Optional[float] = None, gamma=math.inf, n_bundles=1,
                 seed=0, theta0="spread", capped=False, cost_dtype="f64", eta=0.0,
                 workers: Optional[int] = None):
        rho = float(problem.rho if rho is None else rho)
        if rho <= 0:
            raise ValueError("rho must be positive")
        self.prep = _Light(problem)
        self.rho, self.gamma, self.capped = rho, float(gamma), bool(capped)
        self.nb = max(1, int(n_bundles))
        self.seed = int(seed)
        self.B = bundles(self.prep.M, self.nb)
        M, R = self.prep.M, self.prep.R
        self.k = 0
        self.w_hat_m = np.zeros(M)
        self.phat_m = [np.zeros(R) for _ in range(M)]
        self.lam = [np.zeros(len(q)) for q in self.prep.q]
        self.last = {}
        n = workers if workers else (os.cpu_count() or 1)
        self.groups = measure_groups(self.prep.S, n)
        ctx = mp.get_context("spawn")
        self._conns, self._procs, self._owner = [], [], {}
        for gi, g in enumerate(self.groups):
            sub = copy.copy(problem)
            sub.q = [problem.q[m] for m in g]
            sub.zeta = [problem.zeta[m] for m in g]
            sub.alpha = np.asarray(problem.alpha)[g]
            sub.cost = None if problem.cost is None else [problem.cost[m] for m in g]
            a, b = ctx.Pipe()
            proc = ctx.Process(target=_serve, args=(b,), daemon=True)
            proc.start()
            a.send((sub, list(g), rho, cost_dtype, float(eta), theta0, self.capped))
            self._conns.append(a)
            self._procs.append(proc)
            for m in g:
                self._owner[m] = gi
        pm = {}
        for c in self._conns:
            pm.update(c.recv())
        self.pm = [pm[m] for m in range(M)]

    @property
    def workers(self) -> int:
        return len(self._conns)

    @property
    def theta(self) -> List[np.ndarray]:
        for c, g in zip(self._conns, self.groups):
            c.send(("theta", g))
        out = {}
        for c in self._conns:
            out.update(c.recv())
        return [out[m] for m in range(self.prep.M)]

    def _ask(self, kind, per_measure):
        jobs = [dict() for _ in self._conns]
        for m, v in per_measure.items():
            jobs[self._owner[m]][m] = v
        busy = [i for i, j in enumerate(jobs) if j]
        for i in busy:
            self._conns[i].send((kind, jobs[i]))
        out = {}
        for i in busy:
            out.update(self._conns[i].recv())
        return out

    def step(self, diagnostics: bool = True):
        S = self.prep.S
        p_old = self.barycenter()
        p, D, t = self.average()                              # Step 1
        Mk = self.index_set()
        d_all = [t * (p - self.pm[m]) / S[m] for m in range(self.prep.M)]
        results = self._ask("step", {m: d_all[m] for m in Mk})   # Step 2 (workers)
        res = 0.0
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

    def diagnostics(self, d_all):
        from .mam_oracle import dist_balanced
        w_hat = float(self.w_hat_m.sum())
        dist_hat = dist_balanced(self.phat_m, self.prep.S)
        f_unbal = w_hat + (0.0 if math.isinf(self.gamma) else self.gamma * dist_hat)
        terms = self._ask("lb", {m: self.rho * d_all[m] for m in range(self.prep.M)})
        lb = 0.0
        for m in range(self.prep.M):                        # lower_bound's order
            lb += terms[m]
        return {"w_hat": w_hat, "dist_pihat": dist_hat, "f_unbal": f_unbal,
                "lower_bound": lb}

    def next_pihat(self):
        raise NotImplementedError("the free-support step runs on MamOracle")

    def update_support(self, eta: float = 0.0):
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


__all__ = ["ParallelMamOracle", "measure_groups"]
