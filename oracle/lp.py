"""Exact LP of the fixed-support barycenter (eq. HugeLP), for small instances.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Solved with HiGHS through
``scipy.optimize.linprog``.  Variables are the plans pi^(m) (pruned columns,
stored like the oracle's plans: entry (s, r) of measure m) followed by the
barycenter p.  Rows:
  sum_r pi^(m)_{rs} = q^(m)_s            (column marginals, eq. Pi)
  sum_s pi^(m)_{rs} - p_r = 0            (row marginals, eq. HugeLP)
p is left free: pi >= 0 already makes it nonnegative and the column rows fix
its mass.  The duals (u, v) of the two row families satisfy
c^(m)_{rs} - u^(m)_s - v^(m)_r >= 0 and sum_m v^(m) = 0.

With ``capped=True`` the column rows become sum_r pi^(m)_{rs} <= q^(m)_s:
the full unbalanced extension with g the indicator of L (every plan has the
same row marginals), whose shifted cost alpha_m (d - eta) comes with the
prepared data.
"""
from __future__ import annotations

import numpy as np
from scipy import optimize, sparse


def solve_barycenter_lp(prep, capped: bool = False):
    """Return dict(opt, pi (list of (S_m,R)), p, u (list), v (list))."""
    M, R = prep.M, prep.R
    S = [int(s) for s in prep.S]
    nvar = sum(s * R for s in S) + R
    rows, cols, vals, b = [], [], [], []
    off = 0
    row = 0
    col_rows = []
    for m in range(M):
        for s in range(S[m]):
            for r in range(R):
                rows.append(row); cols.append(off + s * R + r); vals.append(1.0)
            b.append(prep.q[m][s]); row += 1
        off += S[m] * R
    off = 0
    for m in range(M):
        for r in range(R):
            for s in range(S[m]):
                rows.append(row); cols.append(off + s * R + r); vals.append(1.0)
            rows.append(row); cols.append(nvar - R + r); vals.append(-1.0)
            b.append(0.0); row += 1
        off += S[m] * R
    A = sparse.csr_matrix((vals, (rows, cols)), shape=(row, nvar))
    cvec = np.concatenate([prep.c[m].ravel() for m in range(M)] + [np.zeros(R)])
    bounds = [(0, None)] * (nvar - R) + [(None, None)] * R
    b = np.asarray(b)
    if capped:
        ncol = sum(S)  # the column rows come first
        res = optimize.linprog(cvec, A_ub=A[:ncol], b_ub=b[:ncol], A_eq=A[ncol:],
                               b_eq=b[ncol:], bounds=bounds, method="highs")
    else:
        res = optimize.linprog(cvec, A_eq=A, b_eq=b, bounds=bounds, method="highs")
    if res.status != 0:
        raise RuntimeError(res.message)
    x = res.x
    y = (np.concatenate([res.ineqlin.marginals, res.eqlin.marginals]) if capped
         else res.eqlin.marginals)
    pi, u, v = [], [], []
    off = 0
    urow = 0
    for m in range(M):
        pi.append(x[off:off + S[m] * R].reshape(S[m], R))
        off += S[m] * R
        u.append(y[urow:urow + S[m]])
        urow += S[m]
    for m in range(M):
        v.append(y[urow:urow + R])
        urow += R
    return {"opt": float(res.fun), "pi": pi, "p": x[nvar - R:], "u": u, "v": v}
