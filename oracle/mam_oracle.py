"""Plain FP64 oracle of the Method of Averaged Marginals (MAM).

TEST INFRASTRUCTURE ONLY.  This module is the slow, obviously-correct
statement of what the CUDA library computes.  Only ``tests/``, the package's
``smoke()`` check and the CPU-baseline leg of ``bench.py`` may import it; the
library never does, and it shares no code with the CUDA path.

Everything is numpy float64, written step by step in the paper's order and
notation (arXiv 2309.05315):

* eq. (Delta), Remark 1 ......... ``project_simplex`` (sort-based, exact)
* Delta_<=(tau) of the full unbalanced extension ... ``project_capped_simplex``
* Prop. 2, eq. (pr)/(row_sol) ..... ``proj_balanced``
* Section 5 ("Balanced and unbalanced settings") ... ``dist_balanced``
* Section 4.3 "Storage complexity" (pruning), eq. (HugeLP) (cost) ... ``prepare``
* Algorithm 1 (MAM), Remark 2 (bundles) ... ``MamOracle.step``
* eq. (DR) + Lagrangian duality of eq. (HugeLP) ... ``lower_bound``
* Prop. 4 and Algorithm 2 (free-support update) ... ``support_from_plans``,
  ``MamOracle.update_support``

Storage convention: the paper's plan theta^(m) is R x S_m.  Here each
measure's plan is a numpy array of shape (S_m, R): row s holds the paper's
column s, i.e. ``theta[m][s, r]`` is theta^(m)_{rs}.  Columns are therefore
contiguous, as in the CUDA library.

Parity pins (see tests/test_oracle_*.py): every function here is checked
against brute force, closed forms, least squares, the HiGHS LP optimum, the
exact DR fixed point built from LP duals, finite differences, invariants,
hand-derived IEEE 754 rounding results (``round_to_bf16``/``round_to_f16``),
a hand-worked dist_L example, and the minimum of eq. (UWB) from a general
constrained solver (the unbalanced objective F).
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence

import numpy as np

F64 = np.float64


# --------------------------------------------------------------------------
# Simplex projection: eq. (Delta), Prop. 3, Remark 1.
# --------------------------------------------------------------------------

def project_simplex(W, tau):
    """Euclidean projection of each row of W onto Delta_R(tau_i).

    Delta_R(tau) = {u >= 0 : sum(u) = tau} (eq. Delta).  Remark 1: for
    tau = 0 the set is {0}.  For tau > 0 we use the classical sort-based
    exact method (Held, Wolfe and Crowder 1974): sort w in decreasing order
    as u_1 >= ... >= u_R, let K be the largest k with
    u_k - (sum_{j<=k} u_j - tau)/k > 0, set lambda = (sum_{j<=K} u_j - tau)/K
    and return max(w - lambda, 0).  The projection is unique, so this gives
    the same point as the Condat algorithm the paper cites.

    Returns (X, lam) where lam[i] is the threshold of row i (0 when tau=0).
    """
    W = np.atleast_2d(np.asarray(W, dtype=F64))
    n, R = W.shape
    tau = np.broadcast_to(np.asarray(tau, dtype=F64), (n,))
    X = np.zeros_like(W)
    lam = np.zeros(n)
    pos = tau > 0
    if not np.any(pos):
        return X, lam
    Wp = W[pos]
    U = -np.sort(-Wp, axis=1)                       # decreasing order
    css = np.cumsum(U, axis=1) - tau[pos][:, None]  # sum_{j<=k} u_j - tau
    k = np.arange(1, R + 1, dtype=F64)
    cond = U - css / k > 0
    K = R - np.argmax(cond[:, ::-1], axis=1)        # largest k with cond true
    lam_p = css[np.arange(Wp.shape[0]), K - 1] / K
    X[pos] = np.maximum(Wp - lam_p[:, None], 0.0)
    lam[pos] = lam_p
    return X, lam


# --------------------------------------------------------------------------
# Projection onto Delta_<=(tau): the full unbalanced extension of the paper
# (its section "Algorithm's Extension: the Full Unbalanced Setting").
# --------------------------------------------------------------------------

def project_capped_simplex(W, tau):
    """Euclidean projection of each row of W onto Delta_<=(tau_i).

    Delta_<=(tau) = {u >= 0 : sum(u) <= tau}.  The paper's two steps: clip,
    w_check = max(w, 0); if sum(w_check) <= tau the clipped vector is the
    projection, otherwise the projection is the one onto Delta_R(tau).  For
    tau = 0 the set is {0}.

    Returns (X, lam): lam[i] is 0 where the clipped vector is returned, the
    simplex threshold of ``project_simplex`` otherwise.
    """
    W = np.atleast_2d(np.asarray(W, dtype=F64))
    n, _ = W.shape
    tau = np.broadcast_to(np.asarray(tau, dtype=F64), (n,))
    X = np.maximum(W, 0.0)                     # first step: clip
    lam = np.zeros(n)
    over = X.sum(axis=1) > tau                 # second step where the mass exceeds tau
    if np.any(over):
        X_over, lam_over = project_simplex(W[over], tau[over])
        X[over] = X_over
        lam[over] = lam_over
    return X, lam


# --------------------------------------------------------------------------
# Projection onto the balanced subspace L: Prop. 2, eqs. (pr) and (row_sol).
# --------------------------------------------------------------------------

def averaging_weights(S):
    """a_m = (1/S_m) / sum_j (1/S_j), eq. (pr)."""
    inv = 1.0 / np.asarray(S, dtype=F64)
    return inv / inv.sum()


def proj_balanced(thetas: Sequence[np.ndarray]):
    """Proj_L(theta) by the closed form of Prop. 2.

    p^(m)_r = sum_s theta^(m)_{rs}; p = sum_m a_m p^(m);
    pi^(m)_{rs} = theta^(m)_{rs} + (p_r - p^(m)_r) / S_m.
    Returns (list of pi^(m), p).
    """
    S = [t.shape[0] for t in thetas]
    a = averaging_weights(S)
    pm = [t.sum(axis=0) for t in thetas]
    p = sum(a[m] * pm[m] for m in range(len(thetas)))
    return [thetas[m] + ((p - pm[m]) / S[m])[None, :] for m in range(len(thetas))], p


def dist_balanced(pm: Sequence[np.ndarray], S) -> float:
    """dist_L(theta) = sqrt(sum_m ||p - p^(m)||^2 / S_m) (text after Alg. 1).

    ``pm`` are the row marginals of theta; p is their a-weighted average.
    """
    a = averaging_weights(S)
    p = sum(a[m] * pm[m] for m in range(len(pm)))
    return math.sqrt(sum(float(np.dot(p - pm[m], p - pm[m])) / S[m]
                         for m in range(len(pm))))


# --------------------------------------------------------------------------
# Problem data: pruning (Section 4.3) and cost (eq. HugeLP).
# --------------------------------------------------------------------------

def round_to_bf16(x):
    """Round float64 -> float32 (nearest) -> bfloat16 (nearest, ties to even).

    Done with integer bit manipulation on the float32 pattern, so it does not
    depend on any library's bfloat16 support.  Returns float64 values.
    """
    f = np.asarray(x, dtype=np.float32)
    b = f.view(np.uint32).astype(np.uint64)
    lsb = (b >> np.uint64(16)) & np.uint64(1)
    b = (b + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return b.astype(np.uint32).view(np.float32).astype(F64)


def round_to_f16(x):
    """Round float64 -> float32 (nearest) -> IEEE binary16 (nearest even)."""
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(F64)


@dataclasses.dataclass
class Prepared:
    """Pruned problem data (all FP64)."""
    R: int
    S: np.ndarray             # (M,) pruned support sizes S_m
    keep: List[np.ndarray]    # per measure: indices (unpruned) of kept columns
    q: List[np.ndarray]       # per measure (S_m,) positive weights
    zeta: List[np.ndarray]    # per measure (S_m, dim) kept support points
    xi: np.ndarray            # (R, dim)
    alpha: np.ndarray         # (M,)
    c: List[np.ndarray]       # per measure (S_m, R): c[m][s, r] = c^(m)_{rs}
    a: np.ndarray             # (M,) averaging weights of eq. (pr)

    @property
    def M(self):
        return len(self.q)


def sq_euclid_cost(xi, zeta, alpha_m, eta: float = 0.0):
    """c_{rs} = alpha_m (||xi_r - zeta_s||^2 - eta), shape (S, R).

    eta = 0 is eq. (HugeLP); eta > 0 is the shifted distance matrix of the
    full unbalanced extension, alpha_m [d(xi_r, zeta_s) - eta].
    """
    diff = zeta[:, None, :] - xi[None, :, :]
    return alpha_m * (np.einsum("srd,srd->sr", diff, diff) - eta)


def prepare(problem, cost_dtype: str = "f64", eta: float = 0.0,
            round_before_alpha: bool = False) -> Prepared:
    """Drop zero-weight columns (Section 4.3) and build the costs.

    The cost of measure m is alpha_m ||xi_r - zeta_s||^2 (eq. HugeLP), or
    alpha_m * C^(m) when the problem carries a general cost matrix C^(m)
    (the paper notes no assumption on the costs is needed, Section 2).
    With eta > 0 (full unbalanced extension) the distance is shifted first:
    alpha_m (||xi_r - zeta_s||^2 - eta), or alpha_m (C^(m) - eta).
    ``cost_dtype`` in {"f64", "f32", "bf16", "f16"} rounds the stored cost
    the way a reduced-precision store would (FP64 -> FP32 -> target).
    ``round_before_alpha`` rounds the distance matrix before alpha_m scales
    it (a store that keeps one matrix for all measures and applies alpha_m
    afterwards); by default the scaled cost alpha_m d is rounded.
    """
    xi = np.asarray(problem.xi, dtype=F64)
    S, keep, qs, zs, cs = [], [], [], [], []
    for m in range(problem.M):
        qm = np.asarray(problem.q[m], dtype=F64)
        idx = np.nonzero(qm > 0)[0]
        keep.append(idx)
        qs.append(qm[idx])
        zs.append(np.asarray(problem.zeta[m], dtype=F64)[idx])
        S.append(len(idx))
        am = float(problem.alpha[m])
        scale = 1.0 if round_before_alpha else am
        if problem.cost is not None:
            cm = scale * (np.asarray(problem.cost[m], dtype=F64)[idx] - eta)
        else:
            cm = sq_euclid_cost(xi, zs[-1], scale, eta)
        if cost_dtype == "f32":
            cm = cm.astype(np.float32).astype(F64)
        elif cost_dtype == "bf16":
            cm = round_to_bf16(cm)
        elif cost_dtype == "f16":
            cm = round_to_f16(cm)
        elif cost_dtype != "f64":
            raise ValueError(cost_dtype)
        cs.append(am * cm if round_before_alpha else cm)
    S = np.asarray(S, dtype=np.int64)
    return Prepared(R=xi.shape[0], S=S, keep=keep, q=qs, zeta=zs, xi=xi,
                    alpha=np.asarray(problem.alpha, dtype=F64), c=cs,
                    a=averaging_weights(S))


# --------------------------------------------------------------------------
# Randomized index sets: Remark 2.
# --------------------------------------------------------------------------

_MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """SplitMix64 output function (Steele, Lea and Flood 2014)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def bundles(M: int, nb: int):
    """Partition {0..M-1} into nb contiguous bundles A_i (Remark 2)."""
    return [list(range((i * M) // nb, ((i + 1) * M) // nb)) for i in range(nb)]


def bundle_sequence(alpha, nb: int, seed: int, n_iters: int, start: int = 0):
    """Bundle index drawn at iterations start..start+n_iters-1 (Remark 2).

    Bundle A_i is drawn with probability beta_i = sum_{m in A_i} alpha_m
    (normalised).  Draw k uses the counter-based generator
    u_k = (splitmix64(seed + k * 0x9E3779B97F4A7C15) >> 11) * 2^-53 and picks
    the first i whose cumulative probability exceeds u_k.
    """
    M = len(alpha)
    B = bundles(M, nb)
    beta = [float(sum(alpha[m] for m in A)) for A in B]
    tot = sum(beta)
    cum, acc = [], 0.0
    for b in beta:
        acc += b / tot
        cum.append(acc)
    out = []
    for k in range(start, start + n_iters):
        z = splitmix64((seed + k * 0x9E3779B97F4A7C15) & _MASK64)
        u = (z >> 11) * (1.0 / (1 << 53))
        i = 0
        while i < nb - 1 and not (u < cum[i]):
            i += 1
        out.append(i)
    return out


# --------------------------------------------------------------------------
# Lagrangian lower bound of eq. (HugeLP) / (UWB).
# --------------------------------------------------------------------------

def lower_bound(prep: Prepared, v: Sequence[np.ndarray], capped: bool = False) -> float:
    """LB(v) = sum_m sum_s q_s min_r (c^(m)_{rs} - v^(m)_r).

    Relaxing the coupling rows sum_s pi^(m)_{rs} = p_r of eq. (HugeLP) with
    multipliers v^(m) satisfying sum_m v^(m) = 0 (so that p drops out) leaves
    M independent problems over Pi^(m) whose minimum is attained column by
    column at the cheapest row.  For eq. (UWB) the same value is a lower
    bound whenever, in addition, sum_m S_m ||v^(m)||^2 <= gamma^2, because
    gamma dist_L(pi) >= <u, pi> for every u in L^perp with ||u|| <= gamma.
    With capped columns (sum_r pi_{rs} <= q_s, the full unbalanced
    extension) a column may also carry no mass, so its term is
    q_s min(0, min_r (c_{rs} - v_r)).
    """
    tot = 0.0
    for m in range(prep.M):
        col = (prep.c[m] - v[m][None, :]).min(axis=1)
        if capped:
            col = np.minimum(col, 0.0)
        tot += float(np.dot(prep.q[m], col))
    return tot


# --------------------------------------------------------------------------
# Algorithm 1.
# --------------------------------------------------------------------------

def column_step(theta_m, d, c_m, q_m, rho, capped=False):
    """Step 2 of Algorithm 1 for the plan of one measure.

    w = theta + 2 d - c / rho column by column, pi-hat = the projection of
    each column onto Delta_R(q_s) (onto Delta_<=(q_s) when ``capped``), and
    theta' = pi-hat - d.  Returns (theta', thresholds, <c, pi-hat>, row sums
    of pi-hat).
    """
    w = theta_m + 2.0 * d[None, :] - c_m / rho
    if capped:
        pihat, lam = project_capped_simplex(w, q_m)
    else:
        pihat, lam = project_simplex(w, q_m)
    return pihat - d[None, :], lam, float(np.sum(c_m * pihat)), pihat.sum(axis=0)


class MamOracle:
    """Algorithm 1 (MAM), deterministic or randomized, balanced or not.

    ``capped`` replaces the projection onto Delta_R(q_s) of Step 2 with the
    one onto Delta_<=(q_s) (full unbalanced extension; its shifted cost is
    built by ``prepare(..., eta=...)``).

    State: theta (list of (S_m, R) arrays) and the marginals p^(m) of the
    last update of each measure (Step 0 / Step 3).
    """

    def __init__(self, prep: Prepared, rho: float, gamma: float = math.inf,
                 n_bundles: int = 1, seed: int = 0, theta0: str = "spread",
                 capped: bool = False):
        if rho <= 0:
            raise ValueError("rho must be positive")
        self.prep = prep
        self.rho = float(rho)
        self.gamma = float(gamma)
        self.capped = bool(capped)
        self.nb = max(1, int(n_bundles))
        self.seed = int(seed)
        self.B = bundles(prep.M, self.nb)
        R = prep.R
        # Step 0 (theta^0 is arbitrary, Section 4.4 "Initialization"):
        # "spread" puts q_s/R in every row of column s, "zero" is all zeros.
        if theta0 == "spread":
            self.theta = [np.repeat((q / R)[:, None], R, axis=1) for q in prep.q]
        elif theta0 == "zero":
            self.theta = [np.zeros((len(q), R)) for q in prep.q]
        else:
            raise ValueError(theta0)
        self.pm = [t.sum(axis=0) for t in self.theta]      # Step 0 marginals
        self.k = 0
        # Last pi-hat quantities per measure (diagnostics).
        self.w_hat_m = np.zeros(prep.M)
        self.phat_m = [np.zeros(R) for _ in range(prep.M)]
        self.lam = [np.zeros(len(q)) for q in prep.q]
        self.last = {}

    # Step 1 + the unbalanced factor t^k of Algorithm 1.
    def average(self):
        S, a = self.prep.S, self.prep.a
        p = sum(a[m] * self.pm[m] for m in range(self.prep.M))
        D = math.sqrt(sum(float(np.dot(p - self.pm[m], p - self.pm[m])) / S[m]
                          for m in range(self.prep.M)))
        if math.isinf(self.gamma) or self.rho * D <= self.gamma:
            t = 1.0
        else:
            t = self.gamma / (self.rho * D)
        return p, D, t

    def barycenter(self):
        """p = sum_m a_m p^(m) of the current theta (returned p-bar)."""
        return sum(self.prep.a[m] * self.pm[m] for m in range(self.prep.M))

    def index_set(self):
        """M^k: all measures, or the bundle drawn by Remark 2."""
        if self.nb == 1:
            return list(range(self.prep.M))
        i = bundle_sequence(self.prep.alpha, self.nb, self.seed, 1, self.k)[0]
        return self.B[i]

    def step(self, diagnostics: bool = True):
        """One iteration of Algorithm 1; returns a dict of diagnostics."""
        prep, rho = self.prep, self.rho
        S = prep.S
        theta_old = [t.copy() for t in self.theta] if diagnostics else None
        p_old = self.barycenter()
        p, D, t = self.average()                              # Step 1
        Mk = self.index_set()
        d_all = [t * (p - self.pm[m]) / S[m] for m in range(prep.M)]
        for m in Mk:                                          # Step 2
            (self.theta[m], self.lam[m], self.w_hat_m[m],
             self.phat_m[m]) = column_step(self.theta[m], d_all[m], prep.c[m], prep.q[m],
                                           rho, self.capped)
        for m in Mk:                                          # Step 3
            self.pm[m] = self.theta[m].sum(axis=0)
        self.k += 1
        out = {"t": t, "dist_theta": D, "index_set": Mk}
        if diagnostics:
            out.update(self.diagnostics(d_all))
            out["fp_resid"] = math.sqrt(sum(
                float(np.sum((self.theta[m] - theta_old[m]) ** 2))
                for m in range(prep.M)))
            p_new = self.barycenter()
            out["dp_norm"] = float(np.linalg.norm(p_new - p_old))
        self.last = out
        return out

    def diagnostics(self, d_all):
        """W-hat, dist_L(pi-hat), F(pi-hat) and the lower bound LB."""
        prep = self.prep
        w_hat = float(self.w_hat_m.sum())
        dist_hat = dist_balanced(self.phat_m, prep.S)
        f_unbal = w_hat + (0.0 if math.isinf(self.gamma) else self.gamma * dist_hat)
        lb = lower_bound(prep, [self.rho * d for d in d_all], self.capped)
        return {"w_hat": w_hat, "dist_pihat": dist_hat, "f_unbal": f_unbal,
                "lower_bound": lb}

    def run(self, n_iters: int, diagnostics: bool = False):
        out = None
        for _ in range(n_iters):
            out = self.step(diagnostics)
        return out

    def next_pihat(self):
        """The projected plans pi-hat the next step would compute (Step 1 and
        the projection of Step 2, without the theta update)."""
        prep, rho = self.prep, self.rho
        p, _, t = self.average()
        out = []
        for m in range(prep.M):
            d = t * (p - self.pm[m]) / prep.S[m]
            w = self.theta[m] + 2.0 * d[None, :] - prep.c[m] / rho
            proj = project_capped_simplex if self.capped else project_simplex
            out.append(proj(w, prep.q[m])[0])
        return out

    def update_support(self, eta: float = 0.0):
        """Algorithm 2, support step: xi from Prop. 4 with the plans pi-hat of
        the next step, then the costs of the new support (eta as in
        ``prepare``).  theta and the marginals are kept (warm start)."""
        prep = self.prep
        xi = support_from_plans(prep.xi, prep.zeta, prep.alpha, self.next_pihat())
        for m in range(prep.M):
            prep.c[m] = sq_euclid_cost(xi, prep.zeta[m], float(prep.alpha[m]), eta)
        prep.xi = xi
        return xi


# --------------------------------------------------------------------------
# Free support: Prop. 4 (support step of Algorithm 2).
# --------------------------------------------------------------------------

def support_from_plans(xi, zeta, alpha, plans):
    """xi_r = sum_m alpha_m sum_s zeta^(m)_s pi_{rs} / sum_m alpha_m sum_s pi_{rs}
    (Prop. 4), the minimiser over xi of
    Psi(xi) = sum_m alpha_m sum_{r,s} ||xi_r - zeta_s||^2 pi_{rs} / 2.
    Rows that carry no mass keep their point.  ``plans`` are (S_m, R) arrays
    like the oracle's plans."""
    xi = np.asarray(xi, dtype=F64)
    num = np.zeros_like(xi)
    den = np.zeros(xi.shape[0])
    for m, pl in enumerate(plans):
        num += alpha[m] * (pl.T @ np.asarray(zeta[m], dtype=F64))
        den += alpha[m] * pl.sum(axis=0)
    out = xi.copy()
    nz = den > 0
    out[nz] = num[nz] / den[nz][:, None]
    return out


def free_support(problem, outer: int, inner: int, eta: float = 0.0,
                 gamma: float = math.inf, capped: bool = False):
    """Algorithm 2: ``outer`` rounds of (``inner`` iterations of Algorithm 1
    on the current support, then the support step of Prop. 4).  theta is
    kept across rounds.  Returns the oracle (its prep holds the last
    support and costs)."""
    prep = prepare(problem, eta=eta)
    orc = MamOracle(prep, problem.rho, gamma=gamma, capped=capped)
    for _ in range(outer):
        orc.run(inner)
        orc.update_support(eta)
    return orc


# --------------------------------------------------------------------------
# Reverse mode through K unrolled iterations (balanced, deterministic).
# --------------------------------------------------------------------------

def unrolled_loss_and_grad(problem, K: int, rho: float, target,
                           theta0: str = "spread"):
    """L = ||p^K - target||^2 and its gradient w.r.t. q, zeta and xi.

    The forward pass is Algorithm 1 (t = 1, all measures every iteration).
    The reverse pass differentiates each step exactly where the active sets
    A_s = {r : w_r > lambda_s} are locally constant:
      pi-hat = max(w - lambda, 0) has d(pi-hat)/dw = I_A - 1_A 1_A^T / |A| and
      d(pi-hat)/dq_s = 1_A / |A|;  theta' = pi-hat - d;
      w = theta + 2 d - c/rho;  d^(m) = (p - p^(m)) / S_m;
      p = sum_m a_m p^(m);  p^(m) = row sums of theta^(m);
      c^(m)_{rs} = alpha_m ||xi_r - zeta_s||^2;  theta^0_{rs} = q_s / R.
    Gradients for pruned (q_s = 0) columns are zero (one-sided kink).
    Returns (loss, grad_q list (unpruned), grad_zeta list (unpruned), grad_xi).
    """
    prep = prepare(problem, "f64")
    M, R, S, a = prep.M, prep.R, prep.S, prep.a
    orc = MamOracle(prep, rho, theta0=theta0)
    # The reverse pass needs, of each forward step, only its active sets
    # A_s = {r : w_r > lambda_s}; they are kept as packed bits (one per plan
    # entry) instead of copies of theta^k.
    masks = []
    for _ in range(K):
        p, _, _ = orc.average()
        d = [(p - orc.pm[m]) / S[m] for m in range(M)]
        w = [orc.theta[m] + 2.0 * d[m][None, :] - prep.c[m] / rho for m in range(M)]
        orc.step(diagnostics=False)
        masks.append([np.packbits(w[m] > orc.lam[m][:, None], axis=1) for m in range(M)])
    pK = orc.barycenter()
    diff = pK - np.asarray(target, dtype=F64)
    loss = float(np.dot(diff, diff))
    gp = 2.0 * diff
    # theta-bar^K from p^K = sum_m a_m rowsum(theta^(m),K)
    tbar = [np.repeat((a[m] * gp)[None, :], S[m], axis=0) for m in range(M)]
    gq = [np.zeros(S[m]) for m in range(M)]
    cbar = [np.zeros((S[m], R)) for m in range(M)]
    for k in range(K - 1, -1, -1):
        dbar = []
        new_tbar = []
        for m in range(M):
            A = np.unpackbits(masks[k][m], axis=1, count=R).astype(bool)
            nA = A.sum(axis=1)
            pibar = tbar[m]                                  # theta' = pihat - d
            meanA = np.where(A, pibar, 0.0).sum(axis=1) / nA
            wbar = np.where(A, pibar - meanA[:, None], 0.0)
            gq[m] += meanA
            cbar[m] += -wbar / rho
            dbar.append((2.0 * wbar - pibar).sum(axis=0))    # via w and theta'
            new_tbar.append(wbar)
        pbar = sum(dbar[m] / S[m] for m in range(M))
        for m in range(M):
            pmbar = -dbar[m] / S[m] + a[m] * pbar
            new_tbar[m] = new_tbar[m] + pmbar[None, :]
        tbar = new_tbar
    if theta0 == "spread":
        for m in range(M):
            gq[m] += tbar[m].sum(axis=1) / R
    gxi = np.zeros_like(prep.xi)
    gq_full, gz_full = [], []
    for m in range(M):
        diffz = prep.xi[None, :, :] - prep.zeta[m][:, None, :]   # (S, R, dim)
        coef = 2.0 * prep.alpha[m] * cbar[m]                      # (S, R)
        gz = -np.einsum("sr,srd->sd", coef, diffz)
        gxi += np.einsum("sr,srd->rd", coef, diffz)
        qf = np.zeros(len(problem.q[m]))
        qf[prep.keep[m]] = gq[m]
        zf = np.zeros_like(np.asarray(problem.zeta[m], dtype=F64))
        zf[prep.keep[m]] = gz
        gq_full.append(qf)
        gz_full.append(zf)
    return loss, gq_full, gz_full, gxi


def unrolled_loss(problem, K: int, rho: float, target, theta0="spread"):
    """Forward value of ``unrolled_loss_and_grad`` (for finite differences)."""
    prep = prepare(problem, "f64")
    orc = MamOracle(prep, rho, theta0=theta0)
    orc.run(K)
    diff = orc.barycenter() - np.asarray(target, dtype=F64)
    return float(np.dot(diff, diff))
