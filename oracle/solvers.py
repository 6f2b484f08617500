"""Reference solvers in FP64: FISTA / ISTA with safe screening over a ladder of dictionaries.

Test infrastructure only (see the package docstring).

``fast_l1`` is Algorithm 1 (FastL1) with Algorithm 2 (SwitchDictionary), taken step by step:
restrict to the preserved set, proximal update with the current approximation, stable
dynamic screening with the sphere of Table I, gap ratio gamma_t and look-ahead estimate K_t,
then the switch.  With a single exact level it is plain FISTA + GAP Safe screening (the
reference solution used for parity).  ``kkt_polish`` and ``brute_force`` compute the
minimiser without iterating, for pins and for exact reference values.

Readings of points the paper leaves open:
* FISTA recursion (cited, never written): t_0 = 1, t+ = (1 + sqrt(1 + 4 t^2)) / 2,
  z+ = x+ + ((t - 1) / t+)(x+ - x); momentum kept across dictionary switches; a rejected
  coordinate is zeroed in x and z.
* The gap and the screening use the point where the gradient is taken (z for FISTA, x for
  ISTA), since Algorithm 1 forms rho~_t = y - A~ x_t from the iterate being updated; the
  returned point is the one whose gap was certified.
* The maxima in the dual scalings run over the preserved set (the reduced problem has the
  same primal and dual solution, so its spheres stay safe).
* delta uses e(x) = sum_j eps_j |x_j|, an upper bound of ||(A - A~) x|| (Theorem 1 only needs one).
* Stopping: only at the exact level, when G(x, theta|A) / ||y||^2 <= tol.
* Rejection when the test value is < 1 - tau (tau = 1e-12 absorbs FP64 rounding).
* K_t: conventional GAP test for the approximate problem (centre theta~, radius sqrt(2 G~)/lam).
"""
from __future__ import annotations

import itertools
from dataclasses import dataclass, field

import numpy as np

from . import lasso as L
from .dictionaries import Level, exact_level, power_iteration_sq_norm

GAP, DST, STATIC = "gap", "dst", "static"
FISTA, ISTA = "fista", "ista"


@dataclass
class Result:
    x: np.ndarray
    gap: float                      # relative gap G / ||y||^2 at the returned point (exact level)
    kept: np.ndarray                # preserved set at exit (sorted)
    iters: int
    converged: bool
    level_trace: list = field(default_factory=list)
    kept_trace: list = field(default_factory=list)
    gamma_trace: list = field(default_factory=list)
    gap_trace: list = field(default_factory=list)
    Kt_trace: list = field(default_factory=list)
    rejected_trace: list = field(default_factory=list)   # (iteration, rejected indices)
    lam: float = 0.0
    lam_max: float = 0.0


def fast_l1(levels: list[Level], anorm: np.ndarray, y: np.ndarray, lam: float, tol: float,
            Gamma: float = 0.5, Lip: float | None = None, algo: str = FISTA, rule: str = GAP,
            screen_every: int = 1, max_iter: int = 100000, tau: float = 1e-12, Aty: np.ndarray | None = None,
            trace: bool = False) -> Result:
    """Algorithm 1 (FastL1) over the ladder ``levels`` (increasing precision, last one exact).

    anorm: exact atom norms ||a_j||_2.  Aty: exact correlations A^T y (computed with the last
    level when not given); they give lambda_max (eq:DefLMax) and the Dynamic Safe test.
    """
    I = len(levels) - 1
    exact = levels[I]
    K = exact.op.K
    y = np.asarray(y, dtype=np.float64)
    yy = float(y @ y)
    if Aty is None:
        Aty = exact.op.rmatvec(y)
    lam_max = L.lambda_max(Aty)
    if lam >= lam_max:
        return Result(np.zeros(K), 0.0, np.zeros(0, dtype=np.int64), 0, True, lam=lam, lam_max=lam_max)
    if Lip is None:
        Lip = max(power_iteration_sq_norm(lev.op) for lev in levels)

    x = np.zeros(K)
    z = np.zeros(K)
    t = 1.0
    kept = np.arange(K)
    i = 0
    res = Result(np.zeros(K), np.inf, kept, 0, False, lam=lam, lam_max=lam_max)
    for it in range(max_iter):
        lev = levels[i]
        point = z if algo == FISTA else x
        pk = point[kept]
        nz = np.flatnonzero(pk)
        # ----- restricted residual and correlations with the current approximation
        rho = y - lev.op.matvec(pk[nz], kept[nz]) if nz.size else y.copy()
        g = lev.op.rmatvec(rho, kept)
        # ----- proximal update of the preserved coefficients (eq:ISTA_update with momentum)
        x_new = L.soft_threshold(pk + g / Lip, lam / Lip)
        if algo == FISTA:
            t_new = 0.5 * (1.0 + np.sqrt(1.0 + 4.0 * t * t))
            z_new = x_new + ((t - 1.0) / t_new) * (x_new - x[kept])
        else:
            t_new, z_new = t, x_new
        # ----- dual points theta' (stable, eq:theta_dynamic_approx) and theta~ (eq:theta_dynamic with A~)
        eps = lev.eps[kept]
        rr = float(rho @ rho)
        yr = float(y @ rho)
        nrho = np.sqrt(rr)
        m_stable = float(np.max(np.abs(g) + eps * nrho)) if kept.size else 0.0
        m_tilde = float(np.max(np.abs(g))) if kept.size else 0.0
        s_p = L.theta_dynamic_coef(yr, rr, lam, m_stable)
        s_t = L.theta_dynamic_coef(yr, rr, lam, m_tilde)
        P = 0.5 * rr + lam * float(np.sum(np.abs(pk)))
        Gp = L.duality_gap(P, L.dual_of_multiple(s_p, yr, rr, lam))
        Gt = L.duality_gap(P, L.dual_of_multiple(s_t, yr, rr, lam))
        e = L.weighted_error_bound(eps, pk)
        delta = L.delta_from_error_bound(nrho, e)
        gamma = L.gap_ratio(Gt, Gp)
        if trace:
            res.level_trace.append(i)
            res.kept_trace.append(kept.size)
            res.gamma_trace.append(gamma)
            res.gap_trace.append(Gp / yy)
        # ----- stopping criterion, evaluated with the exact dictionary only
        if i == I and Gp / yy <= tol:
            out = np.zeros(K)
            out[kept] = pk
            res.x, res.gap, res.kept, res.iters, res.converged = out, Gp / yy, kept.copy(), it, True
            return res
        # ----- dynamic screening (Table I) and look-ahead estimate K_t (eq:DefCardinalEstimated)
        keep_mask = np.ones(kept.size, dtype=bool)
        if (it + 1) % screen_every == 0 and rr > 0.0:
            if rule == GAP:
                Rp = L.stable_gap_radius(Gp, delta, lam)
                mu = L.stable_sphere_test(s_p * g, eps, abs(s_p) * nrho, Rp, anorm[kept])
            elif rule == DST:   # Stable Dynamic Safe with exact a^T y (Table I, fourth row, first form)
                d2 = s_p * s_p * rr - 2.0 * s_p * yr / lam + yy / (lam * lam)
                Rp = float(np.sqrt(max(d2, 0.0)))
                mu = np.abs(Aty[kept]) / lam + Rp * anorm[kept]
            else:   # Static Safe sphere (eq:static_sphere) around y / lam, with the exact a^T y
                _, Rs = L.static_sphere(y, lam, lam_max)
                mu = np.abs(Aty[kept]) / lam + Rs * anorm[kept]
            keep_mask = mu >= 1.0 - tau
        Rt = L.gap_safe_radius(Gt, lam)
        K_t = int(np.count_nonzero(L.sphere_test(s_t * g, Rt, lev.atnorm[kept]) >= 1.0))
        if trace:
            res.Kt_trace.append(K_t)
            res.rejected_trace.append((it, kept[~keep_mask].copy()))
        x[kept] = x_new
        z[kept] = z_new
        rej = kept[~keep_mask]
        x[rej] = 0.0
        z[rej] = 0.0
        kept = kept[keep_mask]
        t = t_new
        # ----- Algorithm 2
        i = L.switch_dictionary(i, I, gamma, Gamma, K_t, lev.rc, K)
    out = np.zeros(K)
    out[kept] = (z if algo == FISTA else x)[kept]
    res.x, res.kept, res.iters = out, kept.copy(), max_iter
    return res


def fista_gap_safe(A: np.ndarray, y: np.ndarray, lam: float, tol: float, **kw) -> Result:
    """Plain FISTA with GAP Safe screening on the exact dictionary (Algorithm 1 with I = 0)."""
    lev = exact_level(np.asarray(A, dtype=np.float64))
    return fast_l1([lev], lev.atnorm, y, lam, tol, **kw)


# ----------------------------------------------------------------------------- exact minimisers

def support_solution(A: np.ndarray, y: np.ndarray, lam: float, S: np.ndarray, s: np.ndarray) -> np.ndarray:
    """x_S solving the stationarity A_S^T (A_S x_S - y) + lam s_S = 0 for a given support and signs."""
    AS = A[:, S]
    return np.linalg.solve(AS.T @ AS, AS.T @ y - lam * s)


def kkt_check(A: np.ndarray, y: np.ndarray, lam: float, x: np.ndarray, tol: float = 1e-9):
    """KKT conditions (Section II): a_j^T theta* = sign(x_j) on the support, |a_j^T theta*| <= 1 off it.

    theta* = (y - A x) / lam.  Returns (ok, support residual, off-support maximum).
    """
    theta = (y - A @ x) / lam
    c = A.T @ theta
    S = np.flatnonzero(x)
    on = float(np.max(np.abs(c[S] - np.sign(x[S])))) if S.size else 0.0
    off_idx = np.setdiff1d(np.arange(A.shape[1]), S)
    off = float(np.max(np.abs(c[off_idx]))) if off_idx.size else 0.0
    return (on <= tol and off <= 1.0 + tol), on, off


def kkt_polish(A: np.ndarray, y: np.ndarray, lam: float, x_approx: np.ndarray, thresh: float = 0.0):
    """Exact minimiser from an approximate one: solve the support system and verify KKT.

    The support and signs are read from ``x_approx`` (entries with |x| > thresh); the closed form
    x_S = (A_S^T A_S)^{-1} (A_S^T y - lam s_S) is the unique Lasso solution iff its signs agree
    and every other atom has |a_j^T (y - A_S x_S)| <= lam.  Returns (x, ok).
    """
    S = np.flatnonzero(np.abs(x_approx) > thresh)
    x = np.zeros(A.shape[1])
    if S.size == 0:
        ok = L.lambda_max(A.T @ y) <= lam
        return x, ok
    s = np.sign(x_approx[S])
    xs = support_solution(A, y, lam, S, s)
    x[S] = xs
    ok_sign = bool(np.all(np.sign(xs) == s))
    ok, _, _ = kkt_check(A, y, lam, x, tol=1e-9)
    return x, (ok and ok_sign)


def kkt_polish_op(op, y: np.ndarray, lam: float, x_approx: np.ndarray, thresh: float = 0.0, tol: float = 1e-9):
    """``kkt_polish`` for a dictionary given as an operator (matvec / rmatvec / col), as the
    structured dictionaries of Section V-A: the support columns are formed explicitly, the KKT
    conditions are checked with the operator's adjoint over all atoms.  Returns (x, ok)."""
    y = np.asarray(y, dtype=np.float64)
    S = np.flatnonzero(np.abs(x_approx) > thresh)
    x = np.zeros(op.K)
    if S.size == 0:
        return x, L.lambda_max(op.rmatvec(y)) <= lam
    s = np.sign(x_approx[S])
    AS = np.stack([op.col(j) for j in S], axis=1)
    xs = np.linalg.solve(AS.T @ AS, AS.T @ y - lam * s)
    x[S] = xs
    c = op.rmatvec((y - AS @ xs) / lam)
    on = float(np.max(np.abs(c[S] - s)))
    off = float(np.max(np.abs(np.delete(c, S)))) if S.size < op.K else 0.0
    return x, bool(np.all(np.sign(xs) == s)) and on <= tol and off <= 1.0 + tol


def brute_force(A: np.ndarray, y: np.ndarray, lam: float) -> np.ndarray:
    """Lasso minimiser by enumerating all 3^K sign patterns (K <= 10, columns in general position).

    For each pattern s in {-1, 0, 1}^K the support system gives a candidate; the minimiser is the
    candidate whose signs match s and whose off-support correlations satisfy |a_j^T r| <= lam.
    Among several valid candidates (degenerate inputs) the one with the smallest objective wins.
    """
    N, K = A.shape
    best, best_obj = np.zeros(K), L.primal(y, np.zeros(K), lam)
    for pattern in itertools.product((-1, 0, 1), repeat=K):
        s = np.array(pattern, dtype=np.float64)
        S = np.flatnonzero(s)
        if S.size == 0 or S.size > N:
            continue
        try:
            xs = support_solution(A, y, lam, S, s[S])
        except np.linalg.LinAlgError:
            continue
        if not np.all(np.sign(xs) == s[S]):
            continue
        x = np.zeros(K)
        x[S] = xs
        r = y - A @ x
        if np.max(np.abs(A.T @ r)) > lam * (1 + 1e-10):
            continue
        obj = L.primal(r, x, lam)
        if obj < best_obj:
            best, best_obj = x, obj
    return best
