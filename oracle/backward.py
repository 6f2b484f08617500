"""Derivative of the Lasso solution x*(y, A) in FP64 (the differentiation pattern).

Test infrastructure only (see the package docstring).  The paper does not differentiate
the solution; this follows from its KKT conditions (Section II): on the support S with signs
s, A_S^T (A_S x_S - y) + lam s = 0, so for a fixed sign pattern x_S = M^{-1}(A_S^T y - lam s)
with M = A_S^T A_S, and x is zero off S.  For a loss with gradient g = dL/dx:

    u = M^{-1} g_S,   dL/dy = A_S u,   dL/dA_S = r u^T - (A_S u) x_S^T   (r = y - A_S x_S),

and dL/dA is zero outside the columns of S.  ``finite_difference`` re-solves the problem to
machine precision (support system + KKT check) at perturbed inputs to pin these formulas.
"""
from __future__ import annotations

import numpy as np

from .solvers import fista_gap_safe, kkt_polish


def support_adjoint(A: np.ndarray, y: np.ndarray, x: np.ndarray, g: np.ndarray):
    """(dL/dy, dL/dA) at the solution x for the loss gradient g = dL/dx."""
    S = np.flatnonzero(x)
    dy = np.zeros(A.shape[0])
    dA = np.zeros_like(A, dtype=np.float64)
    if S.size == 0:
        return dy, dA
    AS = A[:, S]
    u = np.linalg.solve(AS.T @ AS, g[S])
    Au = AS @ u
    r = y - AS @ x[S]
    dy = Au
    dA[:, S] = np.outer(r, u) - np.outer(Au, x[S])
    return dy, dA


def solve_exact(A, y, lam, tol=1e-13):
    """Lasso minimiser to machine precision: FISTA + GAP Safe, then the KKT-verified support system."""
    r = fista_gap_safe(A, y, lam, tol)
    x, ok = kkt_polish(A, y, lam, r.x)
    if not ok:
        raise RuntimeError("KKT polish failed; support not identified")
    return x


def target_loss(x, x_target):
    """L = ||x - x_target||^2 and its gradient 2 (x - x_target)."""
    d = x - x_target
    return float(d @ d), 2.0 * d


def finite_difference(A, y, lam, x_target, which: str, index, h: float = 1e-4, support=None):
    """Central difference of L(x*(y, A)) in one coordinate of y ('y', n) or of A ('A', (n, j)).

    lam is held fixed (absolute).  ``support`` = (S, signs) fixes the sign pattern so that both
    evaluations use the same support system (valid while the perturbation keeps it).
    """
    def loss_at(Ap, yp):
        if support is None:
            x = solve_exact(Ap, yp, lam)
        else:
            S, s = support
            AS = Ap[:, S]
            x = np.zeros(Ap.shape[1])
            x[S] = np.linalg.solve(AS.T @ AS, AS.T @ yp - lam * s)
        return target_loss(x, x_target)[0]

    Ap, Am = A.copy(), A.copy()
    yp, ym = y.copy(), y.copy()
    if which == "y":
        yp[index] += h
        ym[index] -= h
    else:
        Ap[index] += h
        Am[index] -= h
    return (loss_at(Ap, yp) - loss_at(Am, ym)) / (2.0 * h)
