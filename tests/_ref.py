"""Oracle-side reference values for the GPU parity tests (all computed by ``oracle/``)."""
import numpy as np

from oracle import lasso as OL
from oracle import solvers as OS


def exact_solution(A, y, lam, tol=1e-14):
    """Minimiser to machine precision: oracle FISTA + GAP Safe, then the KKT-verified support system."""
    r = OS.fista_gap_safe(A, y, lam, tol, max_iter=400000)
    x, ok = OS.kkt_polish(A, y, lam, r.x)
    assert ok, "oracle polish failed"
    return x


def true_rel_gap(A, y, lam, x):
    """G(x, theta(x)|A) / ||y||^2 in FP64 with the dynamic dual point of eq:theta_dynamic (all atoms)."""
    rho = y - A @ x
    s = OL.theta_dynamic_coef(float(y @ rho), float(rho @ rho), lam, float(np.max(np.abs(A.T @ rho))))
    G = OL.primal(rho, x, lam) - OL.dual_of_multiple(s, float(y @ rho), float(rho @ rho), lam)
    return G / float(y @ y)


def check_solution(A, y, lam, x, xs, gap_gpu, tol, kept=None, x_rtol=None):
    """Parity of a GPU solution with the oracle minimiser xs at tolerance tol.

    * the oracle's FP64 gap of x (full dictionary) is <= tol (up to FP64 rounding) and <= the
      GPU's certificate (which upper-bounds it);
    * ||A (x - x*)||^2 <= 2 G ||y||^2 (P(x) - P* >= 1/2 ||A (x - x*)||^2);
    * safety: the GPU preserved set contains the support of x*;
    * optionally ||x - x*|| <= x_rtol ||x*||.
    """
    yy = float(y @ y)
    g = true_rel_gap(A, y, lam, x)
    assert g <= tol * (1 + 1e-6) + 1e-13, (g, tol)
    assert g <= gap_gpu * (1 + 1e-6) + 1e-13, (g, gap_gpu)
    assert np.linalg.norm(A @ (x - xs)) ** 2 <= 2 * (g + 1e-13) * yy
    if kept is not None:
        assert set(np.flatnonzero(xs).tolist()) <= set(np.asarray(kept).tolist())
    if x_rtol is not None:
        assert np.linalg.norm(x - xs) <= x_rtol * max(np.linalg.norm(xs), 1e-300), \
            np.linalg.norm(x - xs) / np.linalg.norm(xs)
