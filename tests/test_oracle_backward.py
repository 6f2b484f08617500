"""Pins of the oracle's solution derivative against central finite differences (no GPU)."""
import numpy as np

from oracle import backward as B
from oracle import lasso as L
from oracle import solvers as SV


def _stable_instance(seed):
    """Small instance whose support is stable under 1e-4 perturbations (large |x_S|, KKT slack)."""
    r = np.random.default_rng(500 + seed)
    for _ in range(200):
        A = r.standard_normal((30, 60))
        A /= np.linalg.norm(A, axis=0)
        x0 = np.zeros(60)
        idx = r.choice(60, 5, replace=False)
        x0[idx] = r.standard_normal(5) * 2
        y = A @ x0 + 0.1 * r.standard_normal(30)
        lam = 0.4 * L.lambda_max(A.T @ y)
        x = B.solve_exact(A, y, lam)
        S = np.flatnonzero(x)
        theta = (y - A @ x) / lam
        slack = 1 - np.max(np.abs(np.delete(A.T @ theta, S)))
        if S.size and np.min(np.abs(x[S])) > 1e-2 and slack > 1e-2:
            xt = np.zeros(60)
            xt[r.choice(60, 4, replace=False)] = r.standard_normal(4)
            return A, y, lam, x, xt
    raise RuntimeError("no stable instance")


def test_adjoint_matches_central_differences():
    for seed in range(2):
        A, y, lam, x, xt = _stable_instance(seed)
        _, g = B.target_loss(x, xt)
        dy, dA = B.support_adjoint(A, y, x, g)
        r = np.random.default_rng(seed)
        for n in r.choice(30, 6, replace=False):
            fd = B.finite_difference(A, y, lam, xt, "y", n)
            assert abs(fd - dy[n]) <= 1e-6 * max(1.0, abs(dy[n]))
        S = np.flatnonzero(x)
        cols = list(S[:3]) + list(r.choice(np.setdiff1d(np.arange(60), S), 2, replace=False))
        for j in cols:
            n = int(r.integers(30))
            fd = B.finite_difference(A, y, lam, xt, "A", (n, j))
            assert abs(fd - dA[n, j]) <= 1e-6 * max(1.0, abs(dA[n, j]))


def test_adjoint_zero_when_solution_is_zero():
    A, y, lam, x, xt = _stable_instance(0)
    lam_big = 1.01 * L.lambda_max(A.T @ y)
    x0 = SV.fista_gap_safe(A, y, lam_big, 1e-12).x
    dy, dA = B.support_adjoint(A, y, x0, np.ones(60))
    assert np.all(dy == 0) and np.all(dA == 0)
