"""The Lasso problem, its dual, dual scalings and (stable) safe sphere tests, in FP64.

Test infrastructure only (see the package docstring).  Each function states the
passage of the paper it writes out.  Vectors are numpy float64 arrays; ``g`` always
denotes correlations of (approximate) atoms with a residual, so that dictionary
products are done by the caller and these functions stay scalar/vector formulas.
"""
from __future__ import annotations

import numpy as np


def lambda_max(Aty: np.ndarray) -> float:
    """lambda_max = ||A^T y||_inf (eq:DefLMax); above it x* = 0 is the unique solution."""
    return float(np.max(np.abs(Aty)))


def soft_threshold(v: np.ndarray, u: float) -> np.ndarray:
    """ST_u(v) = sign(v) (|v| - u)_+, the proximal operator of u||.||_1 (Section I-B)."""
    return np.sign(v) * np.maximum(np.abs(v) - u, 0.0)


def primal(rho: np.ndarray, x: np.ndarray, lam: float) -> float:
    """P(x|A) = 1/2 ||A x - y||^2 + lam ||x||_1 given the residual rho = y - A x (eq:lasso)."""
    return 0.5 * float(rho @ rho) + lam * float(np.sum(np.abs(x)))


def dual(theta: np.ndarray, y: np.ndarray, lam: float) -> float:
    """D(theta) = 1/2 ||y||^2 - lam^2/2 ||theta - y/lam||^2 (eq:lasso_dual)."""
    d = theta - y / lam
    return 0.5 * float(y @ y) - 0.5 * lam * lam * float(d @ d)


def dual_of_multiple(s: float, yr: float, rr: float, lam: float) -> float:
    """D(s rho) expanded in the scalars yr = y^T rho, rr = ||rho||^2.

    D(s rho) = 1/2||y||^2 - 1/2||lam s rho - y||^2 = lam s yr - lam^2 s^2 rr / 2.
    """
    return lam * s * yr - 0.5 * lam * lam * s * s * rr


def duality_gap(P: float, D: float) -> float:
    """G(x, theta|A) = P(x|A) - D(theta) (eq:duality_gap)."""
    return P - D


def dual_scaling(z: np.ndarray, Atz: np.ndarray) -> np.ndarray:
    """Theta(z|A) = z / max(1, ||A^T z||_inf) (eq:conditional_dual_scaling)."""
    return z / max(1.0, float(np.max(np.abs(Atz))))


def stable_dual_scaling(z: np.ndarray, Attz: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """Theta'(z|A~, eps) = z / max(1, max_j |a~_j^T z| + eps_j ||z||_2) (eq:conditional_dual_scaling_modified, q = 2)."""
    return z / max(1.0, float(np.max(np.abs(Attz) + eps * np.linalg.norm(z))))


def projection_coefficient(y: np.ndarray, z: np.ndarray, lam: float) -> float:
    """beta with proj_z(y/lam) = beta z, beta = y^T z / (lam ||z||^2) (Proposition 1)."""
    return float(y @ z) / (lam * float(z @ z))


def clip(v: float, a: float, b: float) -> float:
    """[v]_a^b = min(max(v, a), b) (eq:theta_dynamic)."""
    return min(max(v, a), b)


def theta_dynamic_coef(yr: float, rr: float, lam: float, m: float) -> float:
    """Coefficient s of theta = s rho in eq:theta_dynamic / eq:theta_dynamic_approx.

    s = [y^T rho / (lam ||rho||^2)] clipped to [-1/m, 1/m], where m = ||A^T rho||_inf for the
    dynamic point (eq:theta_dynamic) or m = max_j(|a~_j^T rho| + eps_j ||rho||) for the stable
    one (eq:theta_dynamic_approx).  rho = 0 gives s = 0 (theta = 0 is feasible).
    """
    if rr <= 0.0:
        return 0.0
    beta = yr / (lam * rr)
    if m <= 0.0:
        return beta
    return clip(beta, -1.0 / m, 1.0 / m)


def sphere_test(atc: np.ndarray, R: float, anorm: np.ndarray) -> np.ndarray:
    """mu(a|B(c, R)) = |a^T c| + R ||a||_2 (eq:sphere_test, p = 2)."""
    return np.abs(atc) + R * anorm


def stable_sphere_test(attc: np.ndarray, eps: np.ndarray, cnorm: float, R: float, anorm: np.ndarray) -> np.ndarray:
    """mu(S'|B(c, R)) = |a~^T c| + eps ||c||_2 + R ||a||_2 (eq:sphere_test_approx_normalized, p = q = 2)."""
    return np.abs(attc) + eps * cnorm + R * anorm


def stable_sphere_test_unnormalized(attc, eps, cnorm, R, atnorm, C=1.0):
    """Upper bound |a~^T c| + eps ||c|| + R ||a~|| + C R eps (eq:sphere_test_approx; C_{2,2} = 1)."""
    return np.abs(attc) + eps * cnorm + R * atnorm + C * R * eps


def gap_safe_radius(G: float, lam: float) -> float:
    """R = sqrt(2 G) / lam (eq:GAP_sphere)."""
    return float(np.sqrt(max(2.0 * G, 0.0))) / lam


def delta_theorem1(rho_norm: float, E: float, x_r_norm: float) -> float:
    """delta(x) = ||y - A~ x|| E ||x||_r + 1/2 E^2 ||x||_r^2 (eq:DefDelta), E >= ||A - A~||_{r->2}."""
    return rho_norm * E * x_r_norm + 0.5 * E * E * x_r_norm * x_r_norm


def delta_from_error_bound(rho_norm: float, e: float) -> float:
    """delta for any e >= ||(A - A~) x||_2: ||rho|| e + e^2 / 2.

    Theorem 1 only uses E ||x||_r as an upper bound of ||(A - A~) x||_2, so any such bound
    keeps the sphere safe; with r = 1 and E = max_j eps_j it is eq:DefDelta itself.
    """
    return rho_norm * e + 0.5 * e * e


def weighted_error_bound(eps: np.ndarray, x: np.ndarray) -> float:
    """e(x) = sum_j eps_j |x_j| >= ||(A - A~) x||_2 (triangle inequality over the atoms)."""
    return float(np.sum(eps * np.abs(x)))


def stable_gap_radius(Gp: float, delta: float, lam: float) -> float:
    """R' = sqrt(2 G(x, theta'|A~) + 2 delta(x)) / lam (Theorem 1, eq:GAP_sphere_extended)."""
    return float(np.sqrt(max(2.0 * Gp + 2.0 * delta, 0.0))) / lam


def gap_ratio(G_tilde: float, G_prime: float) -> float:
    """gamma_t = G(x, theta~|A~) / G(x, theta'|A~) (eq:DefRatioSwitch); 0 when G' <= 0."""
    if G_prime <= 0.0:
        return 0.0
    return G_tilde / G_prime


def switch_dictionary(i: int, I: int, gamma: float, Gamma: float, K_t: int, rc_i: float, K: int) -> int:
    """Algorithm 2: speed criterion (K_t <= RC_i K) -> I, convergence (gamma <= Gamma) -> i + 1, else i."""
    if i >= I:
        return I
    if K_t <= rc_i * K:
        return I
    if gamma <= Gamma:
        return i + 1
    return i


def static_sphere(y: np.ndarray, lam: float, lam_max: float):
    """Static Safe sphere: c = y / lam, R = |1/lam_max - 1/lam| ||y|| (eq:static_sphere)."""
    return y / lam, abs(1.0 / lam_max - 1.0 / lam) * float(np.linalg.norm(y))


def stable_lambda_max(Atty: np.ndarray, eps: np.ndarray, ynorm: float) -> float:
    """lambda'_max = max_j |a~_j^T y| + eps_j ||y|| >= lambda_max (eq:DefStableLMax)."""
    return float(np.max(np.abs(Atty) + eps * ynorm))
