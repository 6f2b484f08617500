"""General zones and safe regions for (stable) screening tests, in FP64.

Test infrastructure only (see the package docstring).

* l_p spheres and l_q error balls (Section III-B, eq:sphere_test, eq:sphere_test_approx,
  eq:sphere_test_approx_normalized and their proof in the appendix on the stable sphere test):
  an atom known only to lie in the zone B_q(a~, eps) is tested against a safe region
  B_p(c, R) with the dual norms ||.||_{p*}, ||.||_{q*} and the constant C_{p,q}.
* the stable dual scaling of Lemma 2 with the error measured in l_q: theta = alpha z with
  alpha <= 1 / max_j (|a~_j^T z| + eps_j ||z||_{q*}).
* an upper bound of ||(A - A~) x||_2 from per-atom l_q errors (the e(x) that enters delta in
  Theorem 1), through ||v||_2 <= N^{(1/2 - 1/q)+} ||v||_q.
* dome regions: a sphere cut by one half-space (the paper names dome tests as another safe
  region the stable framework applies to).  Any constraint of the dual feasible set,
  s a_k^T theta <= 1, holds at theta*, so it cuts a safe sphere into a safe dome.

Norm exponents are floats in [1, inf]; ``np.inf`` stands for the max norm.
"""
from __future__ import annotations

import numpy as np


def conjugate(p: float) -> float:
    """p* with 1/p + 1/p* = 1 (1 <-> inf)."""
    if p == 1.0:
        return np.inf
    if np.isinf(p):
        return 1.0
    return p / (p - 1.0)


def lq_norm(v: np.ndarray, q: float, axis=None) -> np.ndarray:
    """||v||_q (along `axis`)."""
    v = np.abs(np.asarray(v, dtype=np.float64))
    if np.isinf(q):
        return np.max(v, axis=axis)
    return np.sum(v ** q, axis=axis) ** (1.0 / q)


def C_pq(N: int, p: float, q: float) -> float:
    """C_{p,q} = sup_{u in B_q(0, 1)} ||u||_{p*} = N^{(1/p* - 1/q)+} (Hoelder), the constant of
    eq:sphere_test_approx; 1/p* = 1 - 1/p."""
    inv_pstar = 1.0 - (0.0 if np.isinf(p) else 1.0 / p)
    inv_q = 0.0 if np.isinf(q) else 1.0 / q
    return float(N) ** max(inv_pstar - inv_q, 0.0)


def sphere_test_lp(a: np.ndarray, c: np.ndarray, R: float, p: float) -> float:
    """mu(a | B_p(c, R)) = sup_{theta in B_p(c, R)} |a^T theta| = |a^T c| + R ||a||_{p*}
    (eq:sphere_test)."""
    return abs(float(a @ c)) + R * float(lq_norm(a, conjugate(p)))


def zone_sphere_test(a_t: np.ndarray, eps: float, c: np.ndarray, R: float, p: float, q: float) -> float:
    """Upper bound of sup_{a in B_q(a~, eps)} mu(a | B_p(c, R)) (eq:sphere_test_approx):
    |a~^T c| + eps ||c||_{q*} + R ||a~||_{p*} + C_{p,q} R eps."""
    N = a_t.size
    return (abs(float(a_t @ c)) + eps * float(lq_norm(c, conjugate(q))) + R * float(lq_norm(a_t, conjugate(p)))
            + C_pq(N, p, q) * R * eps)


def zone_sphere_test_normalized(a_t: np.ndarray, eps: float, a_pstar: float, c: np.ndarray, R: float,
                                q: float) -> float:
    """The same test when ||a||_{p*} = a_pstar is known (eq:sphere_test_approx_normalized):
    |a~^T c| + eps ||c||_{q*} + R a_pstar."""
    return abs(float(a_t @ c)) + eps * float(lq_norm(c, conjugate(q))) + R * a_pstar


def zone_first_term_maximiser(a_t: np.ndarray, eps: float, c: np.ndarray, q: float) -> np.ndarray:
    """An atom a in B_q(a~, eps) attaining sup |a^T c| = |a~^T c| + eps ||c||_{q*}: a = a~ + eps u
    with u in B_q(0, 1), sign(a~^T c) u^T c = ||c||_{q*} (the equality case of Hoelder)."""
    s = 1.0 if float(a_t @ c) >= 0.0 else -1.0
    qs = conjugate(q)
    if np.isinf(q):                      # u = sign(c): u^T c = ||c||_1
        u = np.sign(c)
    elif q == 1.0:                       # u = sign(c_k) e_k at the largest |c_k|
        u = np.zeros_like(c)
        k = int(np.argmax(np.abs(c)))
        u[k] = np.sign(c[k])
    else:                                # u_i = sign(c_i) |c_i|^{q*-1} / ||c||_{q*}^{q*-1}
        nrm = float(lq_norm(c, qs))
        u = np.sign(c) * np.abs(c) ** (qs - 1.0) / (nrm ** (qs - 1.0) if nrm > 0 else 1.0)
    return a_t + s * eps * u


def stable_scaling_q(Atz: np.ndarray, eps: np.ndarray, z: np.ndarray, q: float) -> float:
    """alpha = 1 / max(1, max_j (|a~_j^T z| + eps_j ||z||_{q*})) (Lemma 2 with l_q errors): alpha z is
    dual feasible for A and for A~ when ||a~_j - a_j||_q <= eps_j."""
    m = float(np.max(np.abs(Atz) + eps * float(lq_norm(z, conjugate(q)))))
    return 1.0 / max(1.0, m)


def error_columns_lq(approx_cols: np.ndarray, exact_cols: np.ndarray, q: float) -> np.ndarray:
    """eps_j = ||a~_j - a_j||_q for every column (FP64), inflated by 1e-12 to stay an upper bound."""
    return lq_norm(np.asarray(approx_cols) - np.asarray(exact_cols), q, axis=0) * (1.0 + 1e-12)


def error_bound_q(eps: np.ndarray, x: np.ndarray, N: int, q: float) -> float:
    """e(x) >= ||(A - A~) x||_2 from l_q errors: sum_j |x_j| ||a_j - a~_j||_2 and
    ||v||_2 <= N^{(1/2 - 1/q)+} ||v||_q."""
    inv_q = 0.0 if np.isinf(q) else 1.0 / q
    return float(N) ** max(0.5 - inv_q, 0.0) * float(np.sum(eps * np.abs(x)))


# ----------------------------------------------------------------------------- domes

def dome_max(a: np.ndarray, c: np.ndarray, R: float, n: np.ndarray, psi: float) -> float:
    """max a^T theta over the dome {||theta - c||_2 <= R, n^T theta <= psi} (nonempty).

    With v = theta - c and d = psi - n^T c: the sphere's maximiser v = R a/||a|| is kept when
    n^T v <= d; otherwise both constraints are active at the optimum, v = (d/||n||) n^ + w with
    w orthogonal to n^ and ||w||^2 = R^2 - (d/||n||)^2, and w points along the part of a
    orthogonal to n^.
    """
    an = float(np.linalg.norm(a))
    nn = float(np.linalg.norm(n))
    d = psi - float(n @ c)
    base = float(a @ c)
    if an == 0.0:
        return base
    if R * float(n @ a) / an <= d:
        return base + R * an
    nh = n / nn
    alpha = float(a @ nh)
    a_perp = a - alpha * nh
    h = d / nn                              # signed offset of the cutting plane from c
    if h < -R:
        raise ValueError("empty dome")
    return base + alpha * h + float(np.linalg.norm(a_perp)) * float(np.sqrt(max(R * R - h * h, 0.0)))


def dome_test(a: np.ndarray, c: np.ndarray, R: float, n: np.ndarray, psi: float) -> float:
    """mu(a | dome) = sup |a^T theta| over the dome = max(dome_max(a), dome_max(-a))."""
    return max(dome_max(a, c, R, n, psi), dome_max(-a, c, R, n, psi))


def stable_dome_test(a_t: np.ndarray, eps: float, c: np.ndarray, R: float, n: np.ndarray, psi: float) -> float:
    """sup over a in B_2(a~, eps) of mu(a | dome) <= mu(a~ | dome) + eps sup_{theta in dome} ||theta||_2
    <= mu(a~ | dome) + eps (||c||_2 + R)."""
    return dome_test(a_t, c, R, n, psi) + eps * (float(np.linalg.norm(c)) + R)


def gap_dome(c: np.ndarray, R: float, A_exact: np.ndarray):
    """A safe dome from a safe sphere B_2(c, R): the half-space s a_k^T theta <= 1 of the exact
    atom with the largest |a_k^T c| (s its sign) is a constraint of the dual feasible set, so it
    holds at theta*.  Returns (n, psi)."""
    g = A_exact.T @ c
    k = int(np.argmax(np.abs(g)))
    s = 1.0 if g[k] >= 0.0 else -1.0
    return s * A_exact[:, k], 1.0
