"""Pins of the l_p / l_q zone tests, the l_q stable scaling and the dome regions (no GPU).

Each formula of ``oracle.regions`` is checked against something other than itself: extreme
points of the l_q ball (brute force), sampled suprema over zones and regions, the equality
vectors of Hoelder's inequality, the l_2 formulas of ``oracle.lasso``, a numerical constrained
maximisation (scipy), and the solution of the Lasso (safety of the regions)."""
import itertools

import numpy as np
import pytest

import synthetic as S
from oracle import lasso as L
from oracle import regions as G
from oracle import solvers as SV

PS = [1.0, 1.5, 2.0, 3.0, np.inf]
QS = [1.0, 2.0, np.inf]


def _in_ball(rng, center, radius, p, n_pts):
    """Points of B_p(center, radius): random directions scaled to l_p norm <= radius (half on the
    boundary, where suprema are attained)."""
    N = center.size
    u = rng.standard_normal((n_pts, N))
    u /= G.lq_norm(u, p, axis=1)[:, None]
    scale = np.where(np.arange(n_pts) % 2 == 0, 1.0, rng.random(n_pts))
    return center[None, :] + radius * scale[:, None] * u


@pytest.mark.parametrize("N", [3, 5])
@pytest.mark.parametrize("p", PS)
def test_C_pq_against_extreme_points(N, p):
    """sup_{u in B_q(0,1)} ||u||_{p*} is attained at an extreme point of B_q: +-e_i for q = 1,
    sign vectors for q = inf; for q = 2 it is 1 or N^{1/p* - 1/2} (at e_1 or the flat vector),
    and no sampled unit vector exceeds it."""
    ps = G.conjugate(p)
    ext1 = np.eye(N)
    assert np.max(G.lq_norm(ext1, ps, axis=1)) == pytest.approx(G.C_pq(N, p, 1.0), rel=1e-14)
    signs = np.array(list(itertools.product([-1.0, 1.0], repeat=N)))
    assert np.max(G.lq_norm(signs, ps, axis=1)) == pytest.approx(G.C_pq(N, p, np.inf), rel=1e-14)
    rng = np.random.default_rng(N)
    u = rng.standard_normal((4000, N))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    cands = np.vstack([np.eye(N)[:1], np.full((1, N), 1.0 / np.sqrt(N)), u])
    vals = G.lq_norm(cands, ps, axis=1)
    C = G.C_pq(N, p, 2.0)
    assert np.max(vals) <= C * (1 + 1e-12)
    assert max(vals[0], vals[1]) == pytest.approx(C, rel=1e-12)


@pytest.mark.parametrize("p", PS)
def test_lp_sphere_test_sampled_and_attained(p):
    """eq:sphere_test for an l_p sphere: no point of B_p(c, R) exceeds it, and the Hoelder equality
    point c + R u (||u||_p = 1, u^T a = ||a||_{p*}) attains it."""
    rng = np.random.default_rng(int(10 * min(p, 9)))
    N = 6
    for _ in range(5):
        a, c = rng.standard_normal(N), rng.standard_normal(N)
        R = float(rng.random() + 0.1)
        mu = G.sphere_test_lp(a, c, R, p)
        th = _in_ball(rng, c, R, p, 3000)
        assert np.max(np.abs(th @ a)) <= mu * (1 + 1e-12)
        t_star = G.zone_first_term_maximiser(c, R, a, p)
        assert G.lq_norm(t_star - c, p) <= R * (1 + 1e-12)
        assert abs(float(a @ t_star)) == pytest.approx(mu, rel=1e-12)


@pytest.mark.parametrize("p", PS)
@pytest.mark.parametrize("q", QS)
def test_zone_sphere_test_bounds_sampled_pairs(p, q):
    """eq:sphere_test_approx bounds |a^T theta| for every a in B_q(a~, eps) and theta in B_p(c, R);
    its first two terms are attained by an atom of the zone; eps = 0 gives eq:sphere_test."""
    rng = np.random.default_rng(int(7 * min(p, 9) + 3 * min(q, 9)))
    N = 6
    for _ in range(4):
        a_t, c = rng.standard_normal(N), rng.standard_normal(N)
        eps, R = float(0.3 * rng.random()), float(rng.random() + 0.1)
        bound = G.zone_sphere_test(a_t, eps, c, R, p, q)
        atoms = _in_ball(rng, a_t, eps, q, 300)
        thetas = _in_ball(rng, c, R, p, 300)
        assert np.max(np.abs(atoms @ thetas.T)) <= bound * (1 + 1e-12)
        a_star = G.zone_first_term_maximiser(a_t, eps, c, q)
        assert G.lq_norm(a_star - a_t, q) <= eps * (1 + 1e-12)
        assert abs(float(a_star @ c)) == pytest.approx(abs(float(a_t @ c)) + eps * G.lq_norm(c, G.conjugate(q)),
                                                       rel=1e-12)
        assert G.zone_sphere_test(a_t, 0.0, c, R, p, q) == pytest.approx(G.sphere_test_lp(a_t, c, R, p), rel=1e-15)


def test_zone_tests_reduce_to_the_l2_formulas():
    """p = q = 2: the general tests equal the l_2 stable tests of oracle.lasso (C_{2,2} = 1)."""
    rng = np.random.default_rng(0)
    for _ in range(10):
        a_t, c = rng.standard_normal(8), rng.standard_normal(8)
        eps, R, an = 0.2 * rng.random(), rng.random(), 1.0 + rng.random()
        cn = float(np.linalg.norm(c))
        assert G.zone_sphere_test(a_t, eps, c, R, 2.0, 2.0) == pytest.approx(
            float(L.stable_sphere_test_unnormalized(np.array(a_t @ c), eps, cn, R, np.linalg.norm(a_t))), rel=1e-14)
        assert G.zone_sphere_test_normalized(a_t, eps, an, c, R, 2.0) == pytest.approx(
            float(L.stable_sphere_test(np.array(a_t @ c), eps, cn, R, an)), rel=1e-14)


@pytest.mark.parametrize("q", QS)
def test_normalized_zone_test_bounds_atoms_of_known_norm(q):
    """eq:sphere_test_approx_normalized: an atom a with ||a - a~||_q <= eps and ||a||_{p*} = a_pstar
    (p = 2) never tests above it on the sphere."""
    rng = np.random.default_rng(5)
    N = 7
    for _ in range(6):
        a = rng.standard_normal(N)
        a_t = a + 0.1 * rng.standard_normal(N)
        eps = float(G.lq_norm(a - a_t, q))
        c = rng.standard_normal(N)
        R = float(rng.random())
        bound = G.zone_sphere_test_normalized(a_t, eps, float(np.linalg.norm(a)), c, R, q)
        thetas = _in_ball(rng, c, R, 2.0, 4000)
        assert np.max(np.abs(thetas @ a)) <= bound * (1 + 1e-12)
        assert G.sphere_test_lp(a, c, R, 2.0) <= bound * (1 + 1e-12)


@pytest.mark.parametrize("q", QS)
def test_lemma2_with_lq_errors_gives_feasible_dual_points(q):
    """alpha z with alpha = 1 / max(1, max_j |a~_j^T z| + eps_j ||z||_{q*}) is feasible for A and A~
    when eps_j = ||a~_j - a_j||_q (Lemma 2, general q)."""
    rng = np.random.default_rng(11)
    N, K = 20, 60
    for trial in range(8):
        A = rng.standard_normal((N, K))
        A /= np.linalg.norm(A, axis=0)
        At = A + (0.02 + 0.1 * trial / 8) * rng.standard_normal((N, K))
        eps = G.error_columns_lq(At, A, q)
        z = 3.0 * rng.standard_normal(N)
        alpha = G.stable_scaling_q(At.T @ z, eps, z, q)
        th = alpha * z
        assert np.max(np.abs(A.T @ th)) <= 1 + 1e-12
        assert np.max(np.abs(At.T @ th)) <= 1 + 1e-12
    # adversarial errors that attain Hoelder's bound: a_j = a~_j + s_j eps_j u with u^T z = ||z||_{q*}
    # and s_j the sign of a_j^T z, so |a_j^T z| = |a~_j^T z| + eps_j ||z||_{q*} and the scaled point
    # touches the boundary of the feasible set (any smaller scaling denominator leaves it)
    A = rng.standard_normal((N, K))
    z = rng.standard_normal(N)
    if np.isinf(q):
        u = np.sign(z)
    elif q == 1.0:
        u = np.zeros(N)
        k = int(np.argmax(np.abs(z)))
        u[k] = np.sign(z[k])
    else:
        u = z / np.linalg.norm(z)
    zq = float(u @ z)
    s = np.sign(A.T @ z)
    eps = 0.5 * np.abs(A.T @ z) / zq * rng.random(K)
    At = A - (s * eps)[None, :] * u[:, None]
    np.testing.assert_allclose(G.error_columns_lq(At, A, q), eps, rtol=1e-9)
    th = G.stable_scaling_q(At.T @ z, eps, z, q) * z
    assert np.max(np.abs(A.T @ th)) == pytest.approx(1.0, rel=1e-12)


@pytest.mark.parametrize("q", QS)
def test_error_bound_q_dominates_the_true_error(q):
    """e(x) from l_q errors bounds ||(A - A~) x||_2; for q = 2 it is sum_j eps_j |x_j|."""
    rng = np.random.default_rng(13)
    N, K = 16, 40
    A = rng.standard_normal((N, K))
    At = A + 0.05 * rng.standard_normal((N, K))
    eps = G.error_columns_lq(At, A, q)
    for _ in range(20):
        x = rng.standard_normal(K) * (rng.random(K) < 0.3)
        assert np.linalg.norm((A - At) @ x) <= G.error_bound_q(eps, x, N, q) * (1 + 1e-12) + 1e-15
    x = rng.standard_normal(K)
    if q == 2.0:
        assert G.error_bound_q(eps, x, N, q) == pytest.approx(L.weighted_error_bound(eps, x), rel=1e-12)


def test_dome_max_matches_constrained_maximisation():
    """The closed form of max a^T theta over a dome against scipy's SLSQP from several starts and
    against sampled points of the dome; the dome never tests above its sphere and equals it when
    the half-space does not cut the sphere's maximiser."""
    from scipy.optimize import minimize
    rng = np.random.default_rng(17)
    N = 4
    for trial in range(12):
        a, c, n = rng.standard_normal(N), rng.standard_normal(N), rng.standard_normal(N)
        R = float(rng.random() + 0.3)
        psi = float(n @ c) + (rng.random() * 1.6 - 0.8) * R * np.linalg.norm(n)   # the plane cuts the ball
        closed = G.dome_max(a, c, R, n, psi)
        cons = [{"type": "ineq", "fun": lambda t: R * R - float((t - c) @ (t - c))},
                {"type": "ineq", "fun": lambda t: psi - float(n @ t)}]
        best = -np.inf
        for _ in range(6):
            x0 = c + 0.1 * R * rng.standard_normal(N)
            r = minimize(lambda t: -float(a @ t), x0, constraints=cons, method="SLSQP",
                         options={"ftol": 1e-14, "maxiter": 500})
            if r.success:
                best = max(best, -r.fun)
        assert best == pytest.approx(closed, rel=1e-6, abs=1e-6)
        pts = _in_ball(rng, c, R, 2.0, 20000)
        pts = pts[pts @ n <= psi]
        assert np.max(pts @ a) <= closed + 1e-12
        assert G.dome_test(a, c, R, n, psi) <= G.sphere_test_lp(a, c, R, 2.0) * (1 + 1e-12)
    a, c, n = rng.standard_normal(N), rng.standard_normal(N), rng.standard_normal(N)
    far = float(n @ c) + 10.0 * np.linalg.norm(n)
    assert G.dome_test(a, c, 1.0, n, far) == pytest.approx(G.sphere_test_lp(a, c, 1.0, 2.0), rel=1e-14)


@pytest.mark.parametrize("seed", range(3))
def test_gap_dome_is_safe_and_rejects_at_least_the_sphere(seed):
    """The GAP sphere of an iterate, cut by the most correlated atom's dual constraint, contains
    theta*; every atom the dome test rejects is zero in x*, and the dome rejects every atom the
    sphere rejects.  The stable dome test bounds approximate atoms of the zone B_2(a~, eps)."""
    w = S.dense_small(N=30, K=90, n_signals=3, seed=20 + seed)
    A, y = w.A, w.Y[seed]
    lam = 0.3 * L.lambda_max(A.T @ y)
    ref = SV.fista_gap_safe(A, y, lam, 1e-14, max_iter=400000)
    xs, ok = SV.kkt_polish(A, y, lam, ref.x)
    assert ok
    theta_star = (y - A @ xs) / lam
    for it in (20, 60, 200):
        x = SV.fista_gap_safe(A, y, lam, 0.0, max_iter=it).x
        rho = y - A @ x
        s = L.theta_dynamic_coef(float(y @ rho), float(rho @ rho), lam, float(np.max(np.abs(A.T @ rho))))
        c = s * rho
        Gap = L.primal(rho, x, lam) - L.dual_of_multiple(s, float(y @ rho), float(rho @ rho), lam)
        R = L.gap_safe_radius(Gap, lam)
        n, psi = G.gap_dome(c, R, A)
        assert np.linalg.norm(theta_star - c) <= R * (1 + 1e-9) + 1e-12
        assert float(n @ theta_star) <= psi + 1e-12
        mu_dome = np.array([G.dome_test(A[:, j], c, R, n, psi) for j in range(A.shape[1])])
        mu_sph = np.array([G.sphere_test_lp(A[:, j], c, R, 2.0) for j in range(A.shape[1])])
        assert np.all(mu_dome <= mu_sph * (1 + 1e-12))
        rej = np.flatnonzero(mu_dome < 1.0)
        assert np.all(xs[rej] == 0.0)
        assert set(np.flatnonzero(mu_sph < 1.0)) <= set(rej.tolist())
    rng = np.random.default_rng(seed)
    for j in range(5):
        a_t = A[:, j] + 0.05 * rng.standard_normal(A.shape[0])
        eps = float(np.linalg.norm(a_t - A[:, j]))
        atoms = _in_ball(rng, a_t, eps, 2.0, 200)
        thetas = _in_ball(rng, c, R, 2.0, 4000)
        thetas = thetas[thetas @ n <= psi]
        assert np.max(np.abs(atoms @ thetas.T)) <= G.stable_dome_test(a_t, eps, c, R, n, psi) * (1 + 1e-12)
