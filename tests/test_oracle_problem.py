"""Pins of the FP64 oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: a closed form, brute
force over all sign patterns, the lemmas and theorem of Section III, or a grid search.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import lasso as L
from oracle import dictionaries as D
from oracle import solvers as SV


def _rng(k):
    return np.random.default_rng(1000 + k)


def _small_problem(N, K, seed, ratio):
    r = _rng(seed)
    A = r.standard_normal((N, K))
    A /= np.linalg.norm(A, axis=0)
    x0 = np.zeros(K)
    idx = r.choice(K, size=max(1, K // 8), replace=False)
    x0[idx] = r.standard_normal(idx.size)
    y = A @ x0 + 0.05 * r.standard_normal(N)
    lam = ratio * L.lambda_max(A.T @ y)
    return A, y, lam


# ----------------------------------------------------------------------------- whole solve

def test_lambda_above_lambda_max_gives_zero():
    """eq:DefLMax: lam >= lambda_max  =>  x* = 0 exactly; just below, x* != 0."""
    w = S.c1()
    A, y = w.A, w.Y[0]
    lm = L.lambda_max(A.T @ y)
    r = SV.fista_gap_safe(A, y, lm * (1 + 1e-12), 1e-10)
    assert r.converged and np.all(r.x == 0.0) and r.gap == 0.0
    r = SV.fista_gap_safe(A, y, lm, 1e-10)
    assert np.all(r.x == 0.0)
    r = SV.fista_gap_safe(A, y, lm * 0.99, 1e-12)
    assert np.count_nonzero(r.x) >= 1


def test_orthonormal_dictionary_is_soft_threshold():
    """With orthonormal atoms the Lasso separates: x* = ST_lam(A^T y) (eq:lasso, Section I-B)."""
    Q, y = S.orthonormal_case(64)
    lam = 0.3 * L.lambda_max(Q.T @ y)
    r = SV.fista_gap_safe(Q, y, lam, 1e-15, max_iter=5000)
    ref = np.sign(Q.T @ y) * np.maximum(np.abs(Q.T @ y) - lam, 0.0)
    np.testing.assert_allclose(r.x, ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("ratio", [0.15, 0.5, 0.85])
def test_brute_force_sign_enumeration(seed, ratio):
    """Brute force over all 3^K sign patterns (K = 8) matches the FISTA + GAP Safe oracle."""
    A, y, lam = _small_problem(12, 8, seed, ratio)
    xb = SV.brute_force(A, y, lam)
    r = SV.fista_gap_safe(A, y, lam, 1e-15, max_iter=200000)
    assert r.converged
    # P(x) - P* >= 1/2 ||A (x - x*)||^2 bounds the raw iterate by its certified gap ...
    # (the FP64 gap carries an absolute rounding error of a few ulps of ||y||^2)
    assert np.linalg.norm(A @ (r.x - xb)) ** 2 <= 2 * (max(r.gap, 0.0) + 1e-14) * (y @ y)
    # ... and its support system reproduces the enumerated minimiser to rounding
    xp, ok = SV.kkt_polish(A, y, lam, r.x)
    assert ok
    np.testing.assert_allclose(xp, xb, rtol=0, atol=1e-10)


def test_c1_kkt_and_gap():
    """The c1 reference solution meets KKT to 1e-9 and its certified gap tends to zero."""
    w = S.c1()
    A, y = w.A, w.Y[0]
    lam = 0.5 * L.lambda_max(A.T @ y)
    r = SV.fista_gap_safe(A, y, lam, 1e-13, max_iter=100000)
    assert r.converged and r.gap <= 1e-13
    ok, on, off = SV.kkt_check(A, y, lam, r.x, tol=1e-6)
    assert ok
    xp, okp = SV.kkt_polish(A, y, lam, r.x)
    assert okp
    ok, on, off = SV.kkt_check(A, y, lam, xp, tol=1e-9)
    assert ok and on <= 1e-9 and off < 1.0
    # ||A (x - x*)||^2 <= 2 G  (P(x) - P* >= 1/2 ||A (x - x*)||^2)
    assert np.linalg.norm(A @ (r.x - xp)) ** 2 <= 2 * (max(r.gap, 0.0) + 1e-14) * (y @ y)


def test_gap_monotone_to_zero_and_weak_duality():
    """Weak duality P(x) >= D(theta) for feasible theta; the gap of the final point is >= 0."""
    A, y, lam = _small_problem(20, 40, 3, 0.3)
    r = _rng(7)
    for _ in range(50):
        x = r.standard_normal(40) * (r.random(40) < 0.3)
        z = r.standard_normal(20)
        theta = L.dual_scaling(z, A.T @ z)
        assert np.max(np.abs(A.T @ theta)) <= 1 + 1e-12
        assert L.primal(y - A @ x, x, lam) >= L.dual(theta, y, lam) - 1e-12


def test_proposition1_optimal_scaling_by_grid_search():
    """Prop. 1: clip(y^T z / (lam ||z||^2), +-1/||A^T z||_inf) z is the feasible multiple of z closest to y/lam."""
    A, y, lam = _small_problem(15, 30, 4, 0.4)
    r = _rng(9)
    for _ in range(20):
        z = r.standard_normal(15)
        m = np.max(np.abs(A.T @ z))
        s = L.theta_dynamic_coef(float(y @ z), float(z @ z), lam, m)
        grid = np.linspace(-1.0 / m, 1.0 / m, 200001)
        d = [np.linalg.norm(a * z - y / lam) for a in grid[::100]]
        a_best = grid[::100][int(np.argmin(d))]
        assert abs(s - a_best) <= 2 * (grid[100] - grid[0])
        assert np.linalg.norm(s * z - y / lam) <= min(d) + 1e-12
        assert np.max(np.abs(A.T @ (s * z))) <= 1 + 1e-12


def test_projection_coefficient_is_the_orthogonal_projection():
    """Prop. 1's beta: beta z is the orthogonal projection of y / lam on span(z), i.e. the
    least-squares coefficient of z for y / lam (numpy's lstsq), and the remainder is orthogonal to z."""
    r = _rng(21)
    for _ in range(20):
        N = int(r.integers(3, 40))
        y, z = r.standard_normal(N), r.standard_normal(N)
        lam = float(r.uniform(0.05, 3.0))
        beta = L.projection_coefficient(y, z, lam)
        ls = np.linalg.lstsq(z[:, None], y / lam, rcond=None)[0][0]
        assert abs(beta - ls) <= 1e-12 * max(abs(ls), 1e-300)
        assert abs(float(z @ (y / lam - beta * z))) <= 1e-12 * np.linalg.norm(z) * np.linalg.norm(y / lam)
    # a multiple of z projects onto itself
    z = r.standard_normal(7)
    assert abs(L.projection_coefficient(2.5 * 0.7 * z, z, 0.7) - 2.5) <= 1e-14


def test_stable_lambda_max_bounds_lambda_max():
    """eq:DefStableLMax: lambda'_max = max_j |a~_j^T y| + eps_j ||y|| >= lambda_max for every
    approximation with ||a~_j - a_j|| <= eps_j (Cauchy-Schwarz), with equality when eps = 0 and
    A~ = A, and it is attained when each approximation error points along -sign(a_j^T y) y.
    The Static Safe sphere built on it still contains theta* (y / lambda'_max is dual feasible)."""
    r = _rng(22)
    A, y, lam = _small_problem(25, 60, 7, 0.5)
    lm = L.lambda_max(A.T @ y)
    yn = float(np.linalg.norm(y))
    assert L.stable_lambda_max(A.T @ y, np.zeros(60), yn) == lm
    for _ in range(10):
        E = r.standard_normal(A.shape)
        eps = r.uniform(0.0, 0.2, 60)
        E *= eps / np.linalg.norm(E, axis=0)
        At = A + E
        assert L.stable_lambda_max(At.T @ y, eps, yn) >= lm * (1 - 1e-12)
    # tight case: a~_j = a_j - eps_j sign(a_j^T y) y / ||y|| with eps_j < |a_j^T y| / ||y||
    c = A.T @ y
    eps = 0.5 * np.abs(c) / yn
    At = A - (eps * np.sign(c))[None, :] * (y / yn)[:, None]
    np.testing.assert_allclose(np.abs(At.T @ y), np.abs(c) - eps * yn, rtol=1e-12)
    assert abs(L.stable_lambda_max(At.T @ y, eps, yn) - lm) <= 1e-12 * lm
    xs, ts = _theta_star(A, y, lam)
    cen, R = L.static_sphere(y, lam, L.stable_lambda_max(At.T @ y + 0.0, 2 * eps, yn))
    assert np.linalg.norm(ts - cen) <= R * (1 + 1e-12)


# ----------------------------------------------------------------------------- sphere tests

def test_sphere_test_closed_form_and_maximiser():
    """eq:sphere_test: sup over B(c, R) of |a^T theta| is |a^T c| + R||a||, attained at c +- R a/||a||."""
    r = _rng(11)
    for _ in range(20):
        a, c = r.standard_normal(10), r.standard_normal(10)
        R = float(r.random() * 2)
        mu = float(L.sphere_test(np.array([a @ c]), R, np.array([np.linalg.norm(a)]))[0])
        u = r.standard_normal((20000, 10))
        u /= np.linalg.norm(u, axis=1, keepdims=True)
        u *= r.random((20000, 1)) ** (1 / 10)
        assert np.max(np.abs((c + R * u) @ a)) <= mu + 1e-12
        th = c + np.sign(a @ c) * R * a / np.linalg.norm(a)
        assert abs(abs(a @ th) - mu) <= 1e-12


def test_stable_zone_test_bounds_every_atom_in_the_zone():
    """eq:sphere_test_approx(_normalized): for a in B(a~, eps) (and ||a|| = a0), |a^T theta| <= the stable test."""
    r = _rng(12)
    n = 8
    for _ in range(20):
        at, c = r.standard_normal(n), r.standard_normal(n)
        eps, R = 0.3 * r.random(), r.random()
        e = r.standard_normal((5000, n))
        e /= np.linalg.norm(e, axis=1, keepdims=True)
        a = at[None, :] + eps * r.random((5000, 1)) * e
        th = r.standard_normal((5000, n))
        th /= np.linalg.norm(th, axis=1, keepdims=True)
        th = c[None, :] + R * r.random((5000, 1)) ** (1 / n) * th
        lhs = np.abs(np.einsum("kn,kn->k", a, th))
        anorm = np.linalg.norm(a, axis=1)
        bound_norm = L.stable_sphere_test(np.full(5000, at @ c), eps, np.linalg.norm(c), R, anorm)
        bound = L.stable_sphere_test_unnormalized(at @ c, eps, np.linalg.norm(c), R, np.linalg.norm(at))
        assert np.all(lhs <= bound_norm + 1e-12)
        assert np.all(lhs <= bound + 1e-12)
        # the first two terms are attained: a = a~ + eps sign(a~^T c) c/||c||, theta = c (R = 0)
        a_star = at + eps * np.sign(at @ c) * c / np.linalg.norm(c)
        val = L.stable_sphere_test(np.array([at @ c]), eps, np.linalg.norm(c), 0.0,
                                   np.array([np.linalg.norm(a_star)]))[0]
        assert abs(abs(a_star @ c) - val) <= 1e-12


# ----------------------------------------------------------------------------- Section III lemmas

def _levels_for(A):
    f8, _, _ = D.fp8_quantize(A)
    bf = D.bf16_round(A)
    r = _rng(21)
    pert = A + 0.05 * r.standard_normal(A.shape)
    return [D.dense_level("fp8", f8, A, 0.25), D.dense_level("bf16", bf, A, 0.5),
            D.dense_level("pert", pert, A, 0.3)]


def test_lemma2_stable_scaling_is_feasible_for_both_dictionaries():
    """Lemma 2: Theta'(z|A~, eps) lies in Delta_A and Delta_A~; eps = 0 recovers Theta(z|A)."""
    w = S.dense_small(N=30, K=90, n_signals=1, seed=2)
    A = w.A
    r = _rng(13)
    for lev in _levels_for(A):
        At = lev.op.dense()
        for _ in range(20):
            z = r.standard_normal(30) * 5
            th = L.stable_dual_scaling(z, At.T @ z, lev.eps)
            assert np.max(np.abs(A.T @ th)) <= 1 + 1e-12
            assert np.max(np.abs(At.T @ th)) <= 1 + 1e-12
    z = r.standard_normal(30) * 5
    np.testing.assert_allclose(L.stable_dual_scaling(z, A.T @ z, np.zeros(90)), L.dual_scaling(z, A.T @ z))


def _theta_star(A, y, lam):
    x = SV.fista_gap_safe(A, y, lam, 1e-15, max_iter=200000).x
    xp, ok = SV.kkt_polish(A, y, lam, x)
    assert ok
    return xp, (y - A @ xp) / lam


@pytest.mark.parametrize("seed", range(3))
def test_theorem1_stable_gap_sphere_contains_theta_star(seed):
    """Theorem 1: theta* in B(theta', sqrt(2 G(x, theta'|A~) + 2 delta(x)) / lam) for any x.

    Checked with delta of eq:DefDelta (r = 1, E = max eps) and with e(x) = sum eps_j |x_j|.
    """
    w = S.dense_small(N=25, K=80, n_signals=3, seed=5)
    A = w.A
    y = w.Y[seed]
    lam = 0.3 * L.lambda_max(A.T @ y)
    xs, ts = _theta_star(A, y, lam)
    r = _rng(30 + seed)
    anorm = np.linalg.norm(A, axis=0)
    for lev in _levels_for(A):
        At = lev.op.dense()
        E = float(np.max(lev.eps))
        for k in range(200):
            x = xs + (0.3 * r.random()) * r.standard_normal(80) * (r.random(80) < 0.2)
            if k % 4 == 0:
                x = r.standard_normal(80) * (r.random(80) < 0.1)
            rho = y - At @ x
            g = At.T @ rho
            rr, yr = float(rho @ rho), float(y @ rho)
            m = float(np.max(np.abs(g) + lev.eps * np.sqrt(rr)))
            s = L.theta_dynamic_coef(yr, rr, lam, m)
            P = L.primal(rho, x, lam)
            Gp = P - L.dual_of_multiple(s, yr, rr, lam)
            for delta in (L.delta_theorem1(np.sqrt(rr), E, np.sum(np.abs(x))),
                          L.delta_from_error_bound(np.sqrt(rr), L.weighted_error_bound(lev.eps, x))):
                Rp = L.stable_gap_radius(Gp, delta, lam)
                assert np.linalg.norm(ts - s * rho) <= Rp * (1 + 1e-9) + 1e-12
                mu = L.stable_sphere_test(s * g, lev.eps, abs(s) * np.sqrt(rr), Rp, anorm)
                # every atom the stable test rejects is inactive at the solution
                assert np.all(xs[mu < 1.0] == 0.0)
                assert np.all(np.abs(A.T @ ts)[mu < 1.0] < 1.0)
                # the stable test dominates the exact-dictionary test on the true GAP sphere of theta'
                Gtrue = L.primal(y - A @ x, x, lam) - L.dual(s * rho, y, lam)
                exact_mu = L.sphere_test(A.T @ (s * rho), L.gap_safe_radius(Gtrue, lam), anorm)
                assert np.all(mu >= exact_mu - 1e-9)


def test_gap_safe_sphere_exact_dictionary():
    """eq:GAP_sphere: for feasible theta, theta* lies in B(theta, sqrt(2 G)/lam)."""
    A, y, lam = _small_problem(20, 50, 5, 0.25)
    xs, ts = _theta_star(A, y, lam)
    r = _rng(41)
    for _ in range(200):
        x = xs + 0.5 * r.standard_normal(50) * (r.random(50) < 0.3)
        rho = y - A @ x
        s = L.theta_dynamic_coef(float(y @ rho), float(rho @ rho), lam, float(np.max(np.abs(A.T @ rho))))
        G = L.primal(rho, x, lam) - L.dual(s * rho, y, lam)
        assert G >= -1e-12
        assert np.linalg.norm(ts - s * rho) <= L.gap_safe_radius(G, lam) + 1e-10


def test_weighted_error_bound_dominates_true_error_and_is_tighter_than_r1():
    A = S.dense_small(N=30, K=90, n_signals=1, seed=2).A
    r = _rng(17)
    for lev in _levels_for(A):
        At = lev.op.dense()
        for _ in range(50):
            x = r.standard_normal(90) * (r.random(90) < 0.3)
            e = L.weighted_error_bound(lev.eps, x)
            assert np.linalg.norm((A - At) @ x) <= e * (1 + 1e-12)
            assert e <= np.max(lev.eps) * np.sum(np.abs(x)) * (1 + 1e-12)


# ----------------------------------------------------------------------------- Algorithm 1 / 2

def test_switch_dictionary_algorithm2():
    assert L.switch_dictionary(0, 3, 0.9, 0.5, 10, 0.2, 100) == 3      # speed criterion first
    assert L.switch_dictionary(0, 3, 0.4, 0.5, 50, 0.2, 100) == 1      # convergence criterion
    assert L.switch_dictionary(1, 3, 0.6, 0.5, 50, 0.2, 100) == 1      # stay
    assert L.switch_dictionary(3, 3, 0.0, 0.5, 0, 0.2, 100) == 3       # exact is kept


@pytest.mark.parametrize("seed", range(4))
def test_fast_l1_ladder_is_safe_and_matches_minimiser(seed):
    """Algorithm 1 over FP8 -> BF16 -> exact: safe rejections, nested preserved sets,
    non-decreasing level index, 0 <= gamma_t <= 1, and the exact minimiser at the end."""
    w = S.dense_small(N=48, K=160, n_signals=4, seed=8)
    A = w.A
    y = w.Y[seed]
    lam = w.lam_ratio[seed] * L.lambda_max(A.T @ y)
    xs, ts = _theta_star(A, y, lam)
    f8, _, _ = D.fp8_quantize(A)
    levels = [D.dense_level("fp8", f8, A, 0.1), D.dense_level("bf16", D.bf16_round(A), A, 0.2), D.exact_level(A)]
    r = SV.fast_l1(levels, levels[-1].atnorm, y, lam, 1e-13, Gamma=0.5, trace=True, max_iter=100000)
    assert r.converged
    for _, rej in r.rejected_trace:
        assert np.all(xs[rej] == 0.0)
        assert np.all(np.abs(A.T @ ts)[rej] < 1.0)
    assert all(a >= b for a, b in zip(r.kept_trace, r.kept_trace[1:]))
    assert all(a <= b for a, b in zip(r.level_trace, r.level_trace[1:]))
    assert all(-1e-12 <= g <= 1 + 1e-12 for g in r.gamma_trace)
    assert np.linalg.norm(r.x - xs) <= 1e-5 * np.linalg.norm(xs)


def test_fast_l1_kronecker_ladder():
    """Kronecker truncations R = 1, 2 then the exact R = 3 sum: safe, and the exact minimiser."""
    w = S.kron_small(R=3, N1=6, K1=8, N2=5, K2=9, n_signals=2, seed=1, p=0.08)
    d = D.kron_unit_scale(w.Bf, w.Cf)
    exact = D.KronDict(w.Bf, w.Cf, d).dense()
    levels = [D.kron_level(w.Bf, w.Cf, d, 1), D.kron_level(w.Bf, w.Cf, d, 2), D.exact_level(exact)]
    for b in range(2):
        y = w.Y[b]
        lam = w.lam_ratio[b] * L.lambda_max(exact.T @ y)
        xs, ts = _theta_star(exact, y, lam)
        r = SV.fast_l1(levels, levels[-1].atnorm, y, lam, 1e-13, Gamma=0.5, trace=True, max_iter=100000)
        assert r.converged
        for _, rej in r.rejected_trace:
            assert np.all(xs[rej] == 0.0)
        assert np.linalg.norm(r.x - xs) <= 1e-5 * max(np.linalg.norm(xs), 1e-30)


def test_fast_l1_sparse_factor_ladder():
    """Products of sparse factors (Section VI) of increasing density, then the exact dense A: the
    rejections are safe and the exact minimiser is reached."""
    w = S.faust_small(N=40, K=120, n_signals=3, levels=((2, 2), (3, 4)), ratio=0.15)
    levels = [D.faust_level(f, w.A, name=f"faust{i}") for i, f in enumerate(w.levels)] + [D.exact_level(w.A)]
    for b in range(3):
        y = w.Y[b]
        lam = w.lam_ratio[b] * L.lambda_max(w.A.T @ y)
        xs, ts = _theta_star(w.A, y, lam)
        r = SV.fast_l1(levels, levels[-1].atnorm, y, lam, 1e-13, Gamma=0.5, trace=True, max_iter=100000)
        assert r.converged
        for _, rej in r.rejected_trace:
            assert np.all(xs[rej] == 0.0)
            assert np.all(np.abs(w.A.T @ ts)[rej] < 1.0)
        assert all(a <= b for a, b in zip(r.level_trace, r.level_trace[1:]))
        assert np.linalg.norm(r.x - xs) <= 1e-5 * max(np.linalg.norm(xs), 1e-30)


@pytest.mark.parametrize("seed", range(3))
def test_structured_polish_matches_brute_force(seed):
    """The operator form of the KKT polish (support columns formed from the Kronecker factors,
    KKT checked with the structured adjoint) reproduces the 3^K sign enumeration (K = 8)."""
    w = S.kron_small(R=2, N1=3, K1=2, N2=5, K2=4, n_signals=1, seed=seed, p=0.3)
    d = D.kron_unit_scale(w.Bf, w.Cf)
    op = D.KronDict(w.Bf, w.Cf, d)
    A = op.dense()
    y = w.Y[0]
    lam = max(w.lam_ratio[0], 0.3) * L.lambda_max(A.T @ y)
    xb = SV.brute_force(A, y, lam)
    r = SV.fast_l1([D.kron_level(w.Bf, w.Cf, d, 2)], np.linalg.norm(A, axis=0), y, lam, 1e-15, max_iter=400000)
    x, ok = SV.kkt_polish_op(op, y, lam, r.x, thresh=1e-9)
    assert ok
    np.testing.assert_allclose(x, xb, rtol=0, atol=1e-10)
    # a wrong support is rejected by the structured KKT check
    if np.count_nonzero(xb) >= 1:
        wrong = xb.copy()
        wrong[np.flatnonzero(xb)[0]] = 0.0
        if np.count_nonzero(wrong):
            _, ok_wrong = SV.kkt_polish_op(op, y, lam, wrong)
            assert not ok_wrong


@pytest.mark.parametrize("seed", range(4))
def test_static_sphere_contains_theta_star(seed):
    """The Static Safe sphere (eq:static_sphere) contains the dual solution theta* = (y - A x*)/lam
    (y / lam_max is dual feasible and theta* is the projection of y / lam on the feasible set), and
    the Static rule reaches the same minimiser while rejecting only atoms outside the support."""
    A, y, lam = _small_problem(30, 80, seed, 0.7)
    xs, ts = _theta_star(A, y, lam)
    c, R = L.static_sphere(y, lam, L.lambda_max(A.T @ y))
    assert np.linalg.norm(ts - c) <= R * (1 + 1e-12)
    r = SV.fast_l1([D.exact_level(A)], np.linalg.norm(A, axis=0), y, lam, 1e-13, rule=SV.STATIC, trace=True,
                   max_iter=200000)
    assert r.converged
    for _, rej in r.rejected_trace:
        assert np.all(xs[rej] == 0.0)
    assert np.linalg.norm(r.x - xs) <= 1e-5 * max(np.linalg.norm(xs), 1e-30)


def test_dynamic_safe_rule_and_ista():
    """Stable Dynamic Safe (Table I) and ISTA reach the same minimiser, safely."""
    A, y, lam = _small_problem(30, 90, 6, 0.6)
    xs, ts = _theta_star(A, y, lam)
    f8, _, _ = D.fp8_quantize(A)
    levels = [D.dense_level("fp8", f8, A, 0.1), D.exact_level(A)]
    for algo, rule in [(SV.FISTA, SV.DST), (SV.ISTA, SV.GAP), (SV.ISTA, SV.DST)]:
        r = SV.fast_l1(levels, levels[-1].atnorm, y, lam, 1e-12, algo=algo, rule=rule, trace=True,
                       max_iter=400000)
        assert r.converged
        for _, rej in r.rejected_trace:
            assert np.all(xs[rej] == 0.0)
        assert np.linalg.norm(r.x - xs) <= 1e-4 * np.linalg.norm(xs)
