"""The rounding models folded into the bounds, checked on CPU emulations of the arithmetic.

The sparse-factor levels form A~^T rho and A~ z as FP32 FMA chains along CSR rows, one factor
after another (the chains of the kernels that evaluate products of sparse factors).  Their
bounds claim
    |g^_j - a~_j^T rho| <= gamma_{n_adj + 3} kappa_j ||rho||,
    ||AZ^ - A~ z||      <= gamma_{n_fwd + 5} sum_j kappa_j |z_j|,
with kappa_j = ||(|S_0| ... |S_{J-1}|) e_j||, n_fwd / n_adj the summed longest rows of the S_f /
of the S_f^T, gamma_n = n u / (1 - n u), u = 2^-24 (a reading of Section III-B: the paper
treats products as exact).  Here each FMA is emulated as one rounding to FP32 of the exact
product-sum (the product of two FP32 numbers is exact in FP64; the sum is then correctly
rounded twice, FP64 then FP32, which can only exceed one FP32 rounding by a factor 1 + 2^-29)."""
import numpy as np
import pytest

import synthetic as S
from oracle import dictionaries as D

U = 2.0 ** -24


def gamma(n):
    return n * U / (1.0 - n * U)


def _fma_chain_csr(indptr, indices, data, v):
    """out_i = FMA chain over row i (in stored order), every step rounded to FP32."""
    out = np.zeros(len(indptr) - 1, dtype=np.float32)
    for i in range(len(indptr) - 1):
        acc = np.float32(0.0)
        for p in range(indptr[i], indptr[i + 1]):
            acc = np.float32(float(acc) + float(np.float32(data[p])) * float(v[indices[p]]))
        out[i] = acc
    return out


def _longest_row(M):
    return int(np.max(np.diff(M.indptr))) if M.shape[0] else 0


@pytest.mark.parametrize("seed", range(3))
def test_sparse_factor_chains_stay_within_their_bounds(seed):
    w = S.faust_small(N=48, K=160, n_signals=4, seed=seed, levels=((2, 2), (4, 5), (6, 6)))
    rng = np.random.default_rng(seed)
    for facs in w.levels:
        op = D.FaustDict(facs)
        kappa = np.linalg.norm(op.abs_dense(), axis=0)
        n_fwd = sum(_longest_row(F) for F in facs)
        n_adj = sum(_longest_row(F.T.tocsr()) for F in facs)
        # adjoint: FP32 rho, S_0^T first
        rho = rng.standard_normal(op.N).astype(np.float32)
        v = rho
        for F in facs:
            Ft = F.T.tocsr()
            v = _fma_chain_csr(Ft.indptr, Ft.indices, Ft.data, v)
        g_exact = op.rmatvec(rho.astype(np.float64))
        err = np.abs(v.astype(np.float64) - g_exact)
        bound = gamma(n_adj + 3) * kappa * float(np.linalg.norm(rho.astype(np.float64)))
        assert np.all(err <= bound), float(np.max(err / bound))
        # forward: FP32 z with a few nonzeros, S_{J-1} first
        z = np.zeros(op.K, dtype=np.float32)
        nz = rng.choice(op.K, 12, replace=False)
        z[nz] = rng.standard_normal(12).astype(np.float32)
        v = z
        for F in reversed(facs):
            v = _fma_chain_csr(F.indptr, F.indices, F.data, v)
        az_exact = op.matvec(z.astype(np.float64))
        err_f = float(np.linalg.norm(v.astype(np.float64) - az_exact))
        assert err_f <= gamma(n_fwd + 5) * float(np.sum(kappa * np.abs(z.astype(np.float64))))


def test_bound_is_not_vacuous():
    """The observed chain errors are a visible fraction of the bound on adversarial data (all
    positive entries, so nothing cancels), i.e. the model is not loose by orders of magnitude."""
    w = S.faust_small(N=48, K=160, n_signals=1, seed=7, levels=((6, 6),))
    facs = [F.copy() for F in w.levels[0]]
    for F in facs:
        F.data = np.abs(F.data).astype(np.float32).astype(np.float64)
    op = D.FaustDict(facs)
    kappa = np.linalg.norm(op.abs_dense(), axis=0)
    n_adj = sum(_longest_row(F.T.tocsr()) for F in facs)
    rho = (1.0 + np.random.default_rng(0).random(op.N)).astype(np.float32)
    v = rho
    for F in facs:
        Ft = F.T.tocsr()
        v = _fma_chain_csr(Ft.indptr, Ft.indices, Ft.data, v)
    err = np.abs(v.astype(np.float64) - op.rmatvec(rho.astype(np.float64)))
    bound = gamma(n_adj + 3) * kappa * float(np.linalg.norm(rho.astype(np.float64)))
    assert np.all(err <= bound)
    assert float(np.max(err / bound)) > 1e-3


# ----------------------------------------------------------------------------- dense FP32 level

def _fma32(acc, a, r):
    return np.float32(float(acc) + float(a) * float(r))


def _round_up16(n):
    return (n + 15) // 16 * 16


def _emulate_pair_fma_dot(a, r):
    """The bulk correlation of an FP32 atom (the two-accumulator lane chains of the correlation
    pass): lane l takes the float4 groups l, l + 64, ... into one accumulator and l + 32, l + 96, ...
    into the other, the two are added, then a 5-level butterfly over the 32 lanes."""
    nv = a.size // 4
    lanes = np.zeros(32, dtype=np.float32)
    for lane in range(32):
        s0 = s1 = np.float32(0.0)
        k = lane
        while k + 32 < nv:
            for e in range(4):
                s0 = _fma32(s0, a[4 * k + e], r[4 * k + e])
            for e in range(4):
                s1 = _fma32(s1, a[4 * (k + 32) + e], r[4 * (k + 32) + e])
            k += 64
        if k < nv:
            for e in range(4):
                s0 = _fma32(s0, a[4 * k + e], r[4 * k + e])
        lanes[lane] = np.float32(float(s0) + float(s1))
    m = 16
    while m:
        lanes = np.array([np.float32(float(lanes[i]) + float(lanes[i ^ m])) for i in range(32)], dtype=np.float32)
        m >>= 1
    return float(lanes[0])


def _two_sum(a, b):
    s = np.float32(a + b)
    bb = np.float32(s - a)
    e = np.float32(np.float32(a - np.float32(s - bb)) + np.float32(b - bb))
    return s, e


def _emulate_dot2(a, r):
    """Dot2 as the error-free correlation of the exact level: per lane a double-float (s, c) fed by
    exact product splits p + q and TwoSum, a butterfly of merges, then s + c rounded to FP32."""
    nv = a.size // 4
    S_ = np.zeros(32, dtype=np.float32)
    C_ = np.zeros(32, dtype=np.float32)
    for lane in range(32):
        s = c = np.float32(0.0)
        for k in range(lane, nv, 32):
            for e in range(4):
                x, y = a[4 * k + e], r[4 * k + e]
                p = np.float32(float(x) * float(y))
                q = np.float32(float(x) * float(y) - float(p))      # exact
                t, err = _two_sum(s, p)
                s = t
                c = np.float32(c + np.float32(err + q))
        S_[lane], C_[lane] = s, c
    m = 16
    while m:
        nS, nC = S_.copy(), C_.copy()
        for i in range(32):
            t, err = _two_sum(S_[i], S_[i ^ m])
            nS[i] = t
            nC[i] = np.float32(np.float32(C_[i] + C_[i ^ m]) + err)
        S_, C_ = nS, nC
        m >>= 1
    return float(np.float32(S_[0] + C_[0]))


@pytest.mark.parametrize("N", [100, 2048, 2500])
def test_fp32_level_correlation_models(N):
    """Bulk FMA chains stay within gamma_{nl + 2} sum |a_i rho_i| with nl = ld/32 + 8 (ld = N rounded
    up to 16), and Dot2 within 2 gamma_{2 nl}^2 sum |a_i rho_i| plus the final rounding; random and
    cancellation-free (all positive) data."""
    import math
    ld = _round_up16(N)
    nl = math.ceil(ld / 32.0) + 8
    rng = np.random.default_rng(N)
    for trial in range(4):
        a = np.zeros(ld, dtype=np.float32)
        r = np.zeros(ld, dtype=np.float32)
        if trial < 2:
            a[:N] = rng.standard_normal(N).astype(np.float32)
            r[:N] = rng.standard_normal(N).astype(np.float32)
        else:
            a[:N] = (1.0 + rng.random(N)).astype(np.float32)
            r[:N] = (1.0 + rng.random(N)).astype(np.float32)
        exact = math.fsum(float(x) * float(y) for x, y in zip(a, r))
        mag = math.fsum(abs(float(x) * float(y)) for x, y in zip(a, r))
        g_fast = _emulate_pair_fma_dot(a, r)
        assert abs(g_fast - exact) <= gamma(nl + 2) * mag
        g_tight = _emulate_dot2(a, r)
        assert abs(g_tight - exact) <= 2.0 * gamma(2 * nl) ** 2 * mag + 3.0 * U * abs(g_tight)


# ----------------------------------------------------------------------------- residual

def _emulate_residual_row(yv, w, a_col, d2):
    """One row of the residual y - sum_q w_q a_{j_q}: an FMA chain over the nonzeros (d2 false) or
    Dot2 into a double-float (s, c), then y - (s + c) through TwoSum(y, -s) and the small terms."""
    s = c = np.float32(0.0)
    for wq, aq in zip(w, a_col):
        if d2:
            p = np.float32(float(wq) * float(aq))
            q = np.float32(float(wq) * float(aq) - float(p))
            t, err = _two_sum(s, p)
            s = t
            c = np.float32(c + np.float32(err + q))
        else:
            s = _fma32(s, wq, aq)
    t, e = _two_sum(np.float32(yv), np.float32(-s))
    return float(np.float32(t + np.float32(e - c)))


@pytest.mark.parametrize("nnz", [1, 7, 40])
def test_fp32_residual_models(nnz):
    """The residual bounds: FMA chains gamma_{nnz+4} sum_j kappa_j |z_j| + 2u ||rho^||, Dot2
    3 gamma_{2 nnz + 2}^2 sum_j kappa_j |z_j| + 2u ||rho^|| (kappa_j = ||a_j||; FP32 iterates)."""
    rng = np.random.default_rng(nnz)
    N = 300
    for trial in range(3):
        A = rng.standard_normal((N, nnz)).astype(np.float32)
        if trial == 2:
            A = np.abs(A)
        z = rng.standard_normal(nnz).astype(np.float32)
        y = (A.astype(np.float64) @ z.astype(np.float64) + 0.3 * rng.standard_normal(N)).astype(np.float32)
        exact = y.astype(np.float64) - A.astype(np.float64) @ z.astype(np.float64)
        kap = np.linalg.norm(A.astype(np.float64), axis=0)
        skz = float(np.sum(kap * np.abs(z.astype(np.float64))))
        for d2 in (False, True):
            rho = np.array([_emulate_residual_row(y[i], z, A[i], d2) for i in range(N)])
            err = float(np.linalg.norm(rho - exact))
            nr = float(np.linalg.norm(rho))
            if d2:
                g = gamma(2 * nnz + 2)
                bound = 3.0 * g * g * skz + 2.0 * U * nr
            else:
                bound = gamma(nnz + 4) * skz + 2.0 * U * nr
            assert err <= bound, (d2, err, bound)


U64 = 2.0 ** -53


def _gamma64(n):
    return n * U64 / (1.0 - n * U64)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fp64_kronecker_rung_bound(seed):
    """The FP64 rung of a Kronecker dictionary forms a_j = d_j sum_r b_r (x) c_r entry by entry:
    FP64 products of FP32 factor entries (exact), summed over r in order, then times d_j (FP64).
    Its eps_j claims ||a^_j - a_j|| <= gamma_{R+3}(2^-53) ||d_j sum_r |b_r (x) c_r| ||, and kappa_j
    bounds ||a^_j||.  Checked against exact rational arithmetic, with factor entries of both signs
    (cancelling terms) and spread exponents."""
    from fractions import Fraction
    rng = np.random.default_rng(100 + seed)
    R, N1, K1, N2, K2 = 5, 3, 4, 4, 3
    Bf = (rng.standard_normal((R, N1, K1)) * 2.0 ** rng.integers(-6, 6, (R, N1, K1))).astype(np.float32)
    Cf = (rng.standard_normal((R, N2, K2)) * 2.0 ** rng.integers(-6, 6, (R, N2, K2))).astype(np.float32)
    dcol = rng.uniform(0.5, 2.0, K1 * K2)
    worst = 0.0
    for j in range(K1 * K2):
        k1, k2 = divmod(j, K2)
        d = float(dcol[j])
        err2, norm2 = Fraction(0), Fraction(0)
        sabs, sa = 0.0, 0.0
        for n in range(N1 * N2):
            n1, n2 = divmod(n, N2)
            v, va = 0.0, 0.0
            exact = Fraction(0)
            for r in range(R):
                b, c = float(Bf[r, n1, k1]), float(Cf[r, n2, k2])
                p = b * c                                  # exact: 24 + 24 significant bits
                assert Fraction(p) == Fraction(b) * Fraction(c)
                v += p
                va += abs(p)
                exact += Fraction(b) * Fraction(c)
            v *= d
            va *= abs(d)
            sabs += va * va
            sa += v * v
            err2 += (Fraction(v) - Fraction(d) * exact) ** 2
            norm2 += Fraction(v) ** 2
        eps = _gamma64(R + 3.0) * np.sqrt(sabs) * (1.0 + 1e-12)
        kappa = np.sqrt(sa) * (1.0 + 1e-13)
        err = float(err2) ** 0.5
        assert err <= eps, (j, err, eps)
        # kappa_j >= ||a^_j||, compared in squares to avoid a rounded square root
        assert Fraction(kappa) ** 2 >= norm2, j
        worst = max(worst, err / eps)
    assert worst > 0.0          # the sums did round somewhere: the check is not vacuous
