"""Pins of the oracle's dictionaries, quantisers and error bounds (no GPU)."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import dictionaries as D


def _f32_samples(n, seed):
    r = np.random.default_rng(seed)
    v = (r.standard_normal(n) * np.exp2(r.integers(-12, 12, n))).astype(np.float32)
    # exact ties of the BF16 rounding: 16 low bits = 0x8000
    bits = v.view(np.uint32).copy()
    bits[: n // 8] = (bits[: n // 8] & 0xFFFF0000) | 0x8000
    return bits.view(np.float32)


def test_bf16_matches_torch_cast():
    v = _f32_samples(200000, 1)
    ours = D.bf16_round(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)


def test_e4m3_matches_torch_cast_in_range_and_saturates():
    r = np.random.default_rng(2)
    v = (r.standard_normal(200000) * np.exp2(r.integers(-11, 9, 200000))).astype(np.float32)
    v = np.clip(v, -448, 448)
    # exact midpoints between neighbouring E4M3 values, to pin ties-to-even
    grid = torch.arange(0, 127, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    mids = ((grid[1:] + grid[:-1]) / 2).astype(np.float32)
    v = np.concatenate([v, mids, -mids])
    ours = D.e4m3_round(v)
    ref = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(ours, ref)
    big = np.array([449.0, 463.9, 464.0, 500.0, 1e6, -1e6], dtype=np.float32)
    np.testing.assert_array_equal(D.e4m3_round(big), np.sign(big) * 448.0)


def test_split_bf16_pair():
    """a1 and a2 are torch's BF16 casts of a and of the exact remainder a - a1. Each BF16 rounding
    keeps 8 significant bits, so what both leave is at most 2^-16 |a| entrywise and
    eps_j <= 2^-16 ||a_j||. Entries of at most 16 significant bits split exactly (eps = 0)."""
    v = _f32_samples(60000, 3).reshape(300, 200)
    a1, a2, eps = D.split_bf16(v)
    t = torch.from_numpy(v)
    ref1 = t.to(torch.bfloat16).to(torch.float64)
    np.testing.assert_array_equal(a1, ref1.numpy())
    rem = t.to(torch.float64) - ref1
    assert torch.equal(rem.to(torch.float32).to(torch.float64), rem)          # the remainder is an FP32 value
    np.testing.assert_array_equal(a2, rem.to(torch.float32).to(torch.bfloat16).to(torch.float64).numpy())
    a = v.astype(np.float64)
    e = a - a1 - a2
    assert np.all(np.abs(e) <= 2.0 ** -16 * np.abs(a))
    np.testing.assert_allclose(eps, np.linalg.norm(e, axis=0), rtol=1e-14)
    assert np.all(eps <= 2.0 ** -16 * np.linalg.norm(a, axis=0))
    assert np.any(eps > 0)
    # 16 significant bits (the implicit one and 15 stored): a1 + a2 == a
    v16 = (v.view(np.uint32) & np.uint32(0xFFFFFF00)).view(np.float32)
    b1, b2, eps16 = D.split_bf16(v16)
    np.testing.assert_array_equal(b1 + b2, v16.astype(np.float64))
    assert np.all(eps16 == 0.0)


def test_fp8_atom_scaled_copy():
    A = S.dense_small(N=64, K=100, n_signals=1).A
    At, q, s = D.fp8_quantize(A)
    assert np.all(np.abs(q) <= 448.0)
    np.testing.assert_array_equal(At, q * s[None, :])
    # the largest entry of every atom lands near the top of the FP8 range
    assert np.all(np.max(np.abs(q), axis=0) >= 416.0)
    lev = D.dense_level("fp8", At, A, 0.25)
    np.testing.assert_allclose(lev.eps, np.linalg.norm(At - A, axis=0), rtol=1e-11)
    # E4M3 has a 3-bit mantissa: relative rounding error at most 2^-4 on normal values
    assert np.all(lev.eps <= 2.0 ** -4 * np.linalg.norm(A, axis=0))


def test_kron_operator_against_explicit_kron():
    w = S.kron_small(R=3, N1=4, K1=6, N2=5, K2=7, n_signals=1)
    d = D.kron_unit_scale(w.Bf, w.Cf)
    M = sum(np.kron(w.Bf[r], w.Cf[r]) for r in range(3)) * d[None, :]
    op = D.KronDict(w.Bf, w.Cf, d)
    r = np.random.default_rng(3)
    x, rho = r.standard_normal(op.K), r.standard_normal(op.N)
    np.testing.assert_allclose(op.matvec(x), M @ x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(op.rmatvec(rho), M.T @ rho, rtol=0, atol=1e-13)
    np.testing.assert_allclose(op.dense(), M, rtol=0, atol=1e-14)
    np.testing.assert_allclose(np.linalg.norm(M, axis=0), 1.0, rtol=1e-13)
    idx = np.array([0, 5, 17, 40])
    np.testing.assert_allclose(op.matvec(x[idx], idx), M[:, idx] @ x[idx], atol=1e-13)
    np.testing.assert_allclose(op.rmatvec(rho, idx), M[:, idx].T @ rho, atol=1e-13)


def test_kron_truncation_eps_gram_equals_column_differences():
    w = S.kron_small(R=4, N1=5, K1=6, N2=4, K2=8, n_signals=1)
    d = D.kron_unit_scale(w.Bf, w.Cf)
    full = D.KronDict(w.Bf, w.Cf, d).dense()
    for Rk in (1, 2, 3, 4):
        trunc = D.KronDict(w.Bf, w.Cf, d, Rk).dense()
        np.testing.assert_allclose(D.kron_truncation_eps_gram(w.Bf, w.Cf, d, Rk),
                                   np.linalg.norm(trunc - full, axis=0), rtol=1e-10, atol=1e-14)
        lev = D.kron_level(w.Bf, w.Cf, d, Rk)
        np.testing.assert_allclose(lev.atnorm, np.linalg.norm(trunc, axis=0), rtol=1e-10)


def _dense_factors(factors):
    return [np.asarray(f.toarray(), np.float64) for f in factors]


@pytest.mark.parametrize("dims", [(7, 11), (6, 9, 13), (5, 8, 4, 12)])
def test_faust_operator_against_explicit_product(dims):
    """S_0 ... S_{J-1} applied factor by factor equals the explicit product of the dense factors
    (rectangular shapes, J = 1, 2, 3), adjoint included; restricted products select atoms."""
    r = np.random.default_rng(len(dims))
    facs = []
    for a, b in zip(dims[:-1], dims[1:]):
        M = r.standard_normal((a, b)) * (r.random((a, b)) < 0.4)
        rr, cc = np.nonzero(M)
        facs.append(S.gen._csr(a, b, rr, cc, M[rr, cc]))
    Ds = _dense_factors(facs)
    M = Ds[0] if len(Ds) == 1 else np.linalg.multi_dot(Ds)
    op = D.FaustDict(facs)
    assert (op.N, op.K) == M.shape
    x, rho = r.standard_normal(op.K), r.standard_normal(op.N)
    np.testing.assert_allclose(op.matvec(x), M @ x, rtol=0, atol=1e-13)
    np.testing.assert_allclose(op.rmatvec(rho), M.T @ rho, rtol=0, atol=1e-13)
    np.testing.assert_allclose(op.dense(), M, rtol=0, atol=1e-13)
    assert abs(float(op.matvec(x) @ rho) - float(x @ op.rmatvec(rho))) <= 1e-12 * (1 + abs(float(x @ op.rmatvec(rho))))
    absM = np.abs(Ds[0]) if len(Ds) == 1 else np.linalg.multi_dot([np.abs(F) for F in Ds])
    np.testing.assert_allclose(op.abs_dense(), absM, rtol=0, atol=1e-13)
    idx = np.array([0, 3, op.K - 1])
    np.testing.assert_allclose(op.matvec(x[idx], idx), M[:, idx] @ x[idx], atol=1e-13)
    np.testing.assert_allclose(op.rmatvec(rho, idx), M[:, idx].T @ rho, atol=1e-13)
    for j in idx:
        np.testing.assert_allclose(op.col(j), M[:, j], atol=1e-14)


def test_faust_level_errors_and_exact_product():
    """eps_j of a sparse-factor level is the column distance to the exact atoms; it vanishes when the
    exact dictionary is the product itself; RC counts the factors' nonzeros over N K."""
    w = S.faust_small(N=24, K=40, levels=((2, 2), (3, 3), (6, 6)))
    for facs in w.levels:
        P = np.linalg.multi_dot(_dense_factors(facs))
        lev = D.faust_level(facs, w.A)
        np.testing.assert_allclose(lev.eps, np.linalg.norm(P - w.A, axis=0), rtol=1e-10, atol=1e-15)
        np.testing.assert_allclose(lev.atnorm, np.linalg.norm(P, axis=0), rtol=1e-12)
        assert lev.rc == pytest.approx(sum(f.nnz for f in facs) / (24 * 40))
        self_lev = D.faust_level(facs, P)
        assert np.all(self_lev.eps <= 1e-13)
    # keeping more entries of each factor brings the product closer to A
    means = [float(D.faust_level(f, w.A).eps.mean()) for f in w.levels]
    assert means[0] > means[1] > means[2]


def test_generator_faust_ladder_matches_section_vi_profile():
    """The source-localisation stand-in: 204 x 8193, unit atoms, four levels with mean eps_j
    decreasing from about 0.2 to about 0.06 (the profile of the paper's FAuST approximations)."""
    w = S.meg_faust(n_signals=3)
    assert w.A.shape == (204, 8193)
    np.testing.assert_allclose(np.linalg.norm(w.A, axis=0), 1.0, atol=1e-6)
    means = []
    for facs in w.levels:
        assert facs[0].shape == (204, 204) and facs[1].shape == (204, 204) and facs[2].shape == (204, 8193)
        means.append(float(D.faust_level(facs, w.A).eps.mean()))
    assert all(a > b for a, b in zip(means, means[1:]))
    assert 0.15 < means[0] < 0.3 and 0.045 < means[-1] < 0.075
    np.testing.assert_allclose(np.linalg.norm(w.Y, axis=1), 1.0, rtol=1e-6)
    assert all(len(s) == 8 for s in w.supports) and np.all(w.lam_ratio == 0.1)


def test_generator_kron_norms_agree_with_oracle():
    w = S.kron_small(R=3, N1=4, K1=6, N2=5, K2=7, n_signals=1)
    np.testing.assert_allclose(1.0 / S.gen.kron_column_norms(w.Bf, w.Cf), D.kron_unit_scale(w.Bf, w.Cf),
                               rtol=1e-12)


def test_power_iteration_matches_spectral_norm():
    A = S.dense_small(N=50, K=120, n_signals=1).A
    L = D.power_iteration_sq_norm(D.DenseDict(A), iters=500, safety=1.0)
    ref = np.linalg.norm(A, 2) ** 2
    assert abs(L - ref) <= 1e-6 * ref
    assert D.power_iteration_sq_norm(D.DenseDict(A), iters=500) >= ref


@pytest.mark.parametrize("decay", [None, 0.5])
def test_c2_levels_shapes_and_errors(decay):
    """c2 dictionary: unit atoms; truncation errors decrease with R and vanish at R = 4."""
    w = S.c2(decay=decay)
    d = 1.0 / S.gen.kron_column_norms(w.Bf, w.Cf)
    e = [D.kron_truncation_eps_gram(w.Bf, w.Cf, d, R) for R in (1, 2, 3, 4)]
    assert all(np.all(a >= b - 1e-12) for a, b in zip(e, e[1:]))
    assert np.max(e[-1]) == 0.0
    assert w.N == 1024 and w.K == 4096
