"""The seeded input generators follow the stated recipes (Section V distributions at the configured
sizes) and are reproducible and shardable; they hold none of the method's arithmetic."""
import numpy as np
import pytest

import synthetic as S


def _is_f32(a):
    return np.array_equal(np.asarray(a, np.float64), np.asarray(a, np.float32).astype(np.float64))


def test_c1_recipe():
    w = S.c1()
    assert w.A.shape == (100, 500) and w.Y.shape == (1, 100) and w.fp64
    np.testing.assert_allclose(np.linalg.norm(w.A, axis=0), 1.0, rtol=0, atol=1e-14)
    assert len(w.supports[0]) == 25 and len(set(w.supports[0].tolist())) == 25
    # y = A x0 + N(0, 0.01^2): the residual has the noise scale
    r = w.Y[0] - w.A[:, w.supports[0]] @ w.coefs[0]
    assert 0.005 < r.std() < 0.02
    assert w.lam_ratio[0] == 0.5 and w.tol == 1e-8


def test_c3_recipe_small_prefix():
    w = S.c3(n_signals=64, N=256, K=1024)
    assert _is_f32(w.A) and _is_f32(w.Y)
    np.testing.assert_allclose(np.linalg.norm(w.A, axis=0), 1.0, rtol=0, atol=1e-6)
    assert np.all((w.lam_ratio >= 0.1) & (w.lam_ratio <= 0.9))
    dens = np.array([len(s) for s in w.supports]) / 1024
    assert 0.005 < dens.min() and dens.max() < 0.08 and 0.015 < dens.mean() < 0.045
    # noiseless: y is exactly A x0 up to the FP32 rounding of y
    for b in range(4):
        y = w.A[:, w.supports[b]] @ w.coefs[b]
        assert np.linalg.norm(w.Y[b] - y) <= 1e-6 * np.linalg.norm(y)


def test_c4_recipe_noise_and_target():
    w = S.c4(n_signals=8, N=256, K=1024)
    assert w.x_target.shape == (8, 1024) and np.all(w.lam_ratio == 0.5)
    for b in range(8):
        clean = w.A[:, w.supports[b]] @ w.coefs[b]
        noise = w.Y[b] - clean
        snr = 20 * np.log10(np.linalg.norm(clean) / np.linalg.norm(noise))
        assert 17.0 < snr < 23.0
        assert 0 < np.count_nonzero(w.x_target[b]) < 0.08 * 1024


def test_kron_recipe_unit_atoms_and_row_major_vectorisation():
    w = S.kron_small(R=3, N1=4, K1=5, N2=3, K2=6, n_signals=2, seed=3, p=0.3)
    d = 1.0 / S.gen.kron_column_norms(w.Bf, w.Cf)
    M = sum(np.kron(w.Bf[r], w.Cf[r]) for r in range(3)) * d[None, :]
    np.testing.assert_allclose(np.linalg.norm(M, axis=0), 1.0, rtol=1e-12)
    for b in range(2):
        x = np.zeros(M.shape[1])
        x[w.supports[b]] = w.coefs[b]
        # noiseless by default: y is A x0 with the row-major Kronecker vectorisation
        np.testing.assert_allclose(w.Y[b], M @ x, rtol=0, atol=1e-5 * np.linalg.norm(M @ x))


def test_c5_sizes_and_ratio_range():
    w = S.c5(n_signals=4)
    assert w.Bf.shape == (8, 64, 256) and w.Cf.shape == (8, 128, 256)
    assert w.Y.shape == (4, 8192) and np.all((w.lam_ratio >= 0.2) & (w.lam_ratio <= 0.7))


@pytest.mark.parametrize("first", [0, 5])
def test_reproducible_and_prefix_shardable(first):
    a = S.c3(n_signals=4, first=first, N=64, K=128)
    b = S.c3(n_signals=4, first=first, N=64, K=128)
    np.testing.assert_array_equal(a.Y, b.Y)
    whole = S.c3(n_signals=9, N=64, K=128)
    np.testing.assert_array_equal(a.Y, whole.Y[first:first + 4])
    np.testing.assert_array_equal(a.A, whole.A)
    # another seed changes everything
    c = S.c3(n_signals=4, first=first, N=64, K=128, seed=1)
    assert not np.array_equal(a.Y, c.Y) and not np.array_equal(a.A, c.A)


def test_faust_recipe_factors_values_and_prefix():
    """Sparse-factor stand-in: FP32 values everywhere, canonical CSR factors with the stated
    entries per row (S_0, S_1) and per column (S_2), nested levels (each keeps a superset of the
    previous level's entries), unit atoms, 8-sparse unit-norm signals, prefix-shardable."""
    levels = ((3, 4), (4, 5))
    w = S.meg_faust(n_signals=5, levels=levels)
    assert _is_f32(w.A) and _is_f32(w.Y)
    np.testing.assert_allclose(np.linalg.norm(w.A, axis=0), 1.0, atol=1e-6)
    for (m0, m2), facs in zip(levels, w.levels):
        S0, S1, S2 = facs
        for F in facs:
            assert F.has_canonical_format and _is_f32(F.data)
            assert np.all(np.diff(F.indptr) >= 0)
        assert np.all(np.diff(S0.indptr) == m0) and np.all(np.diff(S1.indptr) == m0)
        assert np.all(np.diff(S2.tocsc().indptr) == m2)
    for F_lo, F_hi in zip(w.levels[0][:2], w.levels[1][:2]):
        lo = set(zip(*F_lo.nonzero()))
        assert lo <= set(zip(*F_hi.nonzero()))
    a = S.meg_faust(n_signals=3, first=2, levels=levels)
    np.testing.assert_array_equal(a.Y, w.Y[2:5])
    np.testing.assert_array_equal(a.A, w.A)
    assert all(len(s) == 8 for s in w.supports)
    np.testing.assert_allclose(np.linalg.norm(w.Y, axis=1), 1.0, rtol=1e-6)
