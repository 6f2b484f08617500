"""GPU parity of the screened solve (through the C ABI) with the FP64 oracle."""
import numpy as np
import pytest

import synthetic as S
from oracle import dictionaries as OD
from oracle import lasso as OL
from oracle import solvers as OS

from _ref import check_solution, exact_solution, true_rel_gap

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_06635_gb300 as p
    from paper_1812_06635_gb300 import build
    build.build()
    p.load()
    return p


# ----------------------------------------------------------------------------- FP64 single signal

def test_c1_fp64_gap_safe(pkg):
    """c1: 100 x 500 FP64, lambda = 0.5 lambda_max, GAP Safe, rel gap 1e-8 and 1e-12."""
    w = S.c1()
    A, y = w.A, w.Y[0]
    lam = 0.5 * OL.lambda_max(A.T @ y)
    xs = exact_solution(A, y, lam)
    d = pkg.Dictionary.dense(A, dtype="f64")
    for tol, xr in [(1e-8, None), (1e-12, 1e-5)]:
        x, gap, kept, st = d.solve(y, lam, tol)
        assert gap <= tol
        check_solution(A, y, lam, x, xs, gap, tol, kept, xr)
    x, gap, kept, st = d.solve(y, 0.5, tol=1e-12, lambda_relative=1)
    assert abs(st.lambda_max - OL.lambda_max(A.T @ y)) <= 1e-12 * st.lambda_max
    d.close()


def test_lambda_at_or_above_lambda_max_returns_zero(pkg):
    w = S.c1()
    A, y = w.A, w.Y[0]
    lm = OL.lambda_max(A.T @ y)
    d = pkg.Dictionary.dense(A, dtype="f64")
    x, gap, kept, st = d.solve(y, lm * (1 + 1e-9), 1e-10)
    assert np.all(x == 0) and gap == 0.0 and kept.size == 0
    x, gap, kept, st = d.solve(np.zeros(A.shape[0]), 0.1, 1e-10)
    assert np.all(x == 0) and gap == 0.0


def test_empty_batch_and_oversized_signals_are_rejected(pkg):
    """Host-side rejections before any device work: an empty batch (LASSO_ERR_INVALID_ARG) and
    signals longer than the supported 24576 padded entries (LASSO_ERR_UNSUPPORTED).  The
    dictionary stays usable after a rejected call."""
    w = S.dense_small(N=64, K=256, n_signals=2, seed=1)
    d = pkg.Dictionary.dense(w.A, dtype="f32")
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    ratios = torch.tensor(w.lam_ratio, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LassoError) as e:
        d.solve_batch(Y[:0].contiguous(), ratios[:0].contiguous(), 1e-6, lambda_relative=1)
    assert e.value.code == -1
    X, gaps, status, iters, st = d.solve_batch(Y, ratios, 1e-6, lambda_relative=1)
    assert bool((status == 0).all()) and float(gaps.max()) <= 1e-6
    d.close()
    rng = np.random.default_rng(0)
    db = pkg.Dictionary.dense(rng.standard_normal((24577, 8)).astype(np.float32), dtype="f32", normalize=True)
    Yb = torch.tensor(rng.standard_normal((1, 24577)), dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.LassoError) as e:
        db.solve_batch(Yb, torch.tensor([0.5], dtype=torch.float64, device="cuda"), 1e-6, lambda_relative=1)
    assert e.value.code == -6
    db.close()


@pytest.mark.parametrize("seed", range(3))
def test_brute_force_small_fp64(pkg, seed):
    r = np.random.default_rng(70 + seed)
    A = r.standard_normal((12, 8))
    A /= np.linalg.norm(A, axis=0)
    y = A @ (r.standard_normal(8) * (r.random(8) < 0.4)) + 0.05 * r.standard_normal(12)
    lam = 0.3 * OL.lambda_max(A.T @ y)
    xb = OS.brute_force(A, y, lam)
    d = pkg.Dictionary.dense(A, dtype="f64")
    x, gap, kept, st = d.solve(y, lam, 1e-14)
    np.testing.assert_allclose(x, xb, atol=1e-6)
    check_solution(A, y, lam, x, xb, gap, 1e-14, kept, 1e-5)


def test_orthonormal_soft_threshold(pkg):
    Q, y = S.orthonormal_case(64)
    lam = 0.3 * OL.lambda_max(Q.T @ y)
    d = pkg.Dictionary.dense(Q, dtype="f64")
    x, gap, kept, st = d.solve(y, lam, 1e-14)
    np.testing.assert_allclose(x, OL.soft_threshold(Q.T @ y, lam), atol=1e-10)


@pytest.mark.parametrize("algo,rule", [(1, 0), (0, 1), (1, 1), (0, 2), (1, 2)])
def test_ista_and_dynamic_safe(pkg, algo, rule):
    """ISTA / FISTA with the stable GAP, Dynamic Safe and Static Safe rules (Table I)."""
    w = S.c1()
    A, y = w.A, w.Y[0]
    lam = 0.5 * OL.lambda_max(A.T @ y)
    xs = exact_solution(A, y, lam)
    d = pkg.Dictionary.dense(A, dtype="f64")
    x, gap, kept, st = d.solve(y, lam, 1e-10, algo=algo, rule=rule)
    check_solution(A, y, lam, x, xs, gap, 1e-10, kept)


def test_max_iter_returns_partial_point(pkg):
    w = S.c1()
    A, y = w.A, w.Y[0]
    lam = 0.5 * OL.lambda_max(A.T @ y)
    d = pkg.Dictionary.dense(A, dtype="f64")
    with pytest.raises(pkg.LassoError) as e:
        d.solve(y, lam, 1e-14, max_iter=3)
    assert e.value.code == -4


# ----------------------------------------------------------------------------- levels

def test_level_data_matches_oracle_quantisers(pkg):
    w = S.dense_small(N=100, K=300, n_signals=1, seed=4)
    A = w.A
    d = pkg.Dictionary.dense(A, dtype="f32").add_level(pkg.LEVEL_FP8).add_level(pkg.LEVEL_BF16)
    e8, a8 = d.level_data(0)
    eb, ab = d.level_data(1)
    ex, ax = d.level_data(2)
    f8, _, _ = OD.fp8_quantize(A)
    np.testing.assert_array_equal(a8, f8.T)
    np.testing.assert_array_equal(ab, OD.bf16_round(A).T)
    np.testing.assert_array_equal(ax, A.T)
    np.testing.assert_allclose(e8, OD.dense_level("f8", f8, A, 0.25).eps, rtol=1e-10)
    np.testing.assert_allclose(eb, OD.dense_level("bf", OD.bf16_round(A), A, 0.5).eps, rtol=1e-10)
    assert np.all(ex == 0.0)
    info = d.info()
    assert info["n_levels"] == 3 and info["kind"] == [3, 2, -2]


@pytest.mark.parametrize("N,K", [(96, 384), (100, 517), (203, 1000)])
def test_dense_ladder_batch_parity(pkg, N, K):
    """FP8 -> BF16 -> exact FP32 ladder on a ragged batch: certified gap, safety, primal bound."""
    w = S.dense_small(N=N, K=K, n_signals=6, seed=N)
    A = w.A
    d = pkg.Dictionary.dense(A, dtype="f32").add_level(pkg.LEVEL_FP8).add_level(pkg.LEVEL_BF16)
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    lam = np.array([w.lam_ratio[b] * OL.lambda_max(A.T @ w.Y[b]) for b in range(6)])
    X, gaps, status, iters, st = d.solve_batch(Y, torch.tensor(lam, device="cuda"), tol=1e-6, certify_full=1)
    X = X.double().cpu().numpy()
    gaps = gaps.cpu().numpy()
    assert np.all(status.cpu().numpy() == 0)
    for b in range(6):
        xs = exact_solution(A, w.Y[b], lam[b])
        assert gaps[b] <= 1e-6
        check_solution(A, w.Y[b], lam[b], X[b], xs, gaps[b], 1e-6)
    # FP64 final rung: tight tolerance, x within 1e-5 of the minimiser
    X2, gaps2, status2, _, _ = d.solve_batch(Y, torch.tensor(lam, device="cuda"), tol=1e-13, final_fp64=1)
    assert np.all(status2.cpu().numpy() == 0)
    X2 = X2.double().cpu().numpy()
    for b in range(6):
        xs = exact_solution(A, w.Y[b], lam[b])
        assert np.linalg.norm(X2[b] - xs) <= 1e-5 * np.linalg.norm(xs) + 1e-7 * (np.linalg.norm(xs) == 0)
    d.close()


def test_single_signal_fp32_kept_set_is_safe(pkg):
    w = S.dense_small(N=128, K=640, n_signals=3, seed=11)
    A = w.A
    d = pkg.Dictionary.dense(A, dtype="f32").add_level(pkg.LEVEL_BF16)
    for b in range(3):
        y = w.Y[b]
        lam = w.lam_ratio[b] * OL.lambda_max(A.T @ y)
        xs = exact_solution(A, y, lam)
        x, gap, kept, st = d.solve(y, lam, 1e-6)
        check_solution(A, y, lam, x, xs, gap, 1e-6, kept)


# ----------------------------------------------------------------------------- Kronecker

def test_kron_levels_eps_and_parity(pkg):
    w = S.kron_small(R=3, N1=6, K1=8, N2=5, K2=9, n_signals=3, seed=2, p=0.08)
    d = pkg.Dictionary.kron(w.Bf, w.Cf).add_level(pkg.LEVEL_KRON, 1).add_level(pkg.LEVEL_KRON, 2)
    dsc = OD.kron_unit_scale(w.Bf, w.Cf)
    A = OD.KronDict(w.Bf, w.Cf, dsc).dense()
    for i, R in enumerate((1, 2)):
        e, _ = d.level_data(i, atoms=False)
        np.testing.assert_allclose(e, OD.kron_truncation_eps_gram(w.Bf, w.Cf, dsc, R), rtol=1e-9, atol=1e-14)
    e3, a3 = d.level_data(2)
    np.testing.assert_allclose(a3, OD.to_f32(A).T, rtol=0, atol=0)
    np.testing.assert_allclose(e3, np.linalg.norm(OD.to_f32(A) - A, axis=0), rtol=1e-6, atol=1e-14)
    for b in range(3):
        y = w.Y[b]
        lam = w.lam_ratio[b] * OL.lambda_max(A.T @ y)
        xs = exact_solution(A, y, lam)
        x, gap, kept, st = d.solve(y, lam, 1e-6)
        check_solution(A, y, lam, x, xs, gap, 1e-6, kept)


def test_kron_without_normalisation(pkg):
    """normalize = 0 keeps the Kronecker sum as given (d = 1, atoms of any norm): the stored exact
    atoms, the truncations' eps_j and the solutions match the oracle's unscaled operator."""
    w = S.kron_small(R=3, N1=6, K1=8, N2=5, K2=9, n_signals=3, seed=5, p=0.08)
    d = pkg.Dictionary.kron(w.Bf, w.Cf, normalize=False).add_level(pkg.LEVEL_KRON, 1)
    ones = np.ones(w.Bf.shape[2] * w.Cf.shape[2])
    A = OD.KronDict(w.Bf, w.Cf, ones).dense()
    assert np.ptp(np.linalg.norm(A, axis=0)) > 0.1          # the atoms are not unit-norm
    e0, _ = d.level_data(0, atoms=False)
    np.testing.assert_allclose(e0, OD.kron_truncation_eps_gram(w.Bf, w.Cf, ones, 1), rtol=1e-9, atol=1e-14)
    e1, a1 = d.level_data(1)
    np.testing.assert_allclose(a1, OD.to_f32(A).T, rtol=0, atol=0)
    for b in range(3):
        y = w.Y[b]
        lam = w.lam_ratio[b] * OL.lambda_max(A.T @ y)
        xs = exact_solution(A, y, lam)
        x, gap, kept, st = d.solve(y, lam, 1e-6)
        check_solution(A, y, lam, x, xs, gap, 1e-6, kept)
    d.close()


@pytest.mark.parametrize("ratio", [0.3, 0.5, 0.8])
def test_c2_structured(pkg, ratio):
    """c2 at full size: R = 4 terms of 32 x 64, truncations R = 1, 2, then the exact atoms."""
    w = S.c2(seed=0, lam_ratio=ratio)
    dsc = 1.0 / S.gen.kron_column_norms(w.Bf, w.Cf)
    A = OD.KronDict(w.Bf, w.Cf, dsc).dense()
    y = w.Y[0]
    lam = ratio * OL.lambda_max(A.T @ y)
    xs = exact_solution(A, y, lam, tol=1e-13)
    d = pkg.Dictionary.kron(w.Bf, w.Cf).add_level(pkg.LEVEL_KRON, 1).add_level(pkg.LEVEL_KRON, 2)
    x, gap, kept, st = d.solve(y, lam, 1e-6)
    check_solution(A, y, lam, x, xs, gap, 1e-6, kept)
    d.close()


# ----------------------------------------------------------------------------- C3 sampled

def test_c3_full_batch_sampled(pkg):
    """Full c3 batch (4096 signals, 2048 x 8192) in the bench's launch configuration.

    Every signal is checked by its status and certificate; 20 signals (the lambda / lambda_max and
    density extremes, the ragged end of the batch) are compared with the oracle minimisers stored
    in tests/golden/c3_reference.npz (written by make_references.py, which calls only oracle/):
    * tol 1e-6: the oracle's full-dictionary FP64 gap of the GPU point is <= tol and <= the GPU
      certificate, ||A (x - x*)||^2 <= 2 G ||y||^2, and the batch's preserved set (kept_mask)
      contains the support of x* (no unsafe rejection);
    * tol 1e-12 (FP64 rung): ||x - x*|| <= 1e-5 ||x*|| element by element, with the same safety.
    A relative gap of 1e-6 bounds ||A (x - x*)|| by sqrt(2e-6) ||y|| only: signals whose minimiser
    has a few tiny entries (lambda near lambda_max) sit far above 1e-5 in relative x error at that
    tolerance, which is why the element-wise bar is asserted at the tighter one.
    """
    import os
    ref = np.load(os.path.join(os.path.dirname(__file__), "golden", "c3_reference.npz"))
    w = S.c3()
    A = w.A
    d = pkg.Dictionary.dense(A, dtype="f32").add_level(pkg.LEVEL_FP8).add_level(pkg.LEVEL_BF16)
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    lmax = d.lambda_max(Y)
    lam = torch.tensor(w.lam_ratio, dtype=torch.float64, device="cuda") * lmax
    sig = [int(b) for b in ref["signals"]]
    assert len(sig) >= 16 and 4095 in sig
    for b in sig:
        assert abs(float(lmax[b]) - float(ref[f"s{b}_lmax"])) <= 1e-6 * float(ref[f"s{b}_lmax"])
        lam[b] = float(ref[f"s{b}_lam"])
    xs_all = {}
    for b in sig:
        xs = np.zeros(A.shape[1])
        xs[ref[f"s{b}_idx"]] = ref[f"s{b}_val"]
        xs_all[b] = xs
    for tol, kw in ((1e-6, {"certify_full": 1}), (1e-12, {"final_fp64": 1})):
        kept = torch.zeros((4096, A.shape[1]), dtype=torch.uint8, device="cuda")
        X, gaps, status, iters, st = d.solve_batch(Y, lam, tol=tol, kept=kept, **kw)
        assert bool((status == 0).all())
        assert float(gaps.max()) <= tol
        Xh = X.double().cpu().numpy()
        kh = kept.cpu().numpy().astype(bool)
        assert not np.any((Xh != 0) & ~kh)             # x is zero outside the preserved set
        errs = []
        for b in sig:
            xs = xs_all[b]
            assert kh[b][np.flatnonzero(xs)].all(), (tol, b)  # safety: supp(x*) is preserved
            if tol >= 1e-6:
                check_solution(A, w.Y[b], float(ref[f"s{b}_lam"]), Xh[b], xs, float(gaps[b]), tol)
            errs.append(np.linalg.norm(Xh[b] - xs) / np.linalg.norm(xs))
        print(f"c3 tol {tol:g}: relative x error median {np.median(errs):.2e} max {np.max(errs):.2e}")
        if tol <= 1e-12:
            assert max(errs) <= 1e-5, errs
    d.close()


# ----------------------------------------------------------------------------- differentiation

def test_backward_matches_oracle_adjoint(pkg):
    from oracle import backward as OB
    w = S.c4(n_signals=4, N=256, K=1024)
    A = w.A
    d = pkg.Dictionary.dense(A, dtype="f32")
    Xs, G = [], []
    for b in range(4):
        lam = 0.5 * OL.lambda_max(A.T @ w.Y[b])
        xs = exact_solution(A, w.Y[b], lam)
        Xs.append(xs)
        G.append(OB.target_loss(xs, w.x_target[b])[1])
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    Xt = torch.tensor(np.array(Xs), dtype=torch.float32, device="cuda")
    Gt = torch.tensor(np.array(G), dtype=torch.float32, device="cuda")
    dY, dA = d.backward(Y, Xt, Gt)
    dY = dY.double().cpu().numpy()
    dA = dA.double().cpu().numpy()
    dA_ref = np.zeros((A.shape[1], A.shape[0]))
    for b in range(4):
        x32 = Xs[b].astype(np.float32).astype(np.float64)
        g32 = G[b].astype(np.float32).astype(np.float64)
        ry, rA = OB.support_adjoint(A, w.Y[b], x32, g32)
        np.testing.assert_allclose(dY[b], ry, rtol=1e-4, atol=1e-4 * np.max(np.abs(ry)))
        dA_ref += rA.T
    np.testing.assert_allclose(dA, dA_ref, rtol=1e-3, atol=1e-4 * np.max(np.abs(dA_ref)))
    d.close()
