"""Error paths of the batch and single solves through the C ABI (the status codes of the boundary).

Each failure is made on the host: a NaN written into one signal before the copy to the device,
and a wall-clock limit far below the time of one pass.  Nothing here faults or hangs the GPU.
The bar: the call and the per-signal statuses carry the code, every other signal is solved as
usual, and a stopped signal returns a finite partial point with a certificate that bounds its
suboptimality.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import lasso as OL

from _ref import exact_solution

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


def _primal_rel(A, y, lam, x):
    r = y - A @ x
    return (0.5 * float(r @ r) + lam * float(np.abs(x).sum())) / float(y @ y)


def test_nan_in_one_signal_is_reported_and_the_others_solve(pkg):
    """LASSO_ERR_NONFINITE for the signal whose y holds a NaN; its x stays zero (no pass ran) and
    its gap is +inf (nothing was certified); the other signals are certified as usual."""
    w = S.dense_small(N=96, K=384, n_signals=6, seed=8)
    A = w.A
    Yh = w.Y.astype(np.float32).copy()
    Yh[2, 17] = np.nan
    d = pkg.Dictionary.dense(A, dtype="f32").add_level(pkg.LEVEL_BF16)
    Y = torch.tensor(Yh, device="cuda")
    lam = torch.tensor([w.lam_ratio[b] * OL.lambda_max(A.T @ w.Y[b]) if b != 2 else 0.5 for b in range(6)],
                       dtype=torch.float64, device="cuda")
    kept = torch.zeros((6, A.shape[1]), dtype=torch.uint8, device="cuda")
    X, gaps, status, iters, st = d.solve_batch(Y, lam, 1e-6, kept=kept)
    status = status.cpu().numpy()
    X = X.double().cpu().numpy()
    gaps = gaps.cpu().numpy()
    assert status[2] == -3
    assert np.all(X[2] == 0.0) and np.isinf(gaps[2])
    for b in (0, 1, 3, 4, 5):
        assert status[b] == 0 and gaps[b] <= 1e-6
        xs = exact_solution(A, w.Y[b], float(lam[b]))
        assert set(np.flatnonzero(xs)) <= set(np.flatnonzero(kept[b].cpu().numpy()))
    # the host variant reports the same
    Xh, gh, sh, _ = d.solve_batch_host(Yh, lam.cpu().numpy(), 1e-6)
    assert sh[2] == -3 and np.all(sh[[0, 1, 3, 4, 5]] == 0)
    d.close()


def test_time_limit_returns_partial_points_and_their_certificates(pkg):
    """time_limit_s = 1e-6 expires before the first pass: the call returns LASSO_ERR_TIMEOUT, every
    signal stops at its next pass with status TIMEOUT, a finite point and a certificate (relative
    gap of that point) with P(x) - P* <= gap ||y||^2; no atom of the minimiser is rejected."""
    w = S.dense_small(N=256, K=1024, n_signals=80, seed=12)
    A = w.A
    d = pkg.Dictionary.dense(A, dtype="f32").add_level(pkg.LEVEL_FP8).add_level(pkg.LEVEL_BF16)
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    lam = torch.tensor([w.lam_ratio[b] * OL.lambda_max(A.T @ w.Y[b]) for b in range(80)], dtype=torch.float64,
                       device="cuda")
    kept = torch.zeros((80, A.shape[1]), dtype=torch.uint8, device="cuda")
    X, gaps, status, iters, st = d.solve_batch(Y, lam, 1e-6, kept=kept, time_limit_s=1e-6)
    status = status.cpu().numpy()
    assert np.all(status == -5), np.unique(status)
    X = X.double().cpu().numpy()
    gaps = gaps.cpu().numpy()
    kept = kept.cpu().numpy()
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(gaps)) and np.all(gaps > 0)
    for b in (0, 1, 41, 79):
        la = float(lam[b])
        xs = exact_solution(A, w.Y[b], la)
        sub = _primal_rel(A, w.Y[b], la, X[b]) - _primal_rel(A, w.Y[b], la, xs)
        assert -1e-12 <= sub <= gaps[b] * (1 + 1e-6) + 1e-12, (b, sub, gaps[b])
        assert set(np.flatnonzero(xs)) <= set(np.flatnonzero(kept[b]))
    # the dictionary solves normally afterwards
    X2, gaps2, status2, _, _ = d.solve_batch(Y, lam, 1e-6)
    assert bool((status2 == 0).all()) and float(gaps2.max()) <= 1e-6
    d.close()


def test_single_solve_time_limit_raises_with_timeout(pkg):
    w = S.c1()
    A, y = w.A, w.Y[0]
    d = pkg.Dictionary.dense(A, dtype="f64")
    with pytest.raises(pkg.LassoError) as e:
        d.solve(y, 0.5 * OL.lambda_max(A.T @ y), 1e-14, time_limit_s=1e-6)
    assert e.value.code == -5
    x, gap, kept, st = d.solve(y, 0.5 * OL.lambda_max(A.T @ y), 1e-8)
    assert gap <= 1e-8
    d.close()


def test_lassofn_refuses_to_differentiate_an_unsolved_signal(pkg):
    """LassoFn.forward raises when a signal ends with a non-zero status (here: the pass limit)."""
    w = S.c4(n_signals=4, N=128, K=512)
    A = torch.tensor(w.A, dtype=torch.float32)
    d = pkg.Dictionary.dense(w.A, dtype="f32")
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda", requires_grad=True)
    lam = torch.tensor([0.5 * OL.lambda_max(w.A.T @ w.Y[b]) for b in range(4)], dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LassoError):
        pkg.LassoFn.apply(Y, None, d, lam, 1e-6, {"max_iter": 2, "fp64_fallback": 0})
    X = pkg.LassoFn.apply(Y, None, d, lam, 1e-6, None)
    assert X.shape == (4, 512) and bool(torch.isfinite(X).all())
    d.close()
