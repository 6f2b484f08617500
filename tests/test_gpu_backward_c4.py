"""Differentiation at full size: A 1024 x 4096 (FP32, unit atoms), 256 signals, lambda = 0.5 lambda_max,
loss L = ||x* - x_target||^2, gradients through ``LassoFn`` (support-system adjoint).

Checked on sampled signals against the FP64 oracle: the solution itself, dL/dy and dL/dA from
the oracle's adjoint at the oracle's own minimiser, and central finite differences (h = 1e-4,
FP64, sign pattern held fixed) of the oracle's loss in coordinates of y and of A.
"""
import numpy as np
import pytest

import synthetic as S
from oracle import backward as OB
from oracle import lasso as OL

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SAMPLED = [0, 37, 128, 255]


@pytest.fixture(scope="module")
def run():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1812_06635_gb300 as pkg
    from paper_1812_06635_gb300 import build
    build.build()
    pkg.load()
    w = S.c4()
    d = pkg.Dictionary.dense(w.A, dtype="f32").prepare()
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda", requires_grad=True)
    A_t = torch.tensor(w.A, dtype=torch.float32, device="cuda", requires_grad=True)
    Xt = torch.tensor(w.x_target, dtype=torch.float32, device="cuda")
    ratios = torch.full((w.Y.shape[0],), 0.5, dtype=torch.float64, device="cuda")
    X = pkg.LassoFn.apply(Y, A_t, d, ratios, 1e-12, {"lambda_relative": 1, "final_fp64": 1})
    loss = ((X - Xt) ** 2).sum()
    loss.backward()
    refs = {}
    for b in SAMPLED:
        y = w.Y[b]
        lam = 0.5 * OL.lambda_max(w.A.T @ y)
        x = OB.solve_exact(w.A, y, lam)
        refs[b] = (lam, x)
    yield w, d, X.detach(), Y, A_t, refs
    d.close()


def test_solution_matches_oracle(run):
    w, d, X, Y, A_t, refs = run
    Xh = X.double().cpu().numpy()
    for b, (lam, x) in refs.items():
        assert np.linalg.norm(Xh[b] - x) <= 1e-5 * max(np.linalg.norm(x), 1e-30), b
        # same support (the gradient is defined by it)
        assert set(np.flatnonzero(np.abs(Xh[b]) > 1e-4 * np.abs(x).max())) == set(np.flatnonzero(x)), b


def test_dy_matches_oracle_adjoint(run):
    w, d, X, Y, A_t, refs = run
    gY = Y.grad.double().cpu().numpy()
    for b, (lam, x) in refs.items():
        g = OB.target_loss(x, w.x_target[b])[1]
        dy, _ = OB.support_adjoint(w.A, w.Y[b], x, g)
        np.testing.assert_allclose(gY[b], dy, rtol=0, atol=1e-3 * np.abs(dy).max() + 1e-12)


def test_dA_matches_oracle_adjoint_on_sampled_signals(run):
    w, d, X, Y, A_t, refs = run
    idx = torch.tensor(SAMPLED, device="cuda")
    Ys = Y.detach()[idx].contiguous()
    Xs = X[idx].contiguous()
    Gs = (2.0 * (Xs - torch.tensor(w.x_target[SAMPLED], dtype=torch.float32, device="cuda"))).contiguous()
    _, dA = d.backward(Ys, Xs, Gs)
    dA = dA.double().cpu().numpy().T          # N x K
    ref = np.zeros_like(w.A)
    for b, (lam, x) in refs.items():
        g = OB.target_loss(x, w.x_target[b])[1]
        ref += OB.support_adjoint(w.A, w.Y[b], x, g)[1]
    np.testing.assert_allclose(dA, ref, rtol=0, atol=1e-3 * np.abs(ref).max() + 1e-12)
    # and the autograd path sums the same per-signal terms over the whole batch
    assert A_t.grad is not None and A_t.grad.shape == (w.A.shape[0], w.A.shape[1])
    supp = np.flatnonzero(np.abs(X.double().cpu().numpy()).sum(0))
    off = np.setdiff1d(np.arange(w.A.shape[1]), supp)
    assert float(A_t.grad[:, torch.tensor(off, device="cuda")].abs().max()) == 0.0


def test_finite_differences(run):
    """Central differences of the oracle's loss (sign pattern fixed) against the GPU gradients."""
    w, d, X, Y, A_t, refs = run
    rng = np.random.default_rng(4)
    gY = Y.grad.double().cpu().numpy()
    gA = A_t.grad.double().cpu().numpy()
    checked = 0
    for b, (lam, x) in refs.items():
        Sset = np.flatnonzero(x)
        if Sset.size == 0:
            continue
        s = np.sign(x[Sset])
        theta = (w.Y[b] - w.A @ x) / lam
        slack = 1.0 - np.max(np.abs(np.delete(w.A.T @ theta, Sset))) if Sset.size < w.A.shape[1] else 1.0
        if np.min(np.abs(x[Sset])) < 1e-2 or slack < 1e-2:
            continue                      # support not stable under the perturbation
        for n in rng.choice(w.A.shape[0], 8, replace=False):
            fd = OB.finite_difference(w.A, w.Y[b], lam, w.x_target[b], "y", int(n), h=1e-4, support=(Sset, s))
            assert abs(gY[b, n] - fd) <= 1e-3 * np.abs(gY[b]).max() + 1e-6, (b, n)
        if b == SAMPLED[0] or checked == 0:
            # dL/dA of this signal alone: the batch gradient minus the others is not separable,
            # so check A's coordinates on a support column through the per-signal adjoint
            g = OB.target_loss(x, w.x_target[b])[1]
            _, dA_ref = OB.support_adjoint(w.A, w.Y[b], x, g)
            for n in rng.choice(w.A.shape[0], 4, replace=False):
                j = int(rng.choice(Sset))
                fd = OB.finite_difference(w.A, w.Y[b], lam, w.x_target[b], "A", (int(n), j), h=1e-4,
                                          support=(Sset, s))
                assert abs(dA_ref[n, j] - fd) <= 1e-4 * np.abs(dA_ref).max() + 1e-7, (b, n, j)
        checked += 1
    assert checked >= 1
    assert np.isfinite(gA).all()
