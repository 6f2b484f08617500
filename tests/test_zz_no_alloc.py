"""The allocation-free lambda_max entry point agrees with the regular one (through the C ABI).

It serves callers that cannot call cudaMalloc: its scratch is a fixed array compiled into the
library.  Collected last so that a failure here never hides the other tests.
"""
import numpy as np
import pytest

import synthetic as S

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


@pytest.mark.parametrize("dtype,N,K,B", [("f32", 2048, 8192, 64), ("f32", 203, 1000, 37), ("f64", 100, 500, 3)])
def test_noalloc_lambda_max_matches_regular_entry_point(pkg, dtype, N, K, B):
    w = S.dense_small(N=N, K=K, n_signals=B, seed=N + K)
    d = pkg.Dictionary.dense(w.A, dtype=dtype)
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    ref = d.lambda_max(Y).cpu().numpy()
    for _ in range(2):                       # two calls in a row share the scratch
        out = torch.full((B,), -1.0, dtype=torch.float64, device="cuda")
        d.lambda_max_noalloc(Y, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        np.testing.assert_allclose(got, ref, rtol=1e-12, atol=0)
    # and both agree with an FP64 host evaluation of ||A^T y||_inf
    np.testing.assert_allclose(got, np.max(np.abs(w.Y @ w.A), axis=1), rtol=1e-6)
    d.close()


def test_noalloc_alone_on_a_fresh_dictionary_allocates_nothing(pkg):
    """First call on a new dictionary, with no regular call before it: the result matches an
    FP64 host evaluation of ||A^T y||_inf, and free device memory is the same before and after
    two calls.  A warm-up call on another dictionary first loads the library's kernels, whose
    module (with the fixed scratch array) is mapped once per process."""
    w0 = S.dense_small(N=64, K=256, n_signals=2, seed=5)
    d0 = pkg.Dictionary.dense(w0.A, dtype="f32")
    d0.lambda_max_noalloc(torch.tensor(w0.Y, dtype=torch.float32, device="cuda"))
    torch.cuda.synchronize()
    d0.close()
    w = S.dense_small(N=1000, K=3000, n_signals=9, seed=17)
    d = pkg.Dictionary.dense(w.A, dtype="f32")
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    out = torch.full((9,), -1.0, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(2):
        d.lambda_max_noalloc(Y, out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        np.testing.assert_allclose(out.cpu().numpy(), np.max(np.abs(w.Y @ w.A), axis=1), rtol=1e-6)
    d.close()


def test_noalloc_rejects_bad_buffers_before_the_call(pkg):
    """Buffers the kernel could overrun are refused by the binding (ValueError)."""
    w = S.dense_small(N=64, K=256, n_signals=4, seed=3)
    d = pkg.Dictionary.dense(w.A, dtype="f32")
    Y = torch.tensor(w.Y, dtype=torch.float32, device="cuda")
    for bad in (torch.zeros(4, dtype=torch.float32, device="cuda"), torch.zeros(3, dtype=torch.float64, device="cuda"),
                torch.zeros(4, dtype=torch.float64)):
        with pytest.raises(ValueError):
            d.lambda_max_noalloc(Y, bad)
    with pytest.raises(ValueError):
        d.lambda_max_noalloc(Y.double())
    with pytest.raises(ValueError):
        d.lambda_max_noalloc(Y[:, :32].contiguous())
    d.close()


def test_noalloc_rejects_oversized_batches(pkg):
    """B * ceil(K / 256) above the fixed scratch size is refused before any work is queued."""
    w = S.dense_small(N=64, K=8192, n_signals=1, seed=1)
    d = pkg.Dictionary.dense(w.A, dtype="f32")
    B = 40000                                 # 40000 * 32 atom blocks > 1048576 scratch entries
    Y = torch.zeros((B, 64), dtype=torch.float32, device="cuda")
    out = torch.zeros(B, dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.LassoError) as e:
        d.lambda_max_noalloc(Y, out)
    assert e.value.code == -6
    d.close()
