"""The tensor-core GEMM (tcgen05 + TMA + TMEM) against an FP64 evaluation of the same products.

The stable test charges the tensor-core accumulation a rounding bound gamma_n(u_tc) sum |a r|
(u_tc = 2^-22 for BF16, 2^-19 for E4M3; n counts the products of all three parts in the split
form a1 r1 + a1 r2 + a2 r1 of the exact level); the measured error must stay well inside it.
"""
import ctypes as C

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1812_06635_gb300 import build, _native
    build.build()
    return _native.load()


@pytest.mark.parametrize("mode", [0, 1, 2])
@pytest.mark.parametrize("K,N,B", [(256, 2048, 512), (200, 1000, 300)])
def test_tensor_core_correlation_within_rounding_model(lib, mode, K, N, B):
    rel = C.c_double()
    ratio = C.c_double()
    code = lib.lasso_tc_selftest(mode, K, N, B, C.byref(rel), C.byref(ratio))
    assert code == 0, lib.lasso_strerror(code)
    # products of BF16 / E4M3 values are exact in FP32: errors come from the accumulation only
    assert rel.value < 1e-4, rel.value
    assert ratio.value < 0.1, ratio.value


def test_selftest_rejects_unknown_mode(lib):
    rel = C.c_double()
    ratio = C.c_double()
    assert lib.lasso_tc_selftest(3, 128, 64, 256, C.byref(rel), C.byref(ratio)) == -1
