"""The C-ABI library builds, loads without a GPU and exports every function include/lasso.h declares."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lasso.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lasso_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1812_06635_gb300 import build, _native
    build.build()
    return _native.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    from paper_1812_06635_gb300 import _native
    assert sorted(n for n, _, _ in _native.SIGNATURES) == _declared()


def test_host_only_calls(lib):
    from paper_1812_06635_gb300 import _native
    o = _native.LassoOpts()
    lib.lasso_opts_default(C.byref(o))
    assert o.Gamma == 0.5 and o.screen_every == 1 and o.certify_full == 0 and o.passes_per_sync == 8
    assert lib.lasso_strerror(-4).decode().startswith("iteration limit")
    assert b"sm_103a" in lib.lasso_build_info()
    # argument validation happens before any device call
    h = C.c_void_p()
    assert lib.lasso_dict_create_dense(None, 1, 10, 10, 10, 1, 0, 1, C.byref(h)) == -1
    assert lib.lasso_dict_create_kron(None, None, 1, 2, 2, 2, 2, 1, 1, C.byref(h)) == -1
    assert lib.lasso_dict_add_level(None, 2, 0) == -1
    assert lib.lasso_dict_add_level_faust(None, 1, None, None, None, None) == -1
    assert lib.lasso_solve(None, None, 1.0, 1e-6, None, None, None, None, None, None) == -1


def test_messages_carry_the_refused_limit_of_the_latest_call(lib):
    """A refusal that records a detail shows it in lasso_strerror; the next call starts clean,
    so a later refusal without a detail shows the plain message (no stale text)."""
    import numpy as np
    h = C.c_void_p()
    buf = np.zeros(4, dtype=np.float32)
    p = buf.ctypes.data_as(C.c_void_p)
    code = lib.lasso_dict_create_dense(p, 1, (1 << 24) + 1, 1, (1 << 24) + 1, 1, 0, 1, C.byref(h))
    assert code == -6 and not h.value
    msg = lib.lasso_strerror(code).decode()
    assert msg.startswith("unsupported size or option") and "2^24" in msg, msg
    assert lib.lasso_dict_create_dense(p, 1, 0, 1, 1, 1, 0, 1, C.byref(h)) == -1
    assert lib.lasso_strerror(-1).decode() == "invalid argument"


def test_library_is_built_for_sm_103a_only():
    from paper_1812_06635_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_noalloc_buffer_checks_reject_bad_tensors():
    """The allocation-free lambda_max writes through raw pointers, so the binding refuses any
    buffer whose dtype, shape, layout or device does not match before calling the library
    (checked here on host tensors; the same function guards the CUDA call)."""
    torch = pytest.importorskip("torch")
    from paper_1812_06635_gb300.lasso import noalloc_args
    N = 8
    Y = torch.zeros((3, N), dtype=torch.float32)
    out = noalloc_args(Y, None, N, device_type="cpu")
    assert out.dtype == torch.float64 and out.numel() == 3
    assert noalloc_args(Y, torch.zeros(5, dtype=torch.float64), N, device_type="cpu").numel() == 5
    bad_Y = [Y.double(), torch.zeros((3, N + 1)), torch.zeros((0, N)), torch.zeros(N),
             torch.zeros((N, 3)).t(), Y.numpy()]
    for b in bad_Y:
        with pytest.raises(ValueError):
            noalloc_args(b, None, N, device_type="cpu")
    with pytest.raises(ValueError):
        noalloc_args(Y, None, N, device_type="cuda")          # host tensor for a device call
    bad_out = [torch.zeros(3, dtype=torch.float32), torch.zeros(2, dtype=torch.float64),
               torch.zeros(6, dtype=torch.float64)[::2], torch.zeros(3, dtype=torch.float64, device="meta")]
    for o in bad_out:
        with pytest.raises(ValueError):
            noalloc_args(Y, o, N, device_type="cpu")
