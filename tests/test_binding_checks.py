"""The Python binding refuses, before any library call, buffers the library would overrun.

The C calls read and write exactly B x N signal entries, B lambdas and B x K solution entries
through plain pointers. A tensor of another shape, type or device (a host tensor passed to a
device call) must raise ValueError in the binding, never reach a kernel. Runs without a GPU: the
dictionary handle is never used, because every call here fails its checks first.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    from paper_1812_06635_gb300 import build
    import paper_1812_06635_gb300 as p
    build.build()
    p.load()
    return p


def test_device_rows_accepts_exactly_the_described_buffer():
    from paper_1812_06635_gb300.lasso import device_rows
    ok = torch.zeros((3, 8), dtype=torch.float32)
    assert device_rows(ok, "Y", 8, torch.float32, device_type="cpu") is ok
    assert device_rows(ok, "Y", 8, torch.float32, rows=3, device_type="cpu") is ok
    empty = torch.zeros((0, 8), dtype=torch.float32)          # the library reports an empty batch itself
    assert device_rows(empty, "Y", 8, torch.float32, device_type="cpu") is empty
    bad = [torch.zeros((3, 7), dtype=torch.float32),           # width
           torch.zeros((3, 8), dtype=torch.float64),           # type
           torch.zeros((8, 3), dtype=torch.float32).t(),       # not contiguous
           torch.zeros(8, dtype=torch.float32),                # not 2-D
           np.zeros((3, 8), dtype=np.float32)]                 # not a tensor
    for b in bad:
        with pytest.raises(ValueError):
            device_rows(b, "Y", 8, torch.float32, device_type="cpu")
    with pytest.raises(ValueError):
        device_rows(ok, "Y", 8, torch.float32, rows=4, device_type="cpu")
    with pytest.raises(ValueError):
        device_rows(ok, "Y", 8, torch.float32)                 # a host tensor for a device call


def test_host_shape():
    from paper_1812_06635_gb300.lasso import host_shape
    a = np.zeros((2, 5))
    assert host_shape(a, "Y", (2, 5)) is a
    with pytest.raises(ValueError):
        host_shape(a, "Y", (2, 6))


def test_every_entry_point_checks_its_buffers(pkg):
    d = pkg.Dictionary(None, 8, 16)                           # never reaches the library
    with pytest.raises(ValueError):
        d.solve(np.zeros(7), 0.5, 1e-6)
    with pytest.raises(ValueError):
        d.solve_batch_host(np.zeros((2, 7), dtype=np.float32), np.ones(2), 1e-6)
    with pytest.raises(ValueError):
        d.solve_batch_host(np.zeros((2, 8), dtype=np.float32), np.ones(3), 1e-6)
    with pytest.raises(ValueError):
        d.solve_batch_host(np.zeros(8, dtype=np.float32), np.ones(1), 1e-6)
    host = torch.zeros((2, 8), dtype=torch.float32)
    with pytest.raises(ValueError):
        d.solve_batch(host, torch.ones(2, dtype=torch.float64), 1e-6)
    with pytest.raises(ValueError):
        d.lambda_max(host)
    with pytest.raises(ValueError):
        d.backward(host, torch.zeros((2, 16)), torch.zeros((2, 16)))
