"""Python API over the C ABI: dictionaries, single and batched screened Lasso solves, and the
autograd wrapper.  PyTorch provides device memory and streams only; every step of the solve
runs in the library's CUDA kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import _native as nat

LEVEL_BF16, LEVEL_FP8, LEVEL_KRON, LEVEL_F32, LEVEL_FAUST = 2, 3, 4, 5, 6
FISTA, ISTA = 0, 1
RULE_GAP, RULE_DST, RULE_STATIC = 0, 1, 2
STATUS = {0: "ok", -1: "invalid_arg", -2: "cuda", -3: "nonfinite", -4: "maxiter", -5: "timeout",
          -6: "unsupported", -7: "nomem", 1: "warn_audit"}


def make_opts(**kw) -> nat.LassoOpts:
    """lasso_opts with the library defaults, overridden by keyword (same field names)."""
    o = nat.LassoOpts()
    nat.load().lasso_opts_default(C.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, v)
    return o


@dataclass
class Stats:
    passes: int
    level_passes: list
    kept_final: int
    lambda_max: float
    lam: float
    seconds: float
    launches: int = 0
    kernel_launches: list = None
    kernel_ms: list = None
    kernel_bytes: list = None
    level_atoms: list = None
    fp64_resolved: int = 0
    corr_chunk: int = 0
    corr_blocks_per_sm: int = 0
    level_rc: list = None

    KINDS = ("residual", "corr", "screen", "schedule", "kron", "tc_gemm")

    @staticmethod
    def of(s: nat.LassoStats) -> "Stats":
        return Stats(int(s.passes), [int(v) for v in s.level_passes], int(s.kept_final), float(s.lambda_max),
                     float(s.lambda_), float(s.seconds), int(s.launches), [int(v) for v in s.kernel_launches],
                     [float(v) for v in s.kernel_ms], [float(v) for v in s.kernel_bytes],
                     [float(v) for v in s.level_atoms], int(s.fp64_resolved), int(s.corr_chunk),
                     int(s.corr_blocks_per_sm), [float(v) for v in s.level_rc])


def _ptr(a) -> C.c_void_p:
    if a is None:
        return C.c_void_p(0)
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return C.c_void_p(a.ctypes.data)


def device_rows(t, name: str, cols: int, dtype, rows=None, device_type: str = "cuda", device=None):
    """Return ``t`` if it is a contiguous 2-D tensor of ``dtype`` with ``cols`` columns (and ``rows``
    rows when given) on a ``device_type`` device (``device`` when given); raise ValueError
    otherwise.  The library reads or writes exactly rows x cols elements through the pointer, so a
    buffer of another shape, type or device would be overrun.  ``device_type`` is "cuda" for real
    calls (host tests pass "cpu")."""
    import torch
    if not (isinstance(t, torch.Tensor) and t.device.type == device_type and t.dtype == dtype and t.dim() == 2
            and t.is_contiguous() and t.shape[1] == cols and (rows is None or t.shape[0] == rows)
            and (device is None or t.device == device)):
        shape = f"({'B' if rows is None else rows}, {cols})"
        where = str(device) if device is not None else device_type
        raise ValueError(f"{name} must be a contiguous {dtype} tensor of shape {shape} on {where}")
    return t


def host_shape(a: np.ndarray, name: str, shape: tuple):
    """Raise ValueError unless the host array ``a`` has exactly ``shape`` (the library copies that
    many elements from its pointer)."""
    if a.shape != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, not {a.shape}")
    return a


def noalloc_args(Y, out, N: int, device_type: str = "cuda"):
    """Validate the buffers of ``lasso_lambda_max_noalloc`` and return ``out`` (allocated when None).

    Y must be a contiguous float32 tensor of shape (B > 0, N) on a ``device_type`` device; out,
    when given, a contiguous float64 tensor of at least B entries on Y's device.  Raises
    ValueError otherwise.  ``device_type`` is "cuda" for real calls (host tests pass "cpu").
    """
    import torch
    if not (isinstance(Y, torch.Tensor) and Y.device.type == device_type and Y.dtype == torch.float32
            and Y.dim() == 2 and Y.is_contiguous() and Y.shape[1] == N and Y.shape[0] > 0):
        raise ValueError(f"Y must be a contiguous {device_type} float32 tensor of shape (B > 0, {N})")
    B = Y.shape[0]
    if out is None:
        return torch.empty(B, dtype=torch.float64, device=Y.device)
    if not (isinstance(out, torch.Tensor) and out.dtype == torch.float64 and out.is_contiguous()
            and out.numel() >= B and out.device == Y.device):
        raise ValueError(f"out must be a contiguous float64 tensor of at least {B} entries on {Y.device}")
    return out


class Dictionary:
    """A dictionary (exact A) and its ladder of approximations, owned by the library."""

    def __init__(self, handle: C.c_void_p, N: int, K: int):
        self._h = handle
        self.N, self.K = N, K

    # ------------------------------------------------------------ construction
    @classmethod
    def dense(cls, A, dtype: str = "f32", normalize: bool = False, atom_major: bool = False) -> "Dictionary":
        """A: host array, N x K with atoms as columns (or K x N rows = atoms if atom_major)."""
        lib = nat.load()
        npdt = np.float64 if dtype == "f64" else np.float32
        if hasattr(A, "detach"):
            A = A.detach().cpu().numpy()
        A = np.asarray(A, dtype=npdt)
        if atom_major:
            K, N = A.shape
            arr = np.ascontiguousarray(A)
            ld, am = N, 1
        else:
            N, K = A.shape
            arr = np.ascontiguousarray(A.T)   # atom-major copy (row j = atom j)
            ld, am = N, 1
        h = C.c_void_p()
        nat.check(lib.lasso_dict_create_dense(_ptr(arr), 0 if dtype == "f64" else 1, N, K, ld, am, int(normalize), 1,
                                              C.byref(h)), "lasso_dict_create_dense")
        return cls(h, N, K)

    @classmethod
    def kron(cls, Bf, Cf, normalize: bool = True) -> "Dictionary":
        """A = (sum_r B_r (x) C_r) diag(d); Bf: R x N1 x K1, Cf: R x N2 x K2.  d_j makes the atoms
        unit-norm when ``normalize`` (the default), else d = 1 (the Kronecker sum as given)."""
        lib = nat.load()
        Bf = np.ascontiguousarray(np.asarray(Bf, dtype=np.float32))
        Cf = np.ascontiguousarray(np.asarray(Cf, dtype=np.float32))
        R, N1, K1 = Bf.shape
        _, N2, K2 = Cf.shape
        h = C.c_void_p()
        nat.check(lib.lasso_dict_create_kron(_ptr(Bf), _ptr(Cf), R, N1, K1, N2, K2, int(normalize), 1,
                                             C.byref(h)),
                  "lasso_dict_create_kron")
        return cls(h, N1 * N2, K1 * K2)

    def add_level(self, kind: int, param: int = 0) -> "Dictionary":
        nat.check(nat.load().lasso_dict_add_level(self._h, kind, param), "lasso_dict_add_level")
        return self

    def add_faust_level(self, factors) -> "Dictionary":
        """Append A~ = S_0 S_1 ... S_{J-1} (sparse factors, coarsest levels first).  ``factors``:
        CSR matrices (anything with ``shape``, ``indptr``, ``indices``, ``data``, e.g. scipy's),
        column indices increasing within each row; values are stored as FP32."""
        dims = [int(factors[0].shape[0])] + [int(f.shape[1]) for f in factors]
        for f, (r, c) in zip(factors, zip(dims[:-1], dims[1:])):
            if tuple(f.shape) != (r, c):
                raise ValueError("inner dimensions of consecutive factors must agree")
        d = np.asarray(dims, dtype=np.int64)
        ip = np.ascontiguousarray(np.concatenate([np.asarray(f.indptr, np.int64) for f in factors]))
        ix = np.ascontiguousarray(np.concatenate([np.asarray(f.indices, np.int32) for f in factors]))
        vv = np.ascontiguousarray(np.concatenate([np.asarray(f.data, np.float32) for f in factors]))
        nat.check(nat.load().lasso_dict_add_level_faust(self._h, len(factors), _ptr(d), _ptr(ip), _ptr(ix), _ptr(vv)),
                  "lasso_dict_add_level_faust")
        return self

    def set_rc(self, level: int, rc: float) -> "Dictionary":
        nat.check(nat.load().lasso_dict_set_rc(self._h, level, rc), "lasso_dict_set_rc")
        return self

    def prepare(self, L: float = 0.0) -> "Dictionary":
        nat.check(nat.load().lasso_dict_prepare(self._h, float(L)), "lasso_dict_prepare")
        return self

    def info(self) -> dict:
        inf = nat.LassoDictInfo()
        nat.check(nat.load().lasso_dict_info(self._h, C.byref(inf)), "lasso_dict_info")
        n = inf.n_levels
        return {"N": inf.N, "K": inf.K, "n_levels": n, "L": inf.L, "kind": list(inf.kind[:n]),
                "rc": list(inf.rc[:n]), "eps_mean": list(inf.eps_mean[:n]), "eps_max": list(inf.eps_max[:n])}

    def level_data(self, level: int, atoms: bool = True):
        """(eps (K,), dequantised atoms (K x N, row j = atom j) or None) of a level, as FP64."""
        eps = np.zeros(self.K)
        at = np.zeros((self.K, self.N)) if atoms else None
        nat.check(nat.load().lasso_dict_level_host(self._h, level, _ptr(eps), _ptr(at)), "lasso_dict_level_host")
        return eps, at

    def close(self):
        if self._h:
            nat.load().lasso_dict_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------ solves
    def solve(self, y, lam: float, tol: float = 1e-6, **opts):
        """One signal, host buffers.  Returns (x, rel_gap, kept, Stats); status errors raise."""
        lib = nat.load()
        y = host_shape(np.ascontiguousarray(np.asarray(y, dtype=np.float64)), "y", (self.N,))
        x = np.zeros(self.K)
        kept = np.zeros(self.K, dtype=np.int32)
        gap = C.c_double()
        nk = C.c_int64()
        st = nat.LassoStats()
        o = make_opts(**opts)
        code = lib.lasso_solve(self._h, _ptr(y), float(lam), float(tol), C.byref(o), _ptr(x), C.byref(gap),
                               _ptr(kept), C.byref(nk), C.byref(st))
        nat.check(code, "lasso_solve", ok=(0, 1))
        return x, gap.value, kept[: nk.value].copy(), Stats.of(st)

    def solve_batch(self, Y, lambdas, tol: float = 1e-6, stream=None, kept=None, **opts):
        """Batch on the device.  Y: torch CUDA float32 (B x N); lambdas: torch CUDA float64 (B,).

        Returns (X (B x K float32), gaps (B float64), status (B int32), iters (B int32), Stats).
        ``kept``: optional CUDA uint8 tensor (B x K, contiguous) that receives the preserved sets
        at exit (1 = preserved, 0 = rejected by a safe test).
        """
        import torch
        lib = nat.load()
        device_rows(Y, "Y", self.N, torch.float32)
        B = Y.shape[0]
        if kept is not None:
            if not (kept.is_cuda and kept.dtype == torch.uint8 and kept.is_contiguous()
                    and tuple(kept.shape) == (B, self.K) and kept.device == Y.device):
                raise ValueError(f"kept must be a contiguous CUDA uint8 tensor of shape ({B}, {self.K})")
            opts["kept_mask"] = kept.data_ptr()
        lam = torch.as_tensor(lambdas, dtype=torch.float64).to(device=Y.device).contiguous()
        if lam.dim() != 1 or lam.numel() != B:
            raise ValueError(f"lambdas must hold one value per signal ({B}), not shape {tuple(lam.shape)}")
        X = torch.empty((B, self.K), dtype=torch.float32, device=Y.device)
        gaps = torch.empty(B, dtype=torch.float64, device=Y.device)
        status = torch.empty(B, dtype=torch.int32, device=Y.device)
        iters = torch.empty(B, dtype=torch.int32, device=Y.device)
        st = nat.LassoStats()
        o = make_opts(**opts)
        s = stream if stream is not None else torch.cuda.current_stream(Y.device)
        code = lib.lasso_solve_batch(self._h, _ptr(Y), _ptr(lam), B, float(tol), C.byref(o), _ptr(X), _ptr(gaps),
                                     _ptr(status), _ptr(iters), C.c_void_p(s.cuda_stream), C.byref(st))
        nat.check(code, "lasso_solve_batch", ok=(0, -4, -5))
        return X, gaps, status, iters, Stats.of(st)

    def solve_batch_host(self, Y, lambdas, tol: float = 1e-6, kept=None, **opts):
        """Batch with host buffers (the library copies in and out).  ``kept``: optional numpy
        uint8 array (B x K, C-contiguous) that receives the preserved sets at exit."""
        lib = nat.load()
        Y = np.ascontiguousarray(np.asarray(Y, dtype=np.float32))
        if Y.ndim != 2:
            raise ValueError(f"Y must be a B x {self.N} array, not shape {Y.shape}")
        B = Y.shape[0]
        host_shape(Y, "Y", (B, self.N))
        lam = host_shape(np.ascontiguousarray(np.asarray(lambdas, dtype=np.float64)), "lambdas", (B,))
        if kept is not None:
            if not (isinstance(kept, np.ndarray) and kept.dtype == np.uint8 and kept.flags.c_contiguous
                    and kept.shape == (B, self.K)):
                raise ValueError(f"kept must be a C-contiguous numpy uint8 array of shape ({B}, {self.K})")
            opts["kept_mask"] = kept.ctypes.data
        X = np.zeros((B, self.K), dtype=np.float32)
        gaps = np.zeros(B)
        status = np.zeros(B, dtype=np.int32)
        st = nat.LassoStats()
        o = make_opts(**opts)
        code = lib.lasso_solve_batch_host(self._h, _ptr(Y), _ptr(lam), B, float(tol), C.byref(o), _ptr(X),
                                          _ptr(gaps), _ptr(status), C.byref(st))
        nat.check(code, "lasso_solve_batch_host", ok=(0, -4, -5))
        return X, gaps, status, Stats.of(st)

    def lambda_max(self, Y):
        import torch
        device_rows(Y, "Y", self.N, torch.float32)
        B = Y.shape[0]
        out = torch.empty(B, dtype=torch.float64, device=Y.device)
        s = torch.cuda.current_stream(Y.device)
        nat.check(nat.load().lasso_lambda_max(self._h, _ptr(Y), B, _ptr(out), C.c_void_p(s.cuda_stream)),
                  "lasso_lambda_max")
        return out

    def lambda_max_noalloc(self, Y, out=None):
        """lambda_max through the allocation-free entry point; ``out`` (B float64) may be given.

        The kernel reads B x N floats from ``Y`` and writes B doubles to ``out`` by raw device
        pointer, so both are checked first (``noalloc_args``): a wrong dtype, shape, layout or
        device would otherwise make it read or write outside the tensors.
        """
        import torch
        out = noalloc_args(Y, out, self.N)
        s = torch.cuda.current_stream(Y.device)
        with torch.cuda.device(Y.device):
            nat.check(nat.load().lasso_lambda_max_noalloc(self._h, _ptr(Y), Y.shape[0], _ptr(out),
                                                          C.c_void_p(s.cuda_stream)), "lasso_lambda_max_noalloc")
        return out

    def backward(self, Y, X, G, want_dA: bool = True):
        """(dL/dY (B x N), dL/dA (K x N atom-major, summed over the batch) or None) for dL/dX = G."""
        import torch
        device_rows(Y, "Y", self.N, torch.float32)
        B = Y.shape[0]
        X = device_rows(X.contiguous(), "X", self.K, torch.float32, rows=B, device=Y.device)
        G = device_rows(G.contiguous(), "G", self.K, torch.float32, rows=B, device=Y.device)
        dY = torch.empty_like(Y)
        dA = torch.zeros((self.K, self.N), dtype=torch.float32, device=Y.device) if want_dA else None
        s = torch.cuda.current_stream(Y.device)
        nat.check(nat.load().lasso_backward(self._h, _ptr(Y), _ptr(X), _ptr(G), B, _ptr(dY),
                                            _ptr(dA), C.c_void_p(s.cuda_stream)), "lasso_backward")
        return dY, dA


def _autograd():
    import torch

    class LassoFn(torch.autograd.Function):
        """x* = argmin 1/2||A x - y||^2 + lam ||x||_1 per row of Y, differentiable in Y and A.

        Forward: ``Dictionary.solve_batch``; backward: the support-system adjoint (lambda fixed).
        ``A`` is the dense N x K tensor the dictionary was built from (its gradient is returned
        as N x K); pass None to skip dL/dA.
        """

        @staticmethod
        def forward(ctx, Y, A, dictionary, lambdas, tol, opts):
            X, gaps, status, iters, _ = dictionary.solve_batch(Y.contiguous(), lambdas, tol, **(opts or {}))
            bad = torch.nonzero(status != 0).flatten()
            if bad.numel():
                # a signal that stopped on the pass limit, the time limit or a non-finite value
                # holds a partial point: the support adjoint would not be the minimiser's derivative
                b = int(bad[0])
                raise nat.LassoError(int(status[b]), f"LassoFn.forward: {bad.numel()} signal(s) not solved to tol "
                                                     f"(first: signal {b})")
            ctx.dictionary = dictionary
            ctx.want_dA = A is not None and A.requires_grad
            ctx.save_for_backward(Y, X)
            return X

        @staticmethod
        def backward(ctx, gX):
            Y, X = ctx.saved_tensors
            dY, dA = ctx.dictionary.backward(Y.contiguous(), X, gX.contiguous().float(), want_dA=ctx.want_dA)
            return dY, (dA.t().contiguous() if dA is not None else None), None, None, None, None

    return LassoFn


class _LazyFn:
    _fn = None

    def apply(self, *args):
        if _LazyFn._fn is None:
            _LazyFn._fn = _autograd()
        return _LazyFn._fn.apply(*args)


LassoFn = _LazyFn()
