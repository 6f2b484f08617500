"""ctypes binding of the C ABI declared in ``include/lasso.h`` (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

_lib = None


class LassoOpts(C.Structure):
    _fields_ = [
        ("Gamma", C.c_double),
        ("algo", C.c_int),
        ("rule", C.c_int),
        ("screen_every", C.c_int),
        ("max_iter", C.c_int),
        ("lambda_relative", C.c_int),
        ("final_fp64", C.c_int),
        ("certify_full", C.c_int),
        ("passes_per_sync", C.c_int),
        ("tensor_cores", C.c_int),
        ("tau", C.c_double),
        ("time_limit_s", C.c_double),
        ("profile", C.c_int),
        ("full_gap", C.c_int),
        ("tc_exact", C.c_int),
        ("split_level", C.c_int),
        ("fp64_fallback", C.c_int),
        ("autotune", C.c_int),
        ("kept_mask", C.c_void_p),
    ]


class LassoStats(C.Structure):
    _fields_ = [
        ("passes", C.c_int64),
        ("level_passes", C.c_int64 * 8),
        ("kept_final", C.c_int64),
        ("lambda_max", C.c_double),
        ("lambda_", C.c_double),
        ("seconds", C.c_double),
        ("launches", C.c_int64),
        ("kernel_launches", C.c_int64 * 6),
        ("kernel_ms", C.c_double * 6),
        ("kernel_bytes", C.c_double * 6),
        ("level_atoms", C.c_double * 8),
        ("fp64_resolved", C.c_int64),
        ("corr_chunk", C.c_int64),
        ("corr_blocks_per_sm", C.c_int64),
        ("level_rc", C.c_double * 8),
    ]


class LassoDictInfo(C.Structure):
    _fields_ = [
        ("N", C.c_int64),
        ("K", C.c_int64),
        ("n_levels", C.c_int),
        ("L", C.c_double),
        ("kind", C.c_int * 8),
        ("rc", C.c_double * 8),
        ("eps_mean", C.c_double * 8),
        ("eps_max", C.c_double * 8),
    ]


P = C.c_void_p
I64 = C.c_int64
PI32 = C.POINTER(C.c_int32)
PI64 = C.POINTER(C.c_int64)
PD = C.POINTER(C.c_double)

# (name, restype, argtypes) for every function of include/lasso.h
SIGNATURES = [
    ("lasso_dict_create_dense", C.c_int, [P, C.c_int, I64, I64, I64, C.c_int, C.c_int, C.c_int, C.POINTER(P)]),
    ("lasso_dict_create_kron", C.c_int, [P, P, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                         C.POINTER(P)]),
    ("lasso_dict_add_level", C.c_int, [P, C.c_int, C.c_int]),
    ("lasso_dict_add_level_faust", C.c_int, [P, C.c_int, P, P, P, P]),
    ("lasso_dict_set_rc", C.c_int, [P, C.c_int, C.c_double]),
    ("lasso_dict_prepare", C.c_int, [P, C.c_double]),
    ("lasso_dict_info", C.c_int, [P, C.POINTER(LassoDictInfo)]),
    ("lasso_dict_level_host", C.c_int, [P, C.c_int, P, P]),
    ("lasso_dict_destroy", None, [P]),
    ("lasso_opts_default", None, [C.POINTER(LassoOpts)]),
    ("lasso_solve", C.c_int, [P, P, C.c_double, C.c_double, C.POINTER(LassoOpts), P, PD, P, PI64,
                              C.POINTER(LassoStats)]),
    ("lasso_solve_batch", C.c_int, [P, P, P, I64, C.c_double, C.POINTER(LassoOpts), P, P, P, P, P,
                                    C.POINTER(LassoStats)]),
    ("lasso_solve_batch_host", C.c_int, [P, P, P, I64, C.c_double, C.POINTER(LassoOpts), P, P, P,
                                         C.POINTER(LassoStats)]),
    ("lasso_lambda_max", C.c_int, [P, P, I64, P, P]),
    ("lasso_lambda_max_noalloc", C.c_int, [P, P, I64, P, P]),
    ("lasso_backward", C.c_int, [P, P, P, P, I64, P, P, P]),
    ("lasso_tc_selftest", C.c_int, [C.c_int, I64, I64, I64, PD, PD]),
    ("lasso_probe_l2_read", C.c_int, [I64, C.c_int, PD]),
    ("lasso_strerror", C.c_char_p, [C.c_int]),
    ("lasso_build_info", C.c_char_p, []),
]


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load the compiled library (once).  Raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"the CUDA library {path} is missing: run "
                           "`python -c 'import __graft_entry__ as g; g.build()'` first (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LassoError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = load().lasso_strerror(code).decode()
        super().__init__(f"{what}: status {code} ({msg})")


def check(code: int, what: str, ok=(0,)):
    if code not in ok:
        raise LassoError(code, what)
    return code
