"""GB300-native screened Lasso solver (stable safe screening over approximate dictionaries).

The compute path is the CUDA library built from ``csrc/`` for sm_103a and reached through
the C ABI of ``include/lasso.h``; this package only marshals arguments.
"""
from .lasso import (Dictionary, LassoFn, Stats, make_opts, FISTA, ISTA, RULE_GAP, RULE_DST, RULE_STATIC,  # noqa: F401
                    LEVEL_BF16, LEVEL_FP8, LEVEL_KRON, LEVEL_F32, LEVEL_FAUST, STATUS)
from ._native import load, library_path, LassoError  # noqa: F401
