"""Seeded synthetic Lasso workloads shared by the oracle, the tests and the bench.

This package only draws inputs (dictionaries or their Kronecker factors, sparse
codes, signals, regularisation ratios).  It holds none of the solver's arithmetic:
no screening, no dual scaling, no soft-thresholding, no gap.
"""
from .gen import *  # noqa: F401,F403
