"""Seeded generators for the five Lasso workloads and their small variants.

Every workload follows the experimental recipe of Section V (Bernoulli-Gaussian
sparse codes, Gaussian dictionaries with unit-norm atoms, sums of Kronecker
products for the structured case) at the sizes the build is measured on:

  c1  dense 100 x 500 FP64, 25-sparse x0, y = A x0 + N(0, 0.01^2), lambda = 0.5 lambda_max
  c2  sum of R = 4 Kronecker terms, B_r, C_r 32 x 64 (N = 1024, K = 4096), x0 Bernoulli(0.02),
      20 dB SNR, lambda / lambda_max in {0.3, 0.5, 0.8}
  c3  dense 2048 x 8192, 4096 signals, x0 Bernoulli(p_i), p_i ~ U[0.01, 0.05], y = A x0,
      lambda_i / lambda_max ~ U[0.1, 0.9]
  c4  dense 1024 x 4096, 256 signals, x0 and x_target Bernoulli(0.02), 20 dB SNR, lambda = 0.5 lambda_max
  c5  sum of R = 8 Kronecker terms, B_r 64 x 256, C_r 128 x 256 (N = 8192, K = 65536),
      512 signals, x0 Bernoulli(0.005), y = A x0, lambda / lambda_max ~ U[0.2, 0.7]

Randomness: numpy PCG64 seeded through ``SeedSequence([seed, config, stream, index])``,
so signal ``i`` of a batch depends only on ``(seed, i)`` and any prefix of a batch
is a valid smaller batch.  Values that the GPU path stores in FP32 (dictionaries,
factors and signals of c2..c5) are rounded to FP32 here, so both the oracle and
the GPU see exactly the same numbers; arrays are returned as float64 holding
those values.

The Kronecker dictionaries are defined as ``A = (sum_r B_r (x) C_r) diag(d)`` with
``d_j`` the inverse FP64 column norm, using the row-major vectorisation
``(B (x) C)[n1 * N2 + n2, k1 * K2 + k2] = B[n1, k1] * C[n2, k2]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "DenseWorkload", "KronWorkload", "rng_for",
    "gaussian_unit_columns", "bernoulli_gaussian",
    "c1", "c2", "c3", "c4", "c5", "dense_small", "kron_small", "orthonormal_case",
    "paper_dense", "paper_kron", "FaustWorkload", "meg_faust", "faust_small",
]

_CFG = {"c1": 1, "c2": 2, "c3": 3, "c4": 4, "c5": 5, "dense_small": 6, "kron_small": 7, "ortho": 8,
        "paper_dense": 9, "paper_kron": 10, "meg_faust": 11, "faust_small": 12, "paper_kron_example": 13}
_DICT, _SIGNAL = 0, 1


def rng_for(seed: int, cfg: str, stream: int, index: int = 0) -> np.random.Generator:
    """Independent PCG64 stream for (seed, config, stream, index)."""
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, _CFG[cfg], stream, index])))


@dataclass
class DenseWorkload:
    """A dense dictionary problem: columns of ``A`` are the atoms."""
    name: str
    A: np.ndarray                 # N x K, float64 array (FP32-representable unless fp64=True)
    Y: np.ndarray                 # B x N signals
    lam_ratio: np.ndarray         # B, lambda_i / lambda_max,i
    tol: float
    supports: list = field(default_factory=list)   # support of x0 per signal
    coefs: list = field(default_factory=list)      # values of x0 on its support
    x_target: np.ndarray | None = None             # B x K (c4 only)
    fp64: bool = False

    @property
    def N(self):
        return self.A.shape[0]

    @property
    def K(self):
        return self.A.shape[1]


@dataclass
class KronWorkload:
    """A sum-of-Kronecker dictionary given by its factors (``A`` is not formed)."""
    name: str
    Bf: np.ndarray                # R x N1 x K1 (FP32 values in float64)
    Cf: np.ndarray                # R x N2 x K2
    Y: np.ndarray                 # B x N
    lam_ratio: np.ndarray
    tol: float
    supports: list = field(default_factory=list)
    coefs: list = field(default_factory=list)

    @property
    def R(self):
        return self.Bf.shape[0]

    @property
    def N(self):
        return self.Bf.shape[1] * self.Cf.shape[1]

    @property
    def K(self):
        return self.Bf.shape[2] * self.Cf.shape[2]


def _f32(a):
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def gaussian_unit_columns(N: int, K: int, rng: np.random.Generator, fp32: bool = True) -> np.ndarray:
    A = rng.standard_normal((N, K))
    A /= np.sqrt(np.einsum("nk,nk->k", A, A))[None, :]
    return _f32(A) if fp32 else A


def bernoulli_gaussian(K: int, p: float, rng: np.random.Generator):
    """Support drawn i.i.d. Bernoulli(p), values N(0, 1); at least one nonzero."""
    mask = rng.random(K) < p
    idx = np.flatnonzero(mask)
    if idx.size == 0:
        idx = np.array([int(rng.integers(K))])
    return idx, rng.standard_normal(idx.size)


def _snr20_noise(clean: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    """White noise at 20 dB SNR: sigma = ||A x0|| / (10 sqrt(N))."""
    sigma = np.linalg.norm(clean) / (10.0 * np.sqrt(clean.size))
    return sigma * rng.standard_normal(clean.size)


# ----------------------------------------------------------------------------- dense configs

def c1(seed: int = 0) -> DenseWorkload:
    """Plain FP64 problem: 100 x 500, 25-sparse x0, noise N(0, 0.01^2), lambda = 0.5 lambda_max."""
    N, K = 100, 500
    A = gaussian_unit_columns(N, K, rng_for(seed, "c1", _DICT), fp32=False)
    r = rng_for(seed, "c1", _SIGNAL, 0)
    idx = np.sort(r.choice(K, size=25, replace=False))
    vals = r.standard_normal(25)
    y = A[:, idx] @ vals + 0.01 * r.standard_normal(N)
    return DenseWorkload("c1", A, y[None, :], np.array([0.5]), 1e-8, [idx], [vals], fp64=True)


def _dense_batch(name, N, K, n_signals, seed, p_range, ratio_range, snr20, first=0, fixed_ratio=None,
                 with_target=False):
    A = gaussian_unit_columns(N, K, rng_for(seed, name, _DICT), fp32=True)
    Y = np.empty((n_signals, N))
    ratios = np.empty(n_signals)
    sups, cfs = [], []
    xt = np.zeros((n_signals, K)) if with_target else None
    for b in range(n_signals):
        r = rng_for(seed, name, _SIGNAL, first + b)
        p = r.uniform(*p_range) if isinstance(p_range, tuple) else p_range
        idx, vals = bernoulli_gaussian(K, p, r)
        y = A[:, idx] @ vals
        if snr20:
            y = y + _snr20_noise(y, r)
        Y[b] = y
        ratios[b] = fixed_ratio if fixed_ratio is not None else r.uniform(*ratio_range)
        sups.append(idx)
        cfs.append(vals)
        if with_target:
            ti, tv = bernoulli_gaussian(K, p, r)
            xt[b, ti] = tv
    return A, _f32(Y), ratios, sups, cfs, xt


def c3(n_signals: int = 4096, seed: int = 0, first: int = 0, N: int = 2048, K: int = 8192) -> DenseWorkload:
    """Batched mixed-precision workload: 2048 x 8192, p_i ~ U[0.01, 0.05], lambda_i/lambda_max ~ U[0.1, 0.9]."""
    A, Y, ratios, sups, cfs, _ = _dense_batch("c3", N, K, n_signals, seed, (0.01, 0.05), (0.1, 0.9), False,
                                              first=first)
    return DenseWorkload("c3", A, Y, ratios, 1e-6, sups, cfs)


def c4(n_signals: int = 256, seed: int = 0, first: int = 0, N: int = 1024, K: int = 4096) -> DenseWorkload:
    """Differentiation workload: 1024 x 4096, x0 and x_target Bernoulli(0.02), 20 dB, lambda = 0.5 lambda_max."""
    A, Y, ratios, sups, cfs, xt = _dense_batch("c4", N, K, n_signals, seed, 0.02, None, True, first=first,
                                               fixed_ratio=0.5, with_target=True)
    return DenseWorkload("c4", A, Y, ratios, 1e-6, sups, cfs, x_target=xt)


def dense_small(N: int = 64, K: int = 256, n_signals: int = 8, seed: int = 0, p=(0.01, 0.05),
                ratio=(0.1, 0.9), snr20: bool = False) -> DenseWorkload:
    """Small c3-shaped batch for parity tests (sizes chosen by the caller)."""
    A, Y, ratios, sups, cfs, _ = _dense_batch("dense_small", N, K, n_signals, seed, p, ratio, snr20)
    return DenseWorkload("dense_small", A, Y, ratios, 1e-6, sups, cfs)


def orthonormal_case(n: int = 64, seed: int = 0):
    """Square dictionary with orthonormal columns (QR of a Gaussian matrix) and a Gaussian y."""
    r = rng_for(seed, "ortho", _DICT)
    Q, _ = np.linalg.qr(r.standard_normal((n, n)))
    y = r.standard_normal(n)
    return Q, y


# ----------------------------------------------------------------------------- Kronecker configs

def kron_column_norms(Bf: np.ndarray, Cf: np.ndarray) -> np.ndarray:
    """FP64 norms of the atoms of sum_r B_r (x) C_r (row-major atom index k1 * K2 + k2).

    ||sum_r b_r (x) c_r||^2 = sum_{r,s} (b_r . b_s)(c_r . c_s) for the columns b_r = B_r[:, k1], c_r = C_r[:, k2].
    """
    GB = np.einsum("rnk,snk->rsk", Bf, Bf)
    GC = np.einsum("rnk,snk->rsk", Cf, Cf)
    return np.sqrt(np.einsum("rsa,rsb->ab", GB, GC).reshape(-1))


def _kron_signals(name, Bf, Cf, n_signals, seed, p, ratio_range, snr20, first=0, fixed_ratio=None):
    R, N1, K1 = Bf.shape
    _, N2, K2 = Cf.shape
    N, K = N1 * N2, K1 * K2
    d = 1.0 / kron_column_norms(Bf, Cf)
    Y = np.empty((n_signals, N))
    ratios = np.empty(n_signals)
    sups, cfs = [], []
    for b in range(n_signals):
        r = rng_for(seed, name, _SIGNAL, first + b)
        idx, vals = bernoulli_gaussian(K, p, r)
        X = np.zeros(K)
        X[idx] = vals * d[idx]
        X = X.reshape(K1, K2)
        y = np.einsum("rnk,kl,rml->nm", Bf, X, Cf, optimize=True).reshape(-1)  # sum_r B_r X C_r^T, row-major vec
        if snr20:
            y = y + _snr20_noise(y, r)
        Y[b] = y
        ratios[b] = fixed_ratio if fixed_ratio is not None else r.uniform(*ratio_range)
        sups.append(idx)
        cfs.append(vals)
    return _f32(Y), ratios, sups, cfs


def _kron_factors(name, R, N1, K1, N2, K2, seed, decay=None):
    r = rng_for(seed, name, _DICT)
    Bf = r.standard_normal((R, N1, K1))
    Cf = r.standard_normal((R, N2, K2))
    if decay is not None:
        Bf *= (decay ** np.arange(R))[:, None, None]
    return _f32(Bf), _f32(Cf)


def c2(seed: int = 0, lam_ratio: float = 0.5, decay: float | None = None, n_signals: int = 1) -> KronWorkload:
    """Structured workload: R = 4 terms of 32 x 64 factors, x0 Bernoulli(0.02), 20 dB SNR.

    ``seed`` selects the realisation (the paper averages 25); the dictionary is shared
    across realisations of the same (decay) variant.  ``decay`` = rho weights term r by
    rho^(r-1) (the easy/moderate/hard error profiles of Section V-A); None is the literal
    equal-weight configuration.
    """
    Bf, Cf = _kron_factors("c2", 4, 32, 64, 32, 64, 0, decay)
    Y, ratios, sups, cfs = _kron_signals("c2", Bf, Cf, n_signals, seed, 0.02, None, True, fixed_ratio=lam_ratio)
    return KronWorkload("c2" if decay is None else f"c2-decay{decay}", Bf, Cf, Y, ratios, 1e-6, sups, cfs)


def c5(n_signals: int = 512, seed: int = 0, first: int = 0, decay: float | None = None) -> KronWorkload:
    """Large structured workload: R = 8 terms, B_r 64 x 256, C_r 128 x 256 (N = 8192, K = 65536)."""
    Bf, Cf = _kron_factors("c5", 8, 64, 256, 128, 256, seed, decay)
    Y, ratios, sups, cfs = _kron_signals("c5", Bf, Cf, n_signals, seed, 0.005, (0.2, 0.7), False, first=first)
    return KronWorkload("c5" if decay is None else f"c5-decay{decay}", Bf, Cf, Y, ratios, 1e-6, sups, cfs)


def kron_small(R: int = 3, N1: int = 4, K1: int = 6, N2: int = 5, K2: int = 7, n_signals: int = 4, seed: int = 0,
               p: float = 0.1, ratio=(0.2, 0.8), decay: float | None = None) -> KronWorkload:
    """Small Kronecker problem for parity tests (sizes chosen by the caller)."""
    Bf, Cf = _kron_factors("kron_small", R, N1, K1, N2, K2, seed, decay)
    Y, ratios, sups, cfs = _kron_signals("kron_small", Bf, Cf, n_signals, seed, p, ratio, False)
    return KronWorkload("kron_small", Bf, Cf, Y, ratios, 1e-6, sups, cfs)


# ----------------------------------------------------------------------------- Section V setting

def _unit_rows(Y):
    n = np.linalg.norm(Y, axis=1, keepdims=True)
    return Y / np.where(n > 0, n, 1.0)


def paper_dense(n_signals: int = 25, seed: int = 0, N: int = 2500, K: int = 10000) -> DenseWorkload:
    """The experiments' setting (Section V) with a Gaussian dictionary: N = 2500, K = 10000, unit-norm
    y = A x with x Bernoulli(0.02)-Gaussian, 25 realisations; lambda ratios are chosen by the caller."""
    A, Y, ratios, sups, cfs, _ = _dense_batch("paper_dense", N, K, n_signals, seed, 0.02, None, False,
                                              fixed_ratio=1.0)
    return DenseWorkload("paper_dense", A, _f32(_unit_rows(Y)), ratios, 1e-6, sups, cfs)


def paper_kron(decay: float, n_signals: int = 25, seed: int = 0, R: int = 4) -> KronWorkload:
    """The experiments' setting with a structured dictionary: A = (sum_{r<R} w_r B_r (x) C_r) diag(d),
    B_r, C_r 50 x 100 (N = 2500, K = 10000), term weights w_r = decay^r (small decay: well approximated
    by few terms, the paper's easy scenario; large decay: hard), unit-norm y = A x, x Bernoulli(0.02).
    R = 4 by default; the Section IV example uses more terms so that truncations to 5, 10, 15 and 20
    of them (relative complexity 0.03 per term) form its four approximations."""
    name = "paper_kron" if R == 4 else "paper_kron_example"
    Bf, Cf = _kron_factors(name, R, 50, 100, 50, 100, seed, decay)
    Y, ratios, sups, cfs = _kron_signals(name, Bf, Cf, n_signals, seed, 0.02, None, False, fixed_ratio=1.0)
    return KronWorkload(f"{name}{R}-decay{decay}", Bf, Cf, _f32(_unit_rows(Y)), ratios, 1e-6, sups, cfs)


# ----------------------------------------------------------------------------- sparse-factor products

@dataclass
class FaustWorkload:
    """A dense dictionary with a ladder of products of sparse factors approximating it.

    ``levels[i]`` is a list of J scipy CSR matrices S_0 (N x n_1), ..., S_{J-1} (n_{J-1} x K) whose
    product approximates ``A`` column by column (the column scale of ``A`` is already folded into
    the last factor).  Factor values and ``A`` are FP32 values held in float64.
    """
    name: str
    A: np.ndarray                 # N x K exact dictionary (unit columns up to FP32 rounding)
    levels: list                  # coarsest first
    Y: np.ndarray
    lam_ratio: np.ndarray
    tol: float
    supports: list = field(default_factory=list)
    coefs: list = field(default_factory=list)

    @property
    def N(self):
        return self.A.shape[0]

    @property
    def K(self):
        return self.A.shape[1]


def _ranked_rows(rows: int, cols: int, per_row: int, decay: float, rng: np.random.Generator):
    """Column indices (distinct within a row) and values of a row-sparse matrix whose r-th entry of
    every row has scale decay^r, so that keeping the first m entries of each row keeps the largest."""
    ci = np.stack([rng.choice(cols, per_row, replace=False) for _ in range(rows)])
    v = rng.standard_normal((rows, per_row)) * (decay ** np.arange(per_row))[None, :]
    return ci, v


def _csr(rows: int, cols: int, r_idx, c_idx, vals):
    """Canonical CSR matrix (column indices sorted within each row, int32) from triplets, built with
    an explicit lexicographic sort so that no in-place index sorting is relied on."""
    import scipy.sparse as sps
    r_idx = np.asarray(r_idx, np.int64)
    c_idx = np.asarray(c_idx, np.int64)
    order = np.lexsort((c_idx, r_idx))
    indptr = np.zeros(rows + 1, np.int64)
    np.cumsum(np.bincount(r_idx, minlength=rows), out=indptr[1:])
    return sps.csr_matrix((np.asarray(vals, np.float64)[order].copy(), c_idx[order].astype(np.int32),
                           indptr.astype(np.int32)), shape=(rows, cols))


def _csr_first(ci: np.ndarray, v: np.ndarray, m: int, cols: int, col_scale=None, transpose=False):
    """CSR matrix of the first m entries of every row (FP32 values); optionally transposed (for
    factors drawn column by column) and scaled per column of the result."""
    rows = ci.shape[0]
    r_idx = np.repeat(np.arange(rows), m)
    c_idx = ci[:, :m].reshape(-1)
    vals = v[:, :m].reshape(-1)
    if transpose:
        rows, cols, r_idx, c_idx = cols, rows, c_idx, r_idx
    if col_scale is not None:
        vals = vals * np.asarray(col_scale)[c_idx]
    return _csr(rows, cols, r_idx, c_idx, _f32(vals))


def _faust_problem(name, N, K, n_signals, seed, first, decay, sigma, per_row, per_col, levels, n_active,
                   ratio, unit_y):
    """A = normalise(S_0 S_1 S_2 + E): S_0, S_1 N x N with `per_row` entries per row, S_2 N x K with
    `per_col` entries per column (entry scales decaying with rank), E dense Gaussian with relative
    column norm `sigma` (the part no sparse product captures).  Level (m0, m2) keeps the first m0
    entries of each row of S_0, S_1 and the first m2 of each column of S_2, scaled by the same d."""
    r = rng_for(seed, name, _DICT)
    c0, v0 = _ranked_rows(N, N, per_row, decay, r)
    c1, v1 = _ranked_rows(N, N, per_row, decay, r)
    c2, v2 = _ranked_rows(K, N, per_col, decay, r)
    full = [_csr_first(c0, v0, per_row, N), _csr_first(c1, v1, per_row, N),
            _csr_first(c2, v2, per_col, N, transpose=True)]
    P = (full[0] @ (full[1] @ full[2].toarray()))
    E = r.standard_normal((N, K)) * (np.linalg.norm(P, axis=0) / np.sqrt(N))[None, :] * sigma
    A_raw = P + E
    d = 1.0 / np.linalg.norm(A_raw, axis=0)
    A = _f32(A_raw * d[None, :])
    ladder = [[_csr_first(c0, v0, m0, N), _csr_first(c1, v1, m0, N),
               _csr_first(c2, v2, m2, N, col_scale=d, transpose=True)] for (m0, m2) in levels]
    Y = np.empty((n_signals, N))
    sups, cfs = [], []
    for b in range(n_signals):
        rs = rng_for(seed, name, _SIGNAL, first + b)
        idx = np.sort(rs.choice(K, n_active, replace=False))
        vals = rs.standard_normal(n_active)
        Y[b] = A[:, idx] @ vals
        sups.append(idx)
        cfs.append(vals)
    if unit_y:
        Y = _unit_rows(Y)
    return A, ladder, _f32(Y), np.full(n_signals, ratio), sups, cfs


def meg_faust(n_signals: int = 50, seed: int = 0, first: int = 0, N: int = 204, K: int = 8193,
              decay: float = 0.45, sigma: float = 0.055, levels=((3, 4), (4, 5), (5, 7), (6, 8))) -> FaustWorkload:
    """Stand-in for the source-localisation experiment of Section VI: a 204 x 8193 operator with four
    sparse-factor approximations of decreasing error (mean eps_j from about 0.2 down to the 0.055
    floor of the dense part), 8 active sources with N(0, 1) weights, y = A x unit-norm,
    lambda = 0.1 lambda_max, 50 runs."""
    A, ladder, Y, ratios, sups, cfs = _faust_problem("meg_faust", N, K, n_signals, seed, first, decay, sigma, 12, 16,
                                                    levels, 8, 0.1, True)
    return FaustWorkload("meg_faust", A, ladder, Y, ratios, 1e-6, sups, cfs)


def faust_small(N: int = 48, K: int = 160, n_signals: int = 4, seed: int = 0, decay: float = 0.45,
                sigma: float = 0.05, levels=((2, 2), (3, 4)), n_active: int = 4, ratio: float = 0.2) -> FaustWorkload:
    """Small sparse-factor problem for parity tests (sizes chosen by the caller)."""
    A, ladder, Y, ratios, sups, cfs = _faust_problem("faust_small", N, K, n_signals, seed, 0, decay, sigma, 6, 6,
                                                    levels, n_active, ratio, True)
    return FaustWorkload("faust_small", A, ladder, Y, ratios, 1e-6, sups, cfs)
