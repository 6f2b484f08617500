"""Dictionaries, approximate dictionaries and their per-atom error bounds, in FP64.

Test infrastructure only (see the package docstring).

* ``DenseDict``  explicit N x K matrix (atoms are columns).
* ``KronDict``   A~ = (sum_{r<=R} B_r (x) C_r) diag(d) evaluated with small matrix products
                 (the SuKro structure of Section V-A), row-major vectorisation
                 (B (x) C)[n1 N2 + n2, k1 K2 + k2] = B[n1, k1] C[n2, k2].
* ``FaustDict``  A~ = S_0 S_1 ... S_{J-1}, a product of sparse factors (the FAuST structure of
                 Section VI), applied factor by factor.
* quantisers     BF16 (round to nearest even) and FP8 E4M3 with a per-atom scale
                 s_j = max_i |a_ij| / 448, written from the formats' definitions.
* ``Level``      one rung of the ladder {A~^i} with eps^i_j >= ||a~^i_j - a_j||_2 and RC_i
                 (Section IV, Algorithm 1 inputs).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EPS_SAFETY = 1e-12   # relative inflation of FP64-evaluated eps_j so that they stay upper bounds


# ----------------------------------------------------------------------------- operators

class DenseDict:
    """Explicit dictionary; ``matvec`` / ``rmatvec`` may be restricted to an index set."""

    def __init__(self, M: np.ndarray):
        self.M = np.asarray(M, dtype=np.float64)
        self.N, self.K = self.M.shape

    def matvec(self, x, idx=None):
        if idx is None:
            return self.M @ x
        return self.M[:, idx] @ x

    def rmatvec(self, r, idx=None):
        if idx is None:
            return self.M.T @ r
        return self.M[:, idx].T @ r

    def col(self, j):
        return self.M[:, j]

    def dense(self):
        return self.M

    def atom_norms(self):
        return np.sqrt(np.einsum("nk,nk->k", self.M, self.M))


class KronDict:
    """A~ = (sum_{r < R} B_r (x) C_r) diag(d) with B_r: N1 x K1, C_r: N2 x K2.

    matvec:  A~ x = vec(sum_r B_r X C_r^T),  X = reshape(d * x, K1, K2)
    rmatvec: A~^T rho = d * vec(sum_r B_r^T P C_r),  P = reshape(rho, N1, N2)
    The structure gives no saving on a subset of atoms, so restricted products evaluate
    all atoms and select (the worst case of eq:complexity_model_approx).
    """

    def __init__(self, Bf, Cf, d, R=None):
        self.Bf = np.asarray(Bf, dtype=np.float64)
        self.Cf = np.asarray(Cf, dtype=np.float64)
        self.R = self.Bf.shape[0] if R is None else R
        self.N1, self.K1 = self.Bf.shape[1:]
        self.N2, self.K2 = self.Cf.shape[1:]
        self.N, self.K = self.N1 * self.N2, self.K1 * self.K2
        self.d = np.asarray(d, dtype=np.float64)

    def matvec(self, x, idx=None):
        full = np.zeros(self.K)
        if idx is None:
            full[:] = x
        else:
            full[idx] = x
        X = (self.d * full).reshape(self.K1, self.K2)
        out = np.zeros((self.N1, self.N2))
        for r in range(self.R):
            out += self.Bf[r] @ X @ self.Cf[r].T
        return out.reshape(-1)

    def rmatvec(self, rho, idx=None):
        P = np.asarray(rho, dtype=np.float64).reshape(self.N1, self.N2)
        G = np.zeros((self.K1, self.K2))
        for r in range(self.R):
            G += self.Bf[r].T @ P @ self.Cf[r]
        g = self.d * G.reshape(-1)
        return g if idx is None else g[idx]

    def col(self, j):
        k1, k2 = divmod(int(j), self.K2)
        c = np.zeros(self.N)
        for r in range(self.R):
            c += np.kron(self.Bf[r][:, k1], self.Cf[r][:, k2])
        return self.d[j] * c

    def dense(self):
        M = np.zeros((self.N, self.K))
        for r in range(self.R):
            M += np.kron(self.Bf[r], self.Cf[r])
        return M * self.d[None, :]

    def atom_norms(self):
        return np.array([np.linalg.norm(self.col(j)) for j in range(self.K)])


class FaustDict:
    """A~ = S_0 S_1 ... S_{J-1} with S_f sparse (CSR: row pointers, column indices, values).

    matvec:  A~ x = S_0 (S_1 (... (S_{J-1} x)))
    rmatvec: A~^T rho = S_{J-1}^T (... (S_0^T rho))
    Each factor product is the plain definition (out_i = sum_p v_p in_{c_p} over row i), written
    with ``np.bincount`` in FP64.  Restricted products evaluate every atom and select.
    """

    def __init__(self, factors):
        self.f = []
        for S in factors:
            indptr = np.asarray(S.indptr, np.int64)
            rows, cols = S.shape
            row_of = np.repeat(np.arange(rows), np.diff(indptr))
            self.f.append((rows, cols, row_of, np.asarray(S.indices, np.int64), np.asarray(S.data, np.float64)))
        self.N = self.f[0][0]
        self.K = self.f[-1][1]
        for (r0, c0, *_), (r1, c1, *_) in zip(self.f[:-1], self.f[1:]):
            assert c0 == r1, "inner dimensions of consecutive factors must agree"

    @staticmethod
    def _apply(fac, v):
        rows, cols, row_of, col, val = fac
        return np.bincount(row_of, weights=val * v[col], minlength=rows)

    @staticmethod
    def _apply_t(fac, v):
        rows, cols, row_of, col, val = fac
        return np.bincount(col, weights=val * v[row_of], minlength=cols)

    def matvec(self, x, idx=None):
        v = np.zeros(self.K)
        if idx is None:
            v[:] = x
        else:
            v[idx] = x
        for fac in reversed(self.f):
            v = self._apply(fac, v)
        return v

    def rmatvec(self, rho, idx=None):
        v = np.asarray(rho, dtype=np.float64)
        for fac in self.f:
            v = self._apply_t(fac, v)
        return v if idx is None else v[idx]

    def col(self, j):
        e = np.zeros(self.K)
        e[int(j)] = 1.0
        return self.matvec(e)

    def dense(self):
        M = np.eye(self.K)
        for fac in reversed(self.f):
            rows, cols, row_of, col, val = fac
            out = np.zeros((rows, M.shape[1]))
            np.add.at(out, row_of, val[:, None] * M[col])
            M = out
        return M

    def abs_dense(self):
        """|S_0| |S_1| ... |S_{J-1}| (entrywise absolute values of the factors), explicit."""
        op = FaustDict.__new__(FaustDict)
        op.f = [(r, c, ro, co, np.abs(v)) for (r, c, ro, co, v) in self.f]
        op.N, op.K = self.N, self.K
        return op.dense()

    def nnz(self):
        return int(sum(fac[4].size for fac in self.f))

    def atom_norms(self):
        M = self.dense()
        return np.sqrt(np.einsum("nk,nk->k", M, M))


def kron_unit_scale(Bf, Cf, R=None) -> np.ndarray:
    """d_j = 1 / ||(sum_r B_r (x) C_r) e_j||_2, from the explicit columns (np.kron)."""
    op = KronDict(Bf, Cf, np.ones(Bf.shape[2] * Cf.shape[2]), R)
    return 1.0 / np.array([np.linalg.norm(op.col(j)) for j in range(op.K)])


def kron_truncation_eps_gram(Bf, Cf, d, R_keep) -> np.ndarray:
    """Exact eps_j = ||a~_j - a_j|| for the truncation to the first R_keep terms (closed form).

    a_j - a~_j = d_j sum_{r >= R_keep} B_r[:, k1] (x) C_r[:, k2], and
    ||sum_r b_r (x) c_r||^2 = sum_{r,s} (b_r . b_s)(c_r . c_s).
    """
    tb = Bf[R_keep:]
    tc = Cf[R_keep:]
    if tb.shape[0] == 0:
        return np.zeros(Bf.shape[2] * Cf.shape[2])
    GB = np.einsum("rnk,snk->rsk", tb, tb)
    GC = np.einsum("rnk,snk->rsk", tc, tc)
    sq = np.einsum("rsa,rsb->ab", GB, GC).reshape(-1)
    return d * np.sqrt(np.maximum(sq, 0.0))


# ----------------------------------------------------------------------------- quantisers

def to_f32(a) -> np.ndarray:
    return np.asarray(a, dtype=np.float32).astype(np.float64)


def bf16_round(a) -> np.ndarray:
    """Round FP32 values to BF16 (8 exponent bits, 7 mantissa bits), round to nearest, ties to even.

    BF16 is the top half of the FP32 encoding: add half an ulp of the kept part (plus the
    kept part's last bit, which breaks ties towards even) and truncate the low 16 bits.
    """
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = f.view(np.uint32).astype(np.uint64)
    rounded = (bits + 0x7FFF + ((bits >> 16) & 1)) & 0xFFFF0000
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


E4M3_MAX = 448.0


def e4m3_round(v) -> np.ndarray:
    """Round FP32 values to FP8 E4M3 ('fn' variant: bias 7, no infinities), ties to even, saturating.

    Normal numbers have a 3-bit mantissa, so the spacing at |v| in [2^e, 2^(e+1)) is 2^(e-3);
    below 2^-6 the format is subnormal with fixed spacing 2^-9.  Magnitudes that round above
    the largest finite value 448 saturate to 448.
    """
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    _, ex = np.frexp(a)                 # a = m 2^ex, m in [0.5, 1)
    e = np.maximum(ex - 1, -6)          # floor(log2 a), clamped to the subnormal exponent
    quantum = np.ldexp(1.0, e - 3)
    q = np.rint(a / quantum) * quantum  # np.rint rounds half to even
    q = np.minimum(q, E4M3_MAX)
    return np.sign(v) * q


def fp8_atom_scale(A) -> np.ndarray:
    """Per-atom scale s_j = fl32(max_i |a_ij| / 448) (FP64 quotient, then rounded to FP32)."""
    m = np.max(np.abs(np.asarray(A, dtype=np.float64)), axis=0)
    s = to_f32(m / E4M3_MAX)
    return np.where(s > 0, s, 1.0)


def fp8_quantize(A):
    """Per-atom scaled E4M3 copy: q_ij = E4M3(fl32(a_ij / s_j)), a~_ij = s_j q_ij (exact in FP64)."""
    A32 = np.asarray(A, dtype=np.float32)
    s = fp8_atom_scale(A)
    v = (A32 / s.astype(np.float32)[None, :]).astype(np.float64)   # IEEE FP32 division
    q = e4m3_round(v)
    return q * s[None, :], q, s


def split_bf16(A):
    """The split BF16 pair of an FP32 dictionary, an approximate dictionary in the sense of
    Section III: entrywise a1 = bf16(a), a2 = bf16(a - a1), approximation a~ = a1 + a2.

    a - a1 is exact in FP32: a1 is a rounding of a, so the difference lies on a's own grid with
    at most 16 significant bits.  A is N x K (atoms as columns).  Returns (a1, a2, eps): a1 and
    a2 as FP64 arrays of the BF16 values, and eps_j = ||a_j - a1_j - a2_j||_2 from the exact
    entrywise remainders.
    """
    a = to_f32(A)
    a1 = bf16_round(a.astype(np.float32))
    r = a - a1
    a2 = bf16_round(r.astype(np.float32))
    e = r - a2
    return a1, a2, np.sqrt(np.sum(e * e, axis=0))


# ----------------------------------------------------------------------------- ladder

@dataclass
class Level:
    """One approximate dictionary A~^i with its error bounds and relative complexity."""
    name: str
    op: object                  # DenseDict or KronDict
    eps: np.ndarray             # K, eps_j >= ||a~_j - a_j||_2
    rc: float                   # relative complexity RC(A~^i) (eq:complexity_model_approx)
    atnorm: np.ndarray          # K, ||a~_j||_2 (used by the look-ahead estimate K_t)


def exact_errors(approx_cols: np.ndarray, exact_cols: np.ndarray) -> np.ndarray:
    """eps_j = ||a~_j - a_j||_2 evaluated in FP64, inflated by EPS_SAFETY to stay an upper bound."""
    diff = np.asarray(approx_cols, np.float64) - np.asarray(exact_cols, np.float64)
    return np.sqrt(np.einsum("nk,nk->k", diff, diff)) * (1.0 + EPS_SAFETY)


def dense_level(name, approx: np.ndarray, exact: np.ndarray, rc: float) -> Level:
    op = DenseDict(approx)
    return Level(name, op, exact_errors(approx, exact), rc, op.atom_norms())


def exact_level(A: np.ndarray) -> Level:
    op = DenseDict(A)
    return Level("exact", op, np.zeros(op.K), 1.0, op.atom_norms())


def kron_level(Bf, Cf, d, R_keep, exact_dense=None, rc=None) -> Level:
    """Truncation A~^(R) = (sum_{r < R_keep} B_r (x) C_r) diag(d), d of the full sum.

    eps_j is the closed form of ``kron_truncation_eps_gram`` when the exact dictionary is the
    full Kronecker sum, or the explicit column differences when ``exact_dense`` is given.
    RC defaults to the theoretical ratio R_keep (2 N1 K1 K2 + 2 N1 K2 N2) / (2 N K).
    """
    op = KronDict(Bf, Cf, d, R_keep)
    if exact_dense is None:
        eps = kron_truncation_eps_gram(Bf, Cf, d, R_keep) * (1.0 + EPS_SAFETY)
    else:
        eps = exact_errors(op.dense(), exact_dense)
    if rc is None:
        rc = R_keep * (op.N1 * op.K1 * op.K2 + op.N1 * op.K2 * op.N2) / (op.N * op.K)
    atn = np.sqrt(np.maximum(
        np.einsum("rsa,rsb->ab",
                  np.einsum("rnk,snk->rsk", op.Bf[:R_keep], op.Bf[:R_keep]),
                  np.einsum("rnk,snk->rsk", op.Cf[:R_keep], op.Cf[:R_keep])).reshape(-1), 0.0)) * d
    return Level(f"kron{R_keep}", op, eps, rc, atn)


def faust_level(factors, exact_dense: np.ndarray, rc=None, name="faust") -> Level:
    """Product of sparse factors as a ladder level: eps_j = ||a~_j - a_j|| from the explicit FP64
    product, RC defaulting to the nonzeros of the factors over N K (one multiply-add per nonzero
    against N K for the dense product)."""
    op = FaustDict(factors)
    Ad = op.dense()
    eps = exact_errors(Ad, exact_dense)
    if rc is None:
        rc = op.nnz() / (op.N * op.K)
    return Level(name, op, eps, rc, np.sqrt(np.einsum("nk,nk->k", Ad, Ad)))


def power_iteration_sq_norm(op, iters: int = 200, safety: float = 1.001) -> float:
    """L = safety * ||A||_2^2 estimated by power iteration on A^T A from the all-ones vector."""
    v = np.ones(op.K) / np.sqrt(op.K)
    s = 0.0
    for _ in range(iters):
        w = op.rmatvec(op.matvec(v))
        s = float(np.linalg.norm(w))
        if s == 0.0:
            return 0.0
        v = w / s
    return safety * s
