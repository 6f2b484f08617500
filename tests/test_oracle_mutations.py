"""The pins are sensitive: plant a plausible mistake in the oracle (on the CPU) and check a pin fails.

Each case monkeypatches one oracle formula with a typical slip (a dropped term, a wrong sign,
a missing clip) and runs a pin from ``test_oracle_problem``; the pin must raise.
"""
import numpy as np
import pytest

import test_oracle_backward as TB
import test_oracle_dicts as TD
import test_oracle_problem as P
import test_oracle_regions as TR
from oracle import backward as OB
from oracle import dictionaries as D
from oracle import lasso as L
from oracle import regions as G


def _wrong_threshold(v, u):
    return np.sign(v) * np.maximum(np.abs(v) - 0.5 * u, 0.0)


def _dual_sign_slip(s, yr, rr, lam):
    return -lam * s * yr - 0.5 * lam * lam * s * s * rr


def _stable_test_without_eps(attc, eps, cnorm, R, anorm):
    return np.abs(attc) + R * anorm


def _coef_without_clip(yr, rr, lam, m):
    return yr / (lam * rr) if rr > 0 else 0.0


def _radius_without_delta(Gp, delta, lam):
    return float(np.sqrt(max(2.0 * Gp, 0.0))) / lam


def _projection_without_lam(y, z, lam):
    return float(y @ z) / float(z @ z)


def _stable_lambda_max_without_eps(Atty, eps, ynorm):
    return float(np.max(np.abs(Atty)))


CASES = [
    ("soft_threshold", _wrong_threshold, lambda: P.test_brute_force_sign_enumeration(0, 0.5)),
    ("dual_of_multiple", _dual_sign_slip, lambda: P.test_brute_force_sign_enumeration(1, 0.5)),
    ("stable_sphere_test", _stable_test_without_eps, lambda: P.test_stable_zone_test_bounds_every_atom_in_the_zone()),
    ("theta_dynamic_coef", _coef_without_clip, lambda: P.test_gap_safe_sphere_exact_dictionary()),
    ("stable_gap_radius", _radius_without_delta, lambda: P.test_theorem1_stable_gap_sphere_contains_theta_star(0)),
    ("projection_coefficient", _projection_without_lam, lambda: P.test_projection_coefficient_is_the_orthogonal_projection()),
    ("stable_lambda_max", _stable_lambda_max_without_eps, lambda: P.test_stable_lambda_max_bounds_lambda_max()),
]


@pytest.mark.parametrize("name,bad,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, name, bad, pin):
    monkeypatch.setattr(L, name, bad)
    with pytest.raises((AssertionError, Exception)):
        pin()


# ----------------------------------------------------------------------------- zones, domes, factors

def _C_pq_flipped(N, p, q):
    inv_pstar = 1.0 - (0.0 if np.isinf(p) else 1.0 / p)
    inv_q = 0.0 if np.isinf(q) else 1.0 / q
    return float(N) ** max(inv_q - inv_pstar, 0.0)


def _zone_test_without_eps_term(a_t, eps, c, R, p, q):
    return abs(float(a_t @ c)) + R * float(G.lq_norm(a_t, G.conjugate(p))) + G.C_pq(a_t.size, p, q) * R * eps


def _dome_max_wrong_offset_sign(a, c, R, n, psi):
    an, nn = float(np.linalg.norm(a)), float(np.linalg.norm(n))
    d = psi - float(n @ c)
    if R * float(n @ a) / an <= d:
        return float(a @ c) + R * an
    nh = n / nn
    alpha = float(a @ nh)
    h = d / nn
    return float(a @ c) - alpha * h + float(np.linalg.norm(a - alpha * nh)) * float(np.sqrt(max(R * R - h * h, 0.0)))


def _scaling_q_with_l2_norm(Atz, eps, z, q):
    m = float(np.max(np.abs(Atz) + eps * float(np.linalg.norm(z))))
    return 1.0 / max(1.0, m)


def _apply_t_through_rows(fac, v):
    rows, cols, row_of, col, val = fac
    out = np.zeros(cols)
    np.add.at(out, np.minimum(row_of, cols - 1), val * v[np.minimum(col, rows - 1)])
    return out


def _matvec_wrong_order(self, x, idx=None):
    v = np.zeros(self.K)
    if idx is None:
        v[:] = x
    else:
        v[idx] = x
    for fac in self.f:                       # S_0 applied first instead of last
        rows, cols, row_of, col, val = fac
        v = np.bincount(row_of, weights=val * v[np.minimum(col, v.size - 1)], minlength=rows)
    return v


def _split_without_remainder(A):
    a = D.to_f32(A)
    a1 = D.bf16_round(a.astype(np.float32))
    a2 = D.bf16_round((a - a1).astype(np.float32)) * 0.5       # the second part halved
    e = a - a1 - a2
    return a1, a2, np.sqrt(np.sum(e * e, axis=0))


def _bf16_truncating(a):
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    bits = f.view(np.uint32).astype(np.uint64) & 0xFFFF0000          # chops instead of rounding
    return bits.astype(np.uint32).view(np.float32).astype(np.float64)


_e4m3_right = D.e4m3_round


def _e4m3_ties_away(v):
    v = np.asarray(v, dtype=np.float64)
    up = _e4m3_right(v * (1.0 + 2.0 ** -20))                         # nudges every tie outwards
    return np.where(np.abs(v) > 0, up, 0.0)


def _kron_eps_without_scale(Bf, Cf, d, R_keep):
    tb, tc = Bf[R_keep:], Cf[R_keep:]
    GB = np.einsum("rnk,snk->rsk", tb, tb)
    GC = np.einsum("rnk,snk->rsk", tc, tc)
    return np.sqrt(np.maximum(np.einsum("rsa,rsb->ab", GB, GC).reshape(-1), 0.0))   # d_j dropped


def _kron_matvec_transposed_c(self, x, idx=None):
    full = np.zeros(self.K)
    if idx is None:
        full[:] = x
    else:
        full[idx] = x
    X = (self.d * full).reshape(self.K1, self.K2)
    out = np.zeros((self.N1, self.N2))
    for r in range(self.R):
        out += self.Bf[r] @ X @ self.Cf[r][::-1].T                  # rows of C_r in reverse order
    return out.reshape(-1)


def _adjoint_sign_slip(A, y, x, g):
    dy, dA = _adjoint_right(A, y, x, g)
    S = np.flatnonzero(x)
    if S.size:
        AS = A[:, S]
        u = np.linalg.solve(AS.T @ AS, g[S])
        dA[:, S] = np.outer(y - AS @ x[S], u) + np.outer(AS @ u, x[S])   # + instead of -
    return dy, dA


_adjoint_right = OB.support_adjoint


REGION_CASES = [
    (G, "C_pq", _C_pq_flipped, lambda: TR.test_C_pq_against_extreme_points(3, 3.0)),
    (G, "zone_sphere_test", _zone_test_without_eps_term,
     lambda: TR.test_zone_sphere_test_bounds_sampled_pairs(2.0, np.inf)),
    (G, "dome_max", _dome_max_wrong_offset_sign, lambda: TR.test_dome_max_matches_constrained_maximisation()),
    (G, "stable_scaling_q", _scaling_q_with_l2_norm, lambda: TR.test_lemma2_with_lq_errors_gives_feasible_dual_points(np.inf)),
    (D.FaustDict, "_apply_t", staticmethod(_apply_t_through_rows),
     lambda: TD.test_faust_operator_against_explicit_product((6, 9, 13))),
    (D.FaustDict, "matvec", _matvec_wrong_order, lambda: TD.test_faust_operator_against_explicit_product((6, 9, 13))),
    (D, "split_bf16", _split_without_remainder, lambda: TD.test_split_bf16_pair()),
    (D, "bf16_round", _bf16_truncating, lambda: TD.test_bf16_matches_torch_cast()),
    (D, "e4m3_round", _e4m3_ties_away, lambda: TD.test_e4m3_matches_torch_cast_in_range_and_saturates()),
    (D, "kron_truncation_eps_gram", _kron_eps_without_scale,
     lambda: TD.test_kron_truncation_eps_gram_equals_column_differences()),
    (D.KronDict, "matvec", _kron_matvec_transposed_c, lambda: TD.test_kron_operator_against_explicit_kron()),
    (OB, "support_adjoint", _adjoint_sign_slip, lambda: TB.test_adjoint_matches_central_differences()),
]


@pytest.mark.parametrize("owner,name,bad,pin", REGION_CASES, ids=[c[1] for c in REGION_CASES])
def test_planted_mistake_in_regions_and_factors_is_caught(monkeypatch, owner, name, bad, pin):
    monkeypatch.setattr(owner, name, bad)
    with pytest.raises((AssertionError, Exception)):
        pin()
