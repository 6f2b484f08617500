"""The pins are sensitive: plant a plausible mistake in the oracle (on the CPU) and check a pin fails.

Each case monkeypatches one oracle formula with a typical slip (a dropped term, a wrong sign,
a missing clip) and runs a pin from ``test_oracle_problem``; the pin must raise.
"""
import numpy as np
import pytest

import test_oracle_problem as P
from oracle import lasso as L


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


CASES = [
    ("soft_threshold", _wrong_threshold, lambda: P.test_brute_force_sign_enumeration(0, 0.5)),
    ("dual_of_multiple", _dual_sign_slip, lambda: P.test_brute_force_sign_enumeration(1, 0.5)),
    ("stable_sphere_test", _stable_test_without_eps, lambda: P.test_stable_zone_test_bounds_every_atom_in_the_zone()),
    ("theta_dynamic_coef", _coef_without_clip, lambda: P.test_gap_safe_sphere_exact_dictionary()),
    ("stable_gap_radius", _radius_without_delta, lambda: P.test_theorem1_stable_gap_sphere_contains_theta_star(0)),
]


@pytest.mark.parametrize("name,bad,pin", CASES, ids=[c[0] for c in CASES])
def test_planted_mistake_is_caught(monkeypatch, name, bad, pin):
    monkeypatch.setattr(L, name, bad)
    with pytest.raises((AssertionError, Exception)):
        pin()
