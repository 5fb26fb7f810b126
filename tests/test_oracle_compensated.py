"""Pins for compensated summation of the step updates (Section 3.2, after Kahan):
x and v accumulate their increments with a carried compensation term.

  - exact: a free body (no force) adds the same rounded increment every step;
    the compensated position stays within a few ulps of that sum computed in
    rational arithmetic, the plain sum drifts far from it;
  - Section 3.2: where the energy error of the 8th-order scheme is dominated
    by rounding (a near-circular orbit at a step far below the truncation
    limit), compensation lowers it several times; where truncation dominates
    it changes nothing.
"""
from fractions import Fraction

import numpy as np

from paper_2006_02501_gb300 import inputs as I


def test_free_body_sum_exact(orc):
    m = np.array([1.0])
    x = np.array([[0.1, -0.7, 3.3]])
    v = np.array([[1.0 / 3.0, 2.0 / 7.0, -1.0 / 9.0]])
    dt, K = 0.01, 100000
    out = {}
    for comp in (False, True):
        S = orc.State(8, m, x, v, 0.0)
        S.step(dt, 2, K, compensated=comp)
        out[comp] = S.x[0]
    for c in range(3):
        inc = Fraction(float(v[0, c] * dt))            # the rounded increment every step adds
        exact = Fraction(float(x[0, c])) + K * inc
        ulp = abs(float(np.spacing(float(exact))))
        err_plain = abs(Fraction(float(out[False][c])) - exact)
        err_comp = abs(Fraction(float(out[True][c])) - exact)
        assert err_comp <= 2 * ulp, (c, float(err_comp), ulp)
        assert err_plain > 50 * ulp, (c, float(err_plain), ulp)


def _energy_err(orc, e, k, orbits, comp):
    m, x, v = I.kepler_pair(a=1.0, e=e, M=1.0, m=1e-3)
    S = orc.State(8, m, x, v, 0.0)
    E0 = S.energy()
    worst = 0.0
    for _ in range(orbits // 10):
        S.step(2 * np.pi / k, 3, 10 * k, compensated=comp)
        worst = max(worst, abs(S.energy() / E0 - 1))
    return worst


def test_compensation_lowers_rounding_dominated_energy_error(orc):
    plain = _energy_err(orc, 0.1, 128, 1000, False)
    comp = _energy_err(orc, 0.1, 128, 1000, True)
    assert comp < plain / 3, (plain, comp)


def test_compensation_leaves_truncation_error_alone(orc):
    plain = _energy_err(orc, 0.5, 256, 200, False)
    comp = _energy_err(orc, 0.5, 256, 200, True)
    assert abs(comp / plain - 1) < 0.2, (plain, comp)
