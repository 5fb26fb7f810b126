"""Pins for the oracle's time-symmetric variable shared step (Section 3.3).

H = eta min_{i != j} ((r_ij^2 + eps^2)^(3/2) / (G (m_i + m_j)))^(1/2) (Eq. 24) and
dt = (H- + H+)/2, with H+ re-evaluated at the positions of every evaluation of
P(EC)^n (reading R15).  Checked against what the mathematics fixes:
  - Eq. 24 on configurations with a closed form (one pair, the closest of three,
    the scaling with G);
  - a circular orbit keeps H constant, so the variable step must reduce to the
    constant step dt = H;
  - over one e = 0.9 orbit the step follows the two-body time scale r^(3/2):
    largest / smallest step = ((1 + e)/(1 - e))^(3/2);
  - converged iterations make the scheme reversible: n steps forward then n
    backward return to the start, with the step sizes in reverse order;
  - the converged scheme is of order 8 in eta (error against Kepler's equation);
  - the energy error contracts with the number of passes (the step size and
    the positions converge together).
"""
import numpy as np
import pytest

from paper_2006_02501_gb300 import inputs as I

E = 0.9
MU = 1.0 + 1e-3
T_ORBIT = 2 * np.pi / np.sqrt(MU)


def _ecc_pair():
    return I.kepler_pair(a=1.0, e=E, M=1.0, m=1e-3)


def test_eq24_closed_forms(orc):
    m = np.array([2.0, 0.5])
    x = np.array([[0.0, 0.0, 0.0], [0.3, -0.4, 0.0]])          # distance 0.5
    eps, eta = 0.1, 0.07
    s = 0.5 ** 2 + eps ** 2
    assert orc.timestep_H(m, x, eps, eta) == pytest.approx(eta * (s ** 1.5 / 2.5) ** 0.5, rel=1e-15)
    assert orc.timestep_H(m, x, eps, eta, G=4.0) == pytest.approx(orc.timestep_H(m, x, eps, eta) / 2, rel=1e-15)
    # three bodies: the pair with the shortest two-body time scale sets H
    m3 = np.array([1.0, 1e-3, 1e-3])
    x3 = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [1.0, 0.01, 0.0]])
    planet_pair = (0.01 ** 3 / 2e-3) ** 0.5
    star_pair = (1.0 / (1.0 + 1e-3)) ** 0.5
    assert planet_pair < star_pair
    assert orc.timestep_H(m3, x3, 0.0, 1.0) == pytest.approx(planet_pair, rel=1e-14)


def test_circular_orbit_reduces_to_constant_step(orc):
    m, x, v = I.kepler_pair(a=1.0, e=0.0, M=1.0, m=1e-3)
    eta = 0.05
    H0 = orc.timestep_H(m, x, 0.0, eta)
    assert H0 == pytest.approx(eta / np.sqrt(MU), rel=1e-14)
    S = orc.State(8, m, x, v, 0.0)
    dts = S.step_timesym(eta, 3, 64)
    C = orc.State(8, m, x, v, 0.0)
    C.step(H0, 3, 64)
    assert np.ptp(dts) / H0 < 1e-13
    assert np.abs(S.x - C.x).max() < 1e-13 and np.abs(S.v - C.v).max() < 1e-13
    assert S.t == pytest.approx(64 * H0, rel=1e-13)


def test_step_follows_two_body_time_scale(orc):
    m, x, v = _ecc_pair()
    S = orc.State(8, m, x, v, 0.0)
    dts = []
    while S.t < T_ORBIT:
        dts.append(S.step_timesym(0.02, 3, 1)[0])
    dts = np.array(dts)
    assert dts.max() / dts.min() == pytest.approx(((1 + E) / (1 - E)) ** 1.5, rel=5e-3)


def test_reversible_when_converged(orc):
    m, x, v = _ecc_pair()
    S = orc.State(8, m, x, v, 0.0)
    x0, v0 = S.x.copy(), S.v.copy()
    fwd = S.step_timesym(0.02, 10, 300)
    back = S.step_timesym(0.02, 10, 300, backward=True)
    assert np.all(fwd > 0) and np.all(back < 0)
    assert np.abs(fwd[::-1] + back).max() / fwd.max() < 1e-13
    assert np.abs(S.x - x0).max() < 1e-13 and np.abs(S.v - v0).max() < 1e-13
    assert abs(S.t) < 1e-13


def _orbit_error(orc, eta, n_iter):
    m, x, v = _ecc_pair()
    S = orc.State(8, m, x, v, 0.0)
    while S.t < T_ORBIT:
        S.step_timesym(eta, n_iter, 1)
    r_ref, _ = I.elements_to_cartesian(MU, 1.0, E, 0.0, 0.0, 0.0, np.sqrt(MU) * S.t)
    return np.linalg.norm((S.x[1] - S.x[0]) - r_ref)


def test_eighth_order_in_eta(orc):
    slope = np.log2(_orbit_error(orc, 0.08, 12) / _orbit_error(orc, 0.04, 12))
    assert abs(slope - 8) < 0.3, slope


def test_energy_error_contracts_with_passes(orc):
    m, x, v = _ecc_pair()
    errs = {}
    for n in (3, 5, 8):
        S = orc.State(8, m, x, v, 0.0)
        E0 = S.energy()
        worst = 0.0
        while S.t < 2 * T_ORBIT:
            S.step_timesym(0.02, n, 5)
            worst = max(worst, abs(S.energy() / E0 - 1))
        errs[n] = worst
    assert errs[5] < errs[3] / 1000 and errs[8] < errs[5] / 1000, errs
    assert errs[8] < 1e-12, errs
