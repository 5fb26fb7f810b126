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
  - the scheme is of order 8 in eta (error against Kepler's equation), already
    with n = 3 passes;
  - Section 3.3 / introduction: with the time-symmetric step the energy error
    stays bounded over many orbits, while a variable step that is not
    symmetric (dt = H at the start of each step) drifts secularly.
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


@pytest.mark.parametrize("n_iter", [3, 12])
def test_eighth_order_in_eta(orc, n_iter):
    slope = np.log2(_orbit_error(orc, 0.16, n_iter) / _orbit_error(orc, 0.08, n_iter))
    assert abs(slope - 8) < 0.3, slope


def _energy_errors(orc, advance, orbits=20):
    """max |E/E0 - 1| over the first and over the last 4 orbits."""
    m, x, v = _ecc_pair()
    S = orc.State(8, m, x, v, 0.0)
    E0 = S.energy()
    rows = []
    while S.t < orbits * T_ORBIT:
        advance(S)
        rows.append((S.t, abs(S.energy() / E0 - 1)))
    rows = np.array(rows)
    return rows[rows[:, 0] < 4 * T_ORBIT, 1].max(), rows[rows[:, 0] > (orbits - 4) * T_ORBIT, 1].max()


def test_energy_bounded_unlike_explicit_variable_step(orc):
    eta = 0.08
    sym_first, sym_last = _energy_errors(orc, lambda S: S.step_timesym(eta, 3, 5))

    def explicit(S):
        for _ in range(5):
            S.step(orc.timestep_H(S.m, S.x, S.eps, eta, S.G), 3)

    exp_first, exp_last = _energy_errors(orc, explicit)
    assert sym_last < 1.5 * sym_first, (sym_first, sym_last)
    assert exp_last > 3 * exp_first, (exp_first, exp_last)
    assert sym_last < exp_last / 10
