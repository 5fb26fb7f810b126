"""Pins for the oracle's whole integrator (Sections 2.1 and 3 of Dittmann 2020).

Checked against what the mathematics and the paper fix:
  - the two-body Kepler closed form (Kepler's equation) and energy -G M m / 2a;
  - measured convergence order 2(p+1) = 4, 6, 8;
  - time symmetry of the converged P(EC)^n scheme (forward then backward);
  - Section 3.1: modified correctors keep the argument of periapsis from drifting
    secularly, the standard ones do not; 6th-order energy error ~1e3 below 4th;
    n = 2 far better than n = 1;
  - Appendix A identity d e/dx = -d/dt d e/dv along a Kepler orbit;
  - a 4-body system against an independent integrator (DOP853, rtol 1e-13);
  - the Taylor predictor is exact on polynomial trajectories.
"""
from math import factorial

import numpy as np
import pytest

from paper_2006_02501_gb300 import inputs as I


def _rel_closed(t, a, e, mu):
    n = np.sqrt(mu / a ** 3)
    return I.elements_to_cartesian(mu, a, e, 0.0, 0.0, 0.0, n * t)


def _kepler(orc, order, e, dt, nsteps, n_iter, modified=True, m=1e-3, eps=0.0):
    mm, x, v = I.kepler_pair(a=1.0, e=e, M=1.0, m=m)
    S = orc.State(order, mm, x, v, eps, modified=modified)
    S.step(dt, n_iter, nsteps)
    r_ref, v_ref = _rel_closed(S.t, 1.0, e, 1.0 + m)
    return np.linalg.norm((S.x[1] - S.x[0]) - r_ref), S


@pytest.mark.parametrize("order,e,ks", [(4, 0.5, (128, 256)), (6, 0.5, (128, 256)),
                                        (8, 0.5, (64, 128)), (6, 0.1, (64, 128)),
                                        (10, 0.5, (48, 96)), (12, 0.5, (32, 64))])
def test_measured_convergence_order(orc, order, e, ks):
    errs = [_kepler(orc, order, e, 2 * np.pi / k, k, 6)[0] for k in ks]
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < (0.35 if order <= 8 else 0.6), (errs, slope)


@pytest.mark.parametrize("order,tol", [(4, 2e-4), (6, 1e-7), (8, 1e-10)])
def test_kepler_closed_form_one_orbit_e05(orc, order, tol):
    # e = 0.5, dt = 2 pi / 256, one orbit
    err, S = _kepler(orc, order, 0.5, 2 * np.pi / 256, 256, 3)
    assert err < tol
    E_ref = -1.0 * 1e-3 / 2.0        # -G M m / (2a)
    assert abs(S.energy() / E_ref - 1) < 10 * tol


@pytest.mark.parametrize("order", [4, 6, 8])
def test_time_symmetry_forward_backward(orc, order):
    mm, x, v = I.kepler_pair(a=1.0, e=0.5, M=1.0, m=1e-3)
    S = orc.State(order, mm, x, v, 0.0)
    x0, v0 = S.x.copy(), S.v.copy()
    dt, K = 2 * np.pi / 128, 64
    S.step(dt, 12, K)
    S.step(-dt, 12, K)
    assert np.abs(S.x - x0).max() < 1e-11
    assert np.abs(S.v - v0).max() < 1e-11
    # an unconverged single-correction scheme (n = 1) is not time symmetric
    T = orc.State(order, mm, x, v, 0.0)
    T.step(dt, 1, K)
    T.step(-dt, 1, K)
    assert np.abs(T.x - x0).max() > 100 * max(np.abs(S.x - x0).max(), 1e-15)


def _omega_run(orc, order, modified, eps, dt=2.0 ** -4, e=0.1):
    """Section 3.1 setup: m = 1e-3 about M = 1, a = 1, e = 0.1, dt = 2^-4, n = 3,
    t = 100 pi.  Returns (fitted secular slope of the longitude of periapsis,
    max |dE/E0|)."""
    mm, x, v = I.kepler_pair(a=1.0, e=e, M=1.0, m=1e-3)
    S = orc.State(order, mm, x, v, eps, modified=modified)
    E0 = S.energy()
    nst = int(100 * np.pi / dt)
    ts, om, dE = [], [], []
    for _ in range(50):
        S.step(dt, 3, nst // 50)
        ev = S.ecc()[1]
        ts.append(S.t)
        om.append(np.arctan2(ev[1], ev[0]))
        dE.append(S.energy() / E0 - 1)
    return np.polyfit(ts, np.unwrap(om), 1)[0], np.abs(dE).max()


@pytest.mark.parametrize("order,eps", [(4, 1e-8), (6, 1e-8), (8, 0.0)])
def test_modified_corrector_removes_periapsis_drift(orc, order, eps):
    s_mod, _ = _omega_run(orc, order, True, eps)
    s_std, _ = _omega_run(orc, order, False, eps)
    assert abs(s_mod) < 0.1 * abs(s_std), (s_mod, s_std)


@pytest.mark.parametrize("order,dt,e", [(10, 0.35, 0.1), (12, 0.25, 0.3)])
def test_modified_corrector_orders_10_12(orc, order, dt, e):
    """The beta of Eq. 20 holds for any p: at orders 10 and 12 (correctors not
    printed in the paper) the modified scheme still cuts the secular drift of
    the periapsis, at steps where the leading truncation term dominates."""
    s_mod, _ = _omega_run(orc, order, True, 0.0, dt, e)
    s_std, _ = _omega_run(orc, order, False, 0.0, dt, e)
    assert abs(s_mod) < 0.2 * abs(s_std), (s_mod, s_std)


def test_energy_error_drops_with_order(orc):
    # Section 3.1: 6th order ~1e3 smaller energy error than 4th at dt = 2^-4;
    # 8th order a further 1e2-1e3 (rounding-limited)
    e4 = _omega_run(orc, 4, True, 1e-8)[1]
    e6 = _omega_run(orc, 6, True, 1e-8)[1]
    e8 = _omega_run(orc, 8, True, 0.0)[1]
    assert 3e2 < e4 / e6 < 3e4
    assert e6 / e8 > 1e2
    assert e8 < 1e-13


@pytest.mark.parametrize("order", [4, 6])
def test_n2_much_better_than_n1(orc, order):
    # Section 3.1 (Fig. 4): n = 2 is radically better than n = 1; n = 3 close to n = 4
    res = {}
    for n in (1, 2, 3, 4):
        mm, x, v = I.kepler_pair(a=1.0, e=0.1, M=1.0, m=1e-3)
        S = orc.State(order, mm, x, v, 1e-8)
        E0 = S.energy()
        S.step(2.0 ** -4, n, 20000)                  # about 200 orbits
        res[n] = abs(S.energy() / E0 - 1)
    assert res[2] < 1e-2 * res[1]
    assert 0.1 < res[3] / max(res[4], 1e-300) < 10 or res[3] < 1e-14


def test_ecc_vector_closed_form_and_appendix_identity(orc):
    # at pericentre of a planar orbit with omega = 0 the eccentricity vector is (e, 0, 0)
    mm, x, v = I.kepler_pair(a=1.3, e=0.37, M=1.0, m=1e-3)
    ev = orc.ecc(mm, x, v)
    np.testing.assert_allclose(ev[1], [0.37, 0.0, 0.0], atol=1e-13)
    # Appendix A: d e_i/d r_j = -d/dt (d e_i/d v_j) along the orbit
    mu, a, e = 1.0 + 1e-3, 1.3, 0.37
    def evec(r, u):
        m2 = np.array([1.0, 1e-3])
        return orc.ecc(m2, np.array([np.zeros(3), r]), np.array([np.zeros(3), u]))[1]
    def jac(r, u, wrt):
        J = np.zeros((3, 3))
        h = 1e-6
        for j in range(3):
            dr = np.zeros(3); dr[j] = h
            if wrt == "r":
                J[:, j] = (evec(r + dr, u) - evec(r - dr, u)) / (2 * h)
            else:
                J[:, j] = (evec(r, u + dr) - evec(r, u - dr)) / (2 * h)
        return J
    t, ht = 0.7, 1e-4
    r, u = _rel_closed(t, a, e, mu)
    lhs = jac(r, u, "r")
    rp, up = _rel_closed(t + ht, a, e, mu)
    rm, um = _rel_closed(t - ht, a, e, mu)
    rhs = -(jac(rp, up, "v") - jac(rm, um, "v")) / (2 * ht)
    np.testing.assert_allclose(lhs, rhs, atol=1e-6 * np.abs(lhs).max())


def _nbody_rhs(t, y, m, eps):
    N = len(m)
    x = y[:3 * N].reshape(N, 3)
    v = y[3 * N:].reshape(N, 3)
    a = np.zeros_like(x)
    for i in range(N):
        d = x - x[i]
        s = (d * d).sum(1) + eps * eps
        s[i] = 1.0
        w = m / s ** 1.5
        w[i] = 0.0
        a[i] = (w[:, None] * d).sum(0)
    return np.concatenate([v.ravel(), a.ravel()])


@pytest.mark.parametrize("order,tol", [(6, 1e-9), (8, 1e-10)])
def test_four_body_against_dop853(orc, order, tol):
    from scipy.integrate import solve_ivp
    g = np.random.default_rng(9)
    m, x, v = I.planetesimal_ring(seed=9, n=3, m=3e-4, a_lo=0.7, a_hi=1.6, sigma_e=0.05, sigma_i=0.02)
    eps = 1e-3
    T, nst = 4.0, 400
    S = orc.State(order, m, x, v, eps)
    S.step(T / nst, 4, nst)
    sol = solve_ivp(_nbody_rhs, (0, T), np.concatenate([x.ravel(), v.ravel()]), args=(m, eps),
                    method="DOP853", rtol=1e-13, atol=1e-15)
    ref = sol.y[:, -1]
    np.testing.assert_allclose(S.x.ravel(), ref[:12], atol=tol)
    np.testing.assert_allclose(S.v.ravel(), ref[12:], atol=tol)


@pytest.mark.parametrize("order", [4, 6, 8])
def test_predictor_exact_on_polynomial(orc, order):
    p = order // 2 - 1
    rng = np.random.default_rng(21)
    deg = 2 * p + 1                       # x to dt^(2p+1) uses a^(0..2p-1)
    coef = rng.normal(size=(deg + 1, 3))
    def xk(k, t):
        out = np.zeros(3)
        for j in range(k, deg + 1):
            out += coef[j] * factorial(j) / factorial(j - k) * t ** (j - k)
        return out
    dt = 0.23
    d = np.array([[xk(k + 2, 0.0) for k in range(2 * p)]])
    xp, vp, ap = orc.predict(order, dt, xk(0, 0)[None], xk(1, 0)[None], d)
    np.testing.assert_allclose(xp[0], xk(0, dt), rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(vp[0], xk(1, dt), rtol=1e-14, atol=1e-14)
    for q in range(p - 1):
        np.testing.assert_allclose(ap[0, q], xk(q + 2, dt), rtol=1e-13, atol=1e-13)


def test_planetesimal_ring_energy_bounded(orc):
    # central mass + 64 planetesimals, 6th order, P(EC)^2, dt = 2 pi / 256, 1000 steps, eps = 0
    m, x, v = I.planetesimal_ring(seed=1)
    S = orc.State(6, m, x, v, 0.0)
    E0 = S.energy()
    S.step(2 * np.pi / 256, 2, 1000)
    assert abs(S.energy() / E0 - 1) < 1e-12
