"""Pins for the oracle's pair derivatives and direct summation (Section 3 of
Dittmann 2020: a_ij = G m_j r_ij (r_ij^2 + eps^2)^(-3/2), and its time
derivatives up to the 5th, which the 8th-order initialisation needs).

Independent checks: symbolic differentiation (sympy) along a polynomial
trajectory; finite differences of the acceleration along a numerically
integrated trajectory; the closed-form circular two-body orbit.
"""
from math import factorial

import numpy as np
import pytest


def _sympy_pair_derivs(r_k, eps, Gm, P):
    sp = pytest.importorskip("sympy")
    t = sp.Symbol("t")
    r = [sum(sp.Float(r_k[k][c], 40) * t ** k / sp.factorial(k)
             for k in range(len(r_k))) for c in range(3)]
    s = r[0] ** 2 + r[1] ** 2 + r[2] ** 2 + sp.Float(eps, 40) ** 2
    f = [sp.Float(Gm, 40) * rc * s ** sp.Rational(-3, 2) for rc in r]
    out = np.zeros((P + 1, 3))
    for c in range(3):
        g = f[c]
        for n in range(P + 1):
            out[n, c] = float(g.subs(t, 0).evalf(30))
            g = sp.diff(g, t)
    return out


@pytest.mark.parametrize("P", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("eps", [0.0, 0.3])
def test_pair_derivs_vs_symbolic(orc, P, eps):
    rng = np.random.default_rng(100 + P)
    r_k = rng.normal(size=(P + 1, 3))
    r_k[0] += np.array([1.0, 0.5, -0.2])
    got = orc.pair_derivs(P, r_k, eps, 0.7)
    ref = _sympy_pair_derivs(r_k, eps, 0.7, P)
    for n in range(P + 1):
        np.testing.assert_allclose(got[n], ref[n], rtol=1e-12, atol=1e-13 * np.abs(ref[n]).max())


def test_self_term_skipped_and_softened_zero_distance(orc):
    # Section 3: the sum is over j != i; two bodies at the same point with eps > 0
    # exert no force on each other (r = 0 in the numerator).
    m = np.array([1.0, 2.0])
    traj = np.zeros((2, 2, 3))
    out = orc.evaluate(m, traj, eps=0.1)
    assert np.all(out == 0.0)


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


def test_initialise_vs_finite_differences_of_integrated_trajectory(orc):
    """a^(0..5) at t = 0 from the three initialisation passes against central
    finite differences of a(t) along a DOP853 trajectory (rtol 1e-13), taken as
    the derivatives of the degree-10 interpolant through 11 samples."""
    from scipy.integrate import solve_ivp
    rng = np.random.default_rng(3)
    N = 4
    m = np.array([1.0, 0.01, 0.02, 0.005])
    x = rng.normal(size=(N, 3))
    v = 0.5 * rng.normal(size=(N, 3))
    eps = 0.05
    d = orc.initialise(8, m, x, v, eps)             # a .. a^(5)
    hstep = 0.02
    ts = hstep * np.arange(-5, 6)
    y0 = np.concatenate([x.ravel(), v.ravel()])
    acc = {}
    for sign in (-1, 1):
        tt = sign * hstep * np.arange(0, 6)
        sol = solve_ivp(_nbody_rhs, (0, tt[-1]), y0, t_eval=tt, args=(m, eps), method="DOP853",
                        rtol=1e-13, atol=1e-15)
        for k, tv in enumerate(sol.t):
            acc[int(round(tv / hstep))] = _nbody_rhs(0, sol.y[:, k], m, eps)[3 * N:].reshape(N, 3)
    A = np.array([acc[k] for k in range(-5, 6)])   # (11, N, 3)
    V = np.vander(ts, 11, increasing=True)
    coef = np.linalg.solve(V, A.reshape(11, -1)).reshape(11, N, 3)
    for k in range(6):
        fd = coef[k] * factorial(k)
        tol = [1e-9, 1e-8, 1e-7, 1e-6, 1e-5, 3e-4][k]
        scale = np.abs(d[:, k]).max()
        np.testing.assert_allclose(d[:, k], fd, rtol=0, atol=tol * scale)


@pytest.mark.parametrize("order", [4, 6, 8])
def test_initialise_circular_two_body_closed_form(orc, order):
    """Circular orbit of two bodies: each body moves on a circle of radius R_i
    with angular rate w = sqrt(G M_tot / d^3), so a_i(t) = -w^2 x_i(t) and
    a_i^(k) = -w^2 x_i^(k): every derivative is closed form."""
    M, mm, dsep = 1.0, 0.3, 1.3
    w = np.sqrt((M + mm) / dsep ** 3)
    m = np.array([M, mm])
    R = np.array([-mm / (M + mm) * dsep, M / (M + mm) * dsep])
    # x_i(t) = R_i (cos wt, sin wt, 0)
    def xk(i, k):
        # k-th derivative at t = 0 of R (cos wt, sin wt)
        c = [np.cos, lambda z: -np.sin(z), lambda z: -np.cos(z), np.sin][k % 4](0.0)
        s = [np.sin, np.cos, lambda z: -np.sin(z), lambda z: -np.cos(z)][k % 4](0.0)
        return R[i] * w ** k * np.array([c, s, 0.0])
    x = np.array([xk(0, 0), xk(1, 0)])
    v = np.array([xk(0, 1), xk(1, 1)])
    d = orc.initialise(order, m, x, v, eps=0.0)
    p = order // 2 - 1
    for k in range(2 * p):
        ref = np.array([-w ** 2 * xk(i, k) for i in range(2)])
        np.testing.assert_allclose(d[:, k], ref, rtol=0, atol=2e-14 * np.abs(ref).max())


def test_direct_summation_is_sum_of_pairs(orc):
    rng = np.random.default_rng(5)
    N, P = 7, 3
    m = rng.uniform(0.1, 1.0, N)
    traj = rng.normal(size=(N, P + 1, 3))
    out = orc.evaluate(m, traj, eps=0.01)
    for i in range(N):
        ref = np.zeros((P + 1, 3))
        for j in range(N):
            if j != i:
                ref += orc.pair_derivs(P, traj[j] - traj[i], 0.01, m[j])
        np.testing.assert_allclose(out[i], ref, rtol=1e-14, atol=1e-14)
    # a subrange matches the full evaluation
    np.testing.assert_array_equal(orc.evaluate(m, traj, eps=0.01, i0=2, i1=5), out[2:5])
