"""Seeded synthetic initial conditions for the modified Hermite integrators.

This module draws inputs only: orbital elements from seeded distributions and
their conversion to Cartesian coordinates (Kepler's equation).  It holds none of
the integrator's arithmetic, so both the CUDA path and the CPU oracle can be fed
from it.

Every generator returns (m, x, v) as float64 arrays of shapes (N,), (N, 3), (N, 3)
in the barycentric frame, with body 0 the central mass, G = 1.

Workloads (Section 3 of Dittmann 2020 for the style of the tests):
  kepler_pair         two-body Kepler orbit (Section 3.1)
  planetesimal_ring   central mass + 64 planetesimals, m = 1e-9, a in [0.9, 1.1]
  smbh_disc           SMBH + equal-mass stellar disc, surface density ~ r^-1.5
  disc_100            Section 3.3 disc: 100 bodies of 1e-5 around a unit mass
  planetary_systems   many independent systems of uneven sizes
"""
from __future__ import annotations

import numpy as np


def solve_kepler(M: np.ndarray, e: np.ndarray) -> np.ndarray:
    """Eccentric anomaly E from mean anomaly M: E - e sin E = M (Newton)."""
    M = np.asarray(M, dtype=np.float64)
    e = np.asarray(e, dtype=np.float64)
    E = np.where(e < 0.8, M, np.pi * np.ones_like(M))
    for _ in range(60):
        f = E - e * np.sin(E) - M
        E = E - f / (1.0 - e * np.cos(E))
    return E


def elements_to_cartesian(mu, a, e, inc, Omega, omega, M):
    """Relative position and velocity of an elliptic orbit with gravitational
    parameter mu from (a, e, inclination, node, argument of periapsis, mean anomaly)."""
    mu, a, e, inc, Omega, omega, M = (np.asarray(q, dtype=np.float64) for q in (mu, a, e, inc, Omega, omega, M))
    E = solve_kepler(M, e)
    cE, sE = np.cos(E), np.sin(E)
    b = np.sqrt(1.0 - e * e)
    # perifocal frame
    xp = a * (cE - e)
    yp = a * b * sE
    n = np.sqrt(mu / a ** 3)
    rdot = n * a / (1.0 - e * cE)
    vxp = -rdot * sE
    vyp = rdot * b * cE
    cO, sO, co, so, ci, si = np.cos(Omega), np.sin(Omega), np.cos(omega), np.sin(omega), np.cos(inc), np.sin(inc)
    R = np.stack([
        np.stack([cO * co - sO * so * ci, -cO * so - sO * co * ci], -1),
        np.stack([sO * co + cO * so * ci, -sO * so + cO * co * ci], -1),
        np.stack([so * si, co * si], -1),
    ], -2)                                          # (..., 3, 2)
    r = np.einsum("...ij,...j->...i", R, np.stack([xp, yp], -1))
    v = np.einsum("...ij,...j->...i", R, np.stack([vxp, vyp], -1))
    return r, v


def _to_barycentre(m, x, v):
    mt = m.sum()
    x = x - (m[:, None] * x).sum(0) / mt
    v = v - (m[:, None] * v).sum(0) / mt
    return np.ascontiguousarray(x), np.ascontiguousarray(v)


def _central_plus_orbits(Mc, mb, a, e, inc, Om, om, Ma):
    n = len(mb)
    m = np.concatenate([[Mc], mb]).astype(np.float64)
    r, u = elements_to_cartesian(Mc + mb, a, e, inc, Om, om, Ma)
    x = np.zeros((n + 1, 3))
    v = np.zeros((n + 1, 3))
    x[1:] = r
    v[1:] = u
    x, v = _to_barycentre(m, x, v)
    return m, x, v


def kepler_pair(a=1.0, e=0.5, M=1.0, m=1e-3, mean_anomaly=0.0):
    """Two-body orbit: body 1 of mass m about body 0 of mass M (at pericentre by default)."""
    return _central_plus_orbits(M, np.array([m]), np.array([a]), np.array([e]), np.zeros(1),
                                np.zeros(1), np.zeros(1), np.array([mean_anomaly]))


def planetesimal_ring(seed=1, n=64, m=1e-9, a_lo=0.9, a_hi=1.1, sigma_e=0.01, sigma_i=0.01, Mc=1.0):
    """Central mass plus n planetesimals; e and i Rayleigh-distributed with scale
    parameter sigma, angles uniform, a uniform in [a_lo, a_hi]."""
    g = np.random.default_rng(seed)
    a = g.uniform(a_lo, a_hi, n)
    e = g.rayleigh(sigma_e, n)
    inc = g.rayleigh(sigma_i, n)
    Om, om, Ma = (g.uniform(0.0, 2 * np.pi, n) for _ in range(3))
    return _central_plus_orbits(Mc, np.full(n, m), a, e, inc, Om, om, Ma)


def smbh_disc(seed=2, N=65536, m_total=0.01, r_in=0.1, r_out=1.0, sigma_e=0.05, sigma_i=0.025, M_bh=1.0):
    """SMBH of mass M_bh plus N equal-mass stars (total m_total) with surface
    density proportional to r^-1.5 on [r_in, r_out]: the semi-major-axis pdf is
    then proportional to a^-0.5, sampled as a = (sqrt(r_in) + u (sqrt(r_out) - sqrt(r_in)))^2."""
    g = np.random.default_rng(seed)
    u = g.uniform(0.0, 1.0, N)
    a = (np.sqrt(r_in) + u * (np.sqrt(r_out) - np.sqrt(r_in))) ** 2
    e = np.minimum(g.rayleigh(sigma_e, N), 0.9)
    inc = g.rayleigh(sigma_i, N)
    Om, om, Ma = (g.uniform(0.0, 2 * np.pi, N) for _ in range(3))
    return _central_plus_orbits(M_bh, np.full(N, m_total / N), a, e, inc, Om, om, Ma)


def disc_100(seed=5, n=100, m=1e-5, a_lo=0.1, a_hi=10.0, sigma_e=0.06, sigma_i=0.12, Mc=1.0):
    """Section 3.3 disc: n bodies, log-spaced semi-major axes in [a_lo, a_hi],
    Rayleigh e and i with sigma_i = 2 sigma_e = 0.12."""
    g = np.random.default_rng(seed)
    a = np.geomspace(a_lo, a_hi, n)
    e = g.rayleigh(sigma_e, n)
    inc = g.rayleigh(sigma_i, n)
    Om, om, Ma = (g.uniform(0.0, 2 * np.pi, n) for _ in range(3))
    return _central_plus_orbits(Mc, np.full(n, m), a, e, inc, Om, om, Ma)


def planetary_systems(seed=4, S=4096, nmin=3, nmax=64, m_lo=1e-7, m_hi=1e-3, a_lo=0.5, a_hi=30.0,
                      sigma_e=0.05, sigma_i=0.02, hill_sep=8.0, Mc=1.0):
    """S independent systems; system s has N_s bodies (the star included) with
    N_s uniform in [nmin, nmax]; planet masses and semi-major axes log-uniform;
    adjacent planets closer than hill_sep mutual Hill radii are pushed outward
    (inner to outer) until the separation holds, so a may exceed a_hi.
    Returns (offsets (S+1,), m, x, v, Pmin (S,)) with systems stored contiguously."""
    g = np.random.default_rng(seed)
    offs = [0]
    ms, xs, vs, pmin = [], [], [], []
    for _ in range(S):
        Ns = int(g.integers(nmin, nmax + 1))
        npl = Ns - 1
        mp = np.exp(g.uniform(np.log(m_lo), np.log(m_hi), npl))
        a = np.sort(np.exp(g.uniform(np.log(a_lo), np.log(a_hi), npl)))
        for k in range(1, npl):
            q = hill_sep * 0.5 * ((mp[k - 1] + mp[k]) / (3 * Mc)) ** (1 / 3)
            # mutual Hill separation: a_k - a_{k-1} >= q (a_k + a_{k-1})
            a[k] = max(a[k], a[k - 1] * (1 + q) / (1 - q))
        e = np.minimum(g.rayleigh(sigma_e, npl), 0.5)
        inc = g.rayleigh(sigma_i, npl)
        Om, om, Ma = (g.uniform(0.0, 2 * np.pi, npl) for _ in range(3))
        m, x, v = _central_plus_orbits(Mc, mp, a, e, inc, Om, om, Ma)
        ms.append(m); xs.append(x); vs.append(v)
        pmin.append(2 * np.pi * np.sqrt(a.min() ** 3 / Mc))
        offs.append(offs[-1] + Ns)
    return (np.array(offs, dtype=np.int64), np.concatenate(ms), np.concatenate(xs),
            np.concatenate(vs), np.array(pmin))
