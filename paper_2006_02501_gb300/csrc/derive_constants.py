"""Derivation of the rational constants hard-coded in hermite_consts.cuh.

Run:  python derive_constants.py      (needs sympy; prints the constants)

Method (independent of the quadrature-on-F+- route of Section 2): build the
two-point Hermite interpolant of f on [t0, t1 = t0 + dt] in the monomial basis
centred on t1, matching f^(0..q) at both ends, then
  - integrate it over the step (velocity corrector for f = a, q = p; the
    standard beta = 1 position corrector for f = v, q = p + 1), and
  - differentiate it at t1 (a^(p+1) .. a^(2p-1) for the next predictor).
The modified position correctors are the ones printed in Section 2.1
(Eqs. 21, 22, 23) and are not derived here.
"""
import sympy as sp


def interpolant(q):
    dt, tau = sp.symbols("dt tau")
    c = sp.symbols(f"c0:{2 * q + 2}")
    f1 = sp.symbols(f"f1_0:{q + 1}")
    f0 = sp.symbols(f"f0_0:{q + 1}")
    poly = sum(c[k] * tau ** k for k in range(2 * q + 2))
    eqs = []
    for j in range(q + 1):
        eqs.append(sp.Eq(sp.diff(poly, tau, j).subs(tau, 0), f1[j]))
        eqs.append(sp.Eq(sp.diff(poly, tau, j).subs(tau, -dt), f0[j]))
    sol = sp.solve(eqs, c)
    return poly.subs(sol), tau, dt, f0, f1


def integral_coeffs(q):
    poly, tau, dt, f0, f1 = interpolant(q)
    I = sp.expand(sp.integrate(poly, (tau, -dt, 0)))
    # coefficient of (f1_k +- f0_k) dt^(k+1)
    return [sp.simplify(I.coeff(f1[k]) / dt ** (k + 1)) for k in range(q + 1)], \
           [sp.simplify(I.coeff(f0[k]) / dt ** (k + 1)) for k in range(q + 1)]


def end_derivs(q, orders):
    poly, tau, dt, f0, f1 = interpolant(q)
    out = {}
    for n in orders:
        e = sp.expand(sp.diff(poly, tau, n).subs(tau, 0))
        out[n] = ([sp.simplify(e.coeff(f1[k]) * dt ** (n - k)) for k in range(q + 1)],
                  [sp.simplify(e.coeff(f0[k]) * dt ** (n - k)) for k in range(q + 1)])
    return out


if __name__ == "__main__":
    for p in (1, 2, 3):
        print(f"p={p} velocity (a1^(k), a0^(k)) x dt^(k+1):", integral_coeffs(p))
        print(f"p={p} standard position (v1^(k), v0^(k)) x dt^(k+1):", integral_coeffs(p + 1))
        if p >= 2:
            print(f"p={p} end derivatives x dt^(n-k):", end_derivs(p, range(p + 1, 2 * p)))
