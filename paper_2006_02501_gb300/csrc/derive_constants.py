"""Derivation of the rational constants hard-coded in hermite_consts.cuh.

Run:  python derive_constants.py      (needs sympy; prints the constants)
      python derive_constants.py --dd-header   (writes hermite_consts_dd.cuh: the
      same constants as exact numerator / denominator pairs)

Method (independent of the quadrature-on-F+- route of Section 2): build the
two-point Hermite interpolant of f on [t0, t1 = t0 + dt] in the monomial basis
centred on t1, matching f^(0..q) at both ends, then
  - integrate it over the step (velocity corrector for f = a, q = p; the
    standard beta = 1 position corrector for f = v, q = p + 1),
  - differentiate it at t1 (a^(p+1) .. a^(2p-1) for the next predictor), and
  - for the modified position corrector (Eq. 7, beta of Eq. 20): add
    (beta - 1)/(2p + 3) F_(2p+2) dt, where F_(2p+2) = h^(2p+2) v^(2p+2)(mid)/(2p+2)!
    is the interpolant's scaled derivative at the midpoint (h = dt/2).  For
    orders 4, 6, 8 this reproduces the correctors printed in Section 2.1
    (Eqs. 21, 22, 23), checked below; orders 10 and 12 come from the same formula.
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


def beta(p):
    """Eq. 20: beta = 1 + (-1)^(p+1) (2p+2)!! / (2p+1)!!."""
    return 1 + (-1) ** (p + 1) * sp.factorial2(2 * p + 2) / sp.factorial2(2 * p + 1)


def modified_position_coeffs(p):
    """Coefficients of (v1^(k) +- v0^(k)) dt^(k+1), k = 0 .. p+1, of the modified
    position corrector (Eq. 7 with beta of Eq. 20)."""
    q = p + 1
    poly, tau, dt, f0, f1 = interpolant(q)
    h = dt / 2
    n = 2 * p + 2
    Fn = sp.expand(h ** n * sp.diff(poly, tau, n).subs(tau, -h) / sp.factorial(n))
    extra = sp.expand((beta(p) - 1) / (2 * p + 3) * Fn * dt)
    I = sp.expand(sp.integrate(poly, (tau, -dt, 0))) + extra
    return [sp.simplify(I.coeff(f1[k]) / dt ** (k + 1)) for k in range(q + 1)], \
           [sp.simplify(I.coeff(f0[k]) / dt ** (k + 1)) for k in range(q + 1)]


PRINTED = {   # Section 2.1: Eq. 21 (p = 1), Eq. 22 (p = 2), Eq. 23 (p = 3), on (v1^(k) +- v0^(k)) dt^(k+1)
    1: [sp.Rational(1, 2), sp.Rational(-7, 60), sp.Rational(1, 60)],
    2: [sp.Rational(1, 2), sp.Rational(-4, 35), sp.Rational(13, 840), sp.Rational(-1, 840)],
    3: [sp.Rational(1, 2), sp.Rational(-29, 252), sp.Rational(1, 63), sp.Rational(-1, 720), sp.Rational(1, 15120)],
}


def rational_tables():
    """The constants of hermite_consts.cuh as exact rationals, p = 1 .. 5:
    kv[p][k], kx[p][b][k] (b = 0 modified, 1 standard), e1[p][n][k], e0[p][n][k]."""
    T = {"kv": {}, "kx": {}, "e1": {}, "e0": {}}
    for p in range(1, 6):
        T["kv"][p] = [sp.Rational(c) for c in integral_coeffs(p)[0]]
        T["kx"][p] = [[sp.Rational(c) for c in modified_position_coeffs(p)[0]],
                      [sp.Rational(c) for c in integral_coeffs(p + 1)[0]]]
        d = end_derivs(p, range(p + 1, 2 * p)) if p >= 2 else {}
        T["e1"][p] = {n: [sp.Rational(c) for c in d[n][0]] for n in d}
        T["e0"][p] = {n: [sp.Rational(c) for c in d[n][1]] for n in d}
    return T


def dd_header() -> str:
    """hermite_consts_dd.cuh: the same constants as numerator / denominator pairs,
    from which the double-double kernels form each value to 106 bits."""
    T = rational_tables()
    pair = lambda r: "{%d, %d}" % (r.p, r.q)
    fn = "__host__ __device__ constexpr Ratio"
    L = ["// Rational constants of the modified Hermite corrector and end-of-step",
         "// interpolation (the values of hermite_consts.cuh, same meaning: kv(k),",
         "// kx(beta_mode, k), e1(n, k), e0(n, k) with n = p+1 .. 2p-1) as exact",
         "// numerator / denominator pairs, p = 1 .. 5, for the double-double form.",
         "// Written by `python derive_constants.py --dd-header`.",
         "#pragma once", "", "namespace mh {", "namespace ddc {", "",
         "struct Ratio { long long num, den; };", ""]
    for p in range(1, 6):
        L.append(f"// p = {p} (order {2 * p + 2})")
        L.append(f"{fn} kv{p}(int k)")
        L.append(f"{{ constexpr Ratio t[{p + 1}] = {{{', '.join(pair(r) for r in T['kv'][p])}}}; return t[k]; }}")
        rows = ", ".join("{" + ", ".join(pair(r) for r in T["kx"][p][b]) + "}" for b in (0, 1))
        L.append(f"{fn} kx{p}(int b, int k)")
        L.append(f"{{ constexpr Ratio t[2][{p + 2}] = {{{rows}}}; return t[b][k]; }}")
        if p >= 2:
            for nm in ("e1", "e0"):
                rows = ", ".join("{" + ", ".join(pair(r) for r in T[nm][p][n]) + "}"
                                 for n in range(p + 1, 2 * p))
                L.append(f"{fn} {nm}_{p}(int n, int k)")
                L.append(f"{{ constexpr Ratio t[{p - 1}][{p + 1}] = {{{rows}}}; return t[n - {p + 1}][k]; }}")
        L.append("")
    L += ["}  // namespace ddc", "}  // namespace mh", ""]
    return "\n".join(L)


if __name__ == "__main__":
    import sys
    if "--dd-header" in sys.argv:
        import os
        out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hermite_consts_dd.cuh")
        open(out, "w").write(dd_header())
        print(out)
        sys.exit(0)
    for p in (1, 2, 3):
        c1, c0 = modified_position_coeffs(p)
        assert c1 == PRINTED[p], (p, c1)
        assert all(c0[k] == (-1) ** k * c1[k] for k in range(len(c1))), (p, c0)
    print("modified position correctors of Eqs. 21-23 reproduced")
    for p in (4, 5):
        print(f"p={p} beta = {beta(p)}")
        print(f"p={p} velocity:", integral_coeffs(p)[0])
        print(f"p={p} modified position:", modified_position_coeffs(p)[0])
        print(f"p={p} standard position:", integral_coeffs(p + 1)[0])
        d = end_derivs(p, range(p + 1, 2 * p))
        for n in range(p + 1, 2 * p):
            print(f"p={p} end derivative n={n}: e1 = {d[n][0]}  e0 = {d[n][1]}")
    for p in (1, 2, 3):
        print(f"p={p} velocity (a1^(k), a0^(k)) x dt^(k+1):", integral_coeffs(p))
        print(f"p={p} standard position (v1^(k), v0^(k)) x dt^(k+1):", integral_coeffs(p + 1))
        if p >= 2:
            print(f"p={p} end derivatives x dt^(n-k):", end_derivs(p, range(p + 1, 2 * p)))
