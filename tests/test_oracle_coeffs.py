"""Pins for the oracle's Hermite algebra (Section 2 and 2.1 of Dittmann 2020).

The exact-rational module (oracle/coeffs.py) is checked against the values the
paper prints (tests/golden/printed_correctors.txt), against the paper's own
closed forms (Eqs. 9, 10, 12-14, 17, 20) and against exactness on polynomials;
the C oracle's double-precision weights are then checked against the exact ones.
"""
import os
from fractions import Fraction
from math import comb, factorial

import numpy as np
import pytest

from oracle import coeffs as C

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "printed_correctors.txt")


def _printed():
    rows = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].split()
        if not line:
            continue
        order = int(line[0])
        rows[order] = (Fraction(line[1]), [Fraction(t) for t in line[2:]])
    return rows


@pytest.mark.parametrize("order", [4, 6, 8])
def test_printed_beta_and_position_corrector(order):
    beta_printed, k_printed = _printed()[order]
    p = order // 2 - 1
    assert C.beta_optimal(p) == beta_printed
    _, kx = C.corrector_dt_power(p, modified=True)
    assert kx == k_printed


def test_standard_corrector_is_textbook_4th_order():
    # beta = 1: x1 - x0 = (v1+v0)dt/2 - (a1-a0)dt^2/10 + (adot1+adot0)dt^3/120
    kv, kx = C.corrector_dt_power(1, modified=False)
    assert kx == [Fraction(1, 2), Fraction(-1, 10), Fraction(1, 120)]
    # velocity: (a1+a0)dt/2 - (adot1-adot0)dt^2/12
    assert kv == [Fraction(1, 2), Fraction(-1, 12)]


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_beta_eq20_equals_eq17_with_unit_ratio(p):
    assert C.beta_optimal(p) == C.beta_from_integral_ratio(p)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_eq9_last_velocity_weight(p):
    cv, _ = C.corrector_fpm(p)
    assert cv[p] == Fraction(1, (-2) ** p) * Fraction(C.double_factorial(2 * p), C.double_factorial(2 * p + 1))


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_eq10_is_minus_next_order_weight(p):
    cv_next, _ = C.corrector_fpm(p + 1)
    assert C.truncation_dv(p) == -cv_next[p + 1]


@pytest.mark.parametrize("p", [1, 2, 3, 4])
def test_eq14_beta_shift_of_last_position_weight(p):
    beta = C.beta_optimal(p)
    _, cx_mod = C.corrector_fpm(p, True)
    _, cx_std = C.corrector_fpm(p, False)
    assert cx_mod[p + 1] - cx_std[p + 1] == C.truncation_dx(p, beta)
    # and the (p+1, p+1) element of A^-1 is 1/2^(p+1) (text under Eq. 13)
    Ai = C.mat_inverse(C.pascal_even_A(p + 2))
    assert Ai[p + 1][p + 1] == Fraction(1, 2 ** (p + 1))


@pytest.mark.parametrize("size", [2, 3, 4, 5, 6])
def test_lu_closed_forms_factor_A_transpose(size):
    # Eqs. 12-13 give the inverse factors of A^T: (U^-1 L^-1)^T = A^-1
    Ai = C.mat_inverse(C.pascal_even_A(size))
    prod = C.mat_mul(C.U_inverse_closed(size), C.L_inverse_closed(size))
    assert C.transpose(prod) == Ai


def _fpm_monomial(deg, n, h=Fraction(1)):
    """F+-_n (Eq. 5) of f(t) = t^deg about t = 0 with half-step h."""
    s = 1 if n % 2 == 0 else -1
    return Fraction(1, 2) * comb(deg, n) * (h ** (deg - n) + s * (-h) ** (deg - n)) * h ** n


@pytest.mark.parametrize("p", [1, 2, 3])
def test_quadrature_exact_on_polynomials(p):
    """Velocity weights integrate a(t) exactly through degree 2p+1 (order
    2(p+1)); beta = 1 position weights integrate v exactly through degree 2p+3;
    the beta term of Eq. 7 leaves the error (1-beta)/(2p+3) F_2p+2 on t^(2p+2)."""
    cv, cx_mod = C.corrector_fpm(p, True)
    _, cx_std = C.corrector_fpm(p, False)
    exact = lambda deg: Fraction(1, deg + 1) if deg % 2 == 0 else Fraction(0)  # (1/dt) int_{-h}^{h} t^deg, h=1
    for deg in range(0, 2 * p + 2):
        assert sum(cv[n] * _fpm_monomial(deg, n) for n in range(p + 1)) == exact(deg)
    assert sum(cv[n] * _fpm_monomial(2 * p + 2, n) for n in range(p + 1)) != exact(2 * p + 2)
    for deg in range(0, 2 * p + 4):
        assert sum(cx_std[n] * _fpm_monomial(deg, n) for n in range(p + 2)) == exact(deg)
    beta = C.beta_optimal(p)
    deg = 2 * p + 2
    err = exact(deg) - sum(cx_mod[n] * _fpm_monomial(deg, n) for n in range(p + 2))
    assert err == (1 - beta) / (2 * p + 3)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("modified", [True, False])
def test_c_oracle_weights_match_exact(orc, p, modified):
    cv, cx = orc.corrector_weights(p, modified)
    cv_e, cx_e = C.corrector_fpm(p, modified)
    # the C oracle solves the (p+2)-sized Eq. 8 system in double precision; its
    # rounding grows with the size and conditioning of the Pascal matrix
    # (measured 4.8e-15 relative at p = 4; at p = 5 up to 1.3e-13 relative, 7e-16
    # absolute, on the smallest, highest-order weight)
    rtol = {4: 2e-14, 5: 3e-13}.get(p, 2e-15)
    np.testing.assert_allclose(cv, [float(c) for c in cv_e], rtol=rtol, atol=1e-16)
    np.testing.assert_allclose(cx, [float(c) for c in cx_e], rtol=rtol, atol=1e-16)
    assert orc.beta(p) == pytest.approx(float(C.beta_optimal(p)), rel=1e-15)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_c_oracle_corrector_exact_on_polynomial_trajectory(orc, p):
    """With beta = 1 the corrector integrates a polynomial trajectory of degree
    2p+3 in x exactly; with the modified beta the position error on such a
    trajectory is the beta term alone."""
    order = 2 * (p + 1)
    rng = np.random.default_rng(7)
    deg = 2 * p + 3
    coef = rng.normal(size=(deg + 1, 3))        # x(t) = sum_k coef_k t^k
    dt = 0.37
    def deriv(k, t):
        out = np.zeros(3)
        for j in range(k, deg + 1):
            out += coef[j] * factorial(j) / factorial(j - k) * t ** (j - k)
        return out
    x0, v0 = deriv(0, 0.0)[None], deriv(1, 0.0)[None]
    d0 = np.array([[deriv(k + 2, 0.0) for k in range(p + 1)]])
    d1 = np.array([[deriv(k + 2, dt) for k in range(p + 1)]])
    # velocity update does not use v1; feed exact a-derivatives
    x1, v1 = orc.correct(order, dt, x0, v0, d0, d1, modified=False)
    np.testing.assert_allclose(v1[0], deriv(1, dt), rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(x1[0], deriv(0, dt), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_c_oracle_hermite_interp_exact_on_polynomials(orc, p):
    rng = np.random.default_rng(11)
    deg = 2 * p + 1
    coef = rng.normal(size=(deg + 1, 3))
    dt = 0.29
    def deriv(k, t):
        out = np.zeros(3)
        for j in range(k, deg + 1):
            out += coef[j] * factorial(j) / factorial(j - k) * t ** (j - k)
        return out
    f0 = np.array([deriv(k, 0.0) for k in range(p + 1)])
    f1 = np.array([deriv(k, dt) for k in range(p + 1)])
    out = orc.hermite_interp(p, dt, f0, f1, 2 * p + 2)
    ref = np.array([deriv(k, dt) for k in range(2 * p + 2)])
    scale = np.array([dt ** k / factorial(k) for k in range(2 * p + 2)])[:, None]
    np.testing.assert_allclose(out * scale, ref * scale, rtol=0, atol=1e-12 * np.abs(ref * scale).max())


# --------------------------------------------------------------------------- #
# the GPU library's constants (csrc/hermite_consts.cuh, derived by
# csrc/derive_constants.py through the two-point Hermite interpolant) against
# the oracle's exact algebra (the Eq. 8 system): two independent derivations
# --------------------------------------------------------------------------- #

CSRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2006_02501_gb300", "csrc")


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_derivation_script_matches_exact_algebra(p):
    sp = pytest.importorskip("sympy")
    import importlib.util
    spec = importlib.util.spec_from_file_location("derive_constants", os.path.join(CSRC, "derive_constants.py"))
    D = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(D)
    kv_e, kx_mod_e = C.corrector_dt_power(p, True)
    _, kx_std_e = C.corrector_dt_power(p, False)
    to_f = lambda xs: [Fraction(int(sp.Rational(x).p), int(sp.Rational(x).q)) for x in xs]
    # both give the coefficient of f1^(n) (on f1^(n) + f0^(n) for even n, f1^(n) - f0^(n) for odd n)
    assert to_f(D.integral_coeffs(p)[0]) == kv_e
    assert to_f(D.modified_position_coeffs(p)[0]) == kx_mod_e
    assert to_f(D.integral_coeffs(p + 1)[0]) == kx_std_e


def _header_values():
    """kv, kx (both beta modes), e1, e0 of hermite_consts.cuh, compiled for the host."""
    import subprocess
    import tempfile
    src = r"""
#include <cstdio>
#include "hermite_consts.cuh"
template <int p> void dump() {
    for (int k = 0; k <= p; ++k) std::printf("kv %d %d %.17g\n", p, k, mh::kv<p>(k));
    for (int b = 0; b < 2; ++b)
        for (int k = 0; k <= p + 1; ++k) std::printf("kx%d %d %d %.17g\n", b, p, k, mh::kx<p>(b, k));
    for (int n = p + 1; n < 2 * p; ++n)
        for (int k = 0; k <= p; ++k)
            std::printf("e %d %d %d %.17g %.17g\n", p, n, k, mh::e1<p>(n, k), mh::e0<p>(n, k));
}
int main() { dump<1>(); dump<2>(); dump<3>(); dump<4>(); dump<5>(); return 0; }
"""
    with tempfile.TemporaryDirectory() as td:
        cpp = os.path.join(td, "dump.cpp")
        exe = os.path.join(td, "dump")
        open(cpp, "w").write(src)
        subprocess.run(["g++", "-std=c++17", "-D__host__=", "-D__device__=", "-I", CSRC, cpp, "-o", exe], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    vals = {}
    for line in out.splitlines():
        t = line.split()
        if t[0] == "e":
            vals[("e", int(t[1]), int(t[2]), int(t[3]))] = (float(t[4]), float(t[5]))
        else:
            vals[(t[0], int(t[1]), int(t[2]))] = float(t[3])
    return vals


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_gpu_header_constants_match_oracle(orc, p):
    import shutil
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    H = _header_values()
    kv_e, kx_mod_e = C.corrector_dt_power(p, True)
    _, kx_std_e = C.corrector_dt_power(p, False)
    f = lambda xs: [float(x) for x in xs]
    np.testing.assert_allclose([H[("kv", p, k)] for k in range(p + 1)], f(kv_e), rtol=1e-15)
    np.testing.assert_allclose([H[("kx0", p, k)] for k in range(p + 2)], f(kx_mod_e), rtol=1e-15)
    np.testing.assert_allclose([H[("kx1", p, k)] for k in range(p + 2)], f(kx_std_e), rtol=1e-15)
    # end derivatives: the oracle's interpolation with dt = 1 applied to unit vectors
    for k in range(p + 1):
        for side in (0, 1):
            f0 = np.zeros((p + 1, 3))
            f1 = np.zeros((p + 1, 3))
            (f1 if side else f0)[k, 0] = 1.0
            out = orc.hermite_interp(p, 1.0, f0, f1, 2 * p)
            for n in range(p + 1, 2 * p):
                want = out[n, 0]
                got = H[("e", p, n, k)][0 if side else 1]
                assert got == pytest.approx(want, rel=1e-11, abs=1e-9), (p, n, k, side)
