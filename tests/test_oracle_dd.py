"""Pins for the binary128 oracle of the double-double form (oracle/mh_oracle_q.c)
and for the double-double constants header of the CUDA library.

The binary128 oracle takes the FP64 oracle's steps with every operation in IEEE
binary128.  It is pinned to things other than itself:
  - the exact rational corrector weights (oracle/coeffs.py, itself pinned to the
    correctors printed in Section 2.1) to ~1e-30;
  - Hermite interpolation that is exact on polynomials of degree 2p+1 (Eqs. 2-5);
  - the FP64 oracle on a few-body system, to FP64 rounding (a dropped term, a
    wrong sign or index shows up at O(1) there);
  - Kepler's equation, solved to 45 digits with mpmath: the position error
    after one e = 0.5 orbit keeps falling at the scheme's order (8 and 12) to
    1e-16 and 1e-21, where the FP64 oracle has stalled at its round-off;
  - time symmetry: 100 steps forward and back return to the start to 1e-30;
  - closed forms on exact Kepler states: energy -G M m / (2a) and the
    eccentricity vector (e, 0, 0), to 1e-30;
  - Section 3.1's Kepler test (a = 1, e = 0.1, dt = 2^-4, n = 3): the 10th- and
    12th-order schemes keep the energy error 1e-3 to 1e-7 times below the FP64
    run's round-off level, the extended-precision case of the Discussion.
"""
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

from oracle import coeffs as C
from paper_2006_02501_gb300 import inputs as I

mp = pytest.importorskip("mpmath")
CSRC = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2006_02501_gb300", "csrc")


def _frac(pair):
    return Fraction(float(pair[0])) + Fraction(float(pair[1]))


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("modified", [True, False])
def test_weights_exact_to_binary128(orc, p, modified):
    cv, cx = orc.dd_corrector_weights(p, modified)
    cv_e, cx_e = C.corrector_fpm(p, modified)
    for got, want in list(zip(cv, cv_e)) + list(zip(cx, cx_e)):
        assert abs(_frac(got) - want) <= Fraction(1, 10 ** 30) * abs(want), (p, got, want)


@pytest.mark.parametrize("p", [2, 3, 4, 5])
def test_hermite_interp_exact_on_polynomials(orc, p):
    """Degree-(2p+1) polynomial with small integer coefficients, dt = 1/4: every
    input is an exact double and the interpolant reproduces the polynomial."""
    rng = np.random.default_rng(3 + p)
    deg = 2 * p + 1
    coef = [[int(c) for c in rng.integers(-9, 10, size=3)] for _ in range(deg + 1)]
    dt = Fraction(1, 4)

    def deriv(k, t):
        out = [Fraction(0)] * 3
        for j in range(k, deg + 1):
            fall = 1
            for q in range(k):
                fall *= j - q
            for c in range(3):
                out[c] += coef[j][c] * fall * t ** (j - k)
        return out

    f0 = np.array([[[float(q), 0.0] for q in deriv(k, Fraction(0))] for k in range(p + 1)])
    f1 = np.array([[[float(q), 0.0] for q in deriv(k, dt)] for k in range(p + 1)])
    out = orc.dd_hermite_interp(p, float(dt), f0, f1, 2 * p)
    for n in range(2 * p):
        want = deriv(n, dt)
        scale = max(abs(w) for w in want) + 1
        for c in range(3):
            assert abs(_frac(out[n, c]) - want[c]) <= Fraction(1, 10 ** 27) * scale, (p, n, c)


def _planets(N=7, seed=21):
    offs, m, x, v, pmin = I.planetary_systems(seed=seed, S=1, nmin=N, nmax=N)
    return m, x, v, float(pmin[0])


@pytest.mark.parametrize("order", [4, 8, 12])
def test_agrees_with_fp64_oracle(orc, order):
    m, x, v, pmin = _planets()
    dt = pmin / 64
    p = order // 2 - 1
    x2, v2, d2 = orc.dd_run(order, m, x, v, 0.0, dt, 3, 0)
    d64 = orc.initialise(order, m, x, v, 0.0)
    K = 2 * p
    for k in range(K):
        ref = d64[:, k]
        assert np.abs(orc.dd_value(d2[:, k]) - ref).max() <= 1e-12 * np.abs(ref).max(), k
    x2, v2, d2 = orc.dd_run(order, m, x, v, 0.0, dt, 3, 10)
    S = orc.State(order, m, x, v, 0.0)
    S.step(dt, 3, 10)
    assert np.abs(orc.dd_value(x2) - S.x).max() <= 1e-13 * np.abs(S.x).max()
    assert np.abs(orc.dd_value(v2) - S.v).max() <= 1e-12 * np.abs(S.v).max()


def _kepler_ref(m, x, v, t):
    """Relative position at time t on the exact Kepler orbit through the given
    (double) initial state, from the f and g functions and Kepler's equation in
    eccentric-anomaly differences, solved by Newton's method at 45 digits."""
    with mp.workdps(45):
        r0 = [mp.mpf(x[1, c]) - mp.mpf(x[0, c]) for c in range(3)]
        v0 = [mp.mpf(v[1, c]) - mp.mpf(v[0, c]) for c in range(3)]
        mu = mp.mpf(m[0]) + mp.mpf(m[1])
        rn = mp.sqrt(sum(q * q for q in r0))
        a = 1 / (2 / rn - sum(q * q for q in v0) / mu)
        sig = sum(r0[c] * v0[c] for c in range(3)) / mp.sqrt(mu)
        n = mp.sqrt(mu / a ** 3)
        M = n * t
        E = M
        for _ in range(200):
            f = E + sig / mp.sqrt(a) * (1 - mp.cos(E)) - (1 - rn / a) * mp.sin(E) - M
            fp = 1 + sig / mp.sqrt(a) * mp.sin(E) - (1 - rn / a) * mp.cos(E)
            dE = f / fp
            E -= dE
            if abs(dE) < mp.mpf(10) ** -42:
                break
        F = 1 - a / rn * (1 - mp.cos(E))
        G = t - (E - mp.sin(E)) / n
        return [F * r0[c] + G * v0[c] for c in range(3)]


def _pos_err(x2, ref):
    with mp.workdps(45):
        r = [(mp.mpf(x2[1, c, 0]) + mp.mpf(x2[1, c, 1])) - (mp.mpf(x2[0, c, 0]) + mp.mpf(x2[0, c, 1]))
             for c in range(3)]
        return float(mp.sqrt(sum((r[c] - ref[c]) ** 2 for c in range(3))))


@pytest.mark.parametrize("order,steps,floor", [(8, (512, 1024), 1e-16), (12, (256, 512), 1e-20)])
def test_kepler_order_below_fp64_roundoff(orc, order, steps, floor):
    m, x, v = I.kepler_pair(a=1.0, e=0.5, M=1.0, m=1e-3)
    T = 2 * np.pi / np.sqrt(1.001)
    errs, errs64 = [], []
    for n in steps:
        dt = T / n
        with mp.workdps(45):
            ref = _kepler_ref(m, x, v, mp.mpf(dt) * n)
        x2, _, _ = orc.dd_run(order, m, x, v, 0.0, dt, 3, n)
        errs.append(_pos_err(x2, ref))
        S = orc.State(order, m, x, v, 0.0)
        S.step(dt, 3, n)
        errs64.append(_pos_err(np.stack([S.x, np.zeros_like(S.x)], -1), ref))
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.4, (errs, slope)
    assert errs[1] < floor, errs
    # the FP64 oracle cannot follow: its error at the finer step is round-off
    assert errs64[1] > 50 * errs[1], (errs64, errs)


@pytest.mark.parametrize("order,bound", [(10, 1e-17), (12, 1e-21)])
def test_section31_energy_below_fp64(orc, order, bound):
    """a = 1, e = 0.1, dt = 2^-4, n = 3 (the Section 3.1 Kepler test), 10 orbits."""
    m, x, v = I.kepler_pair(a=1.0, e=0.1, M=1.0, m=1e-3)
    dt = 2.0 ** -4
    E0 = orc.dd_energy(m, orc.as_dd(x), orc.as_dd(v), 0.0)
    x2, v2, d2 = orc.dd_run(order, m, x, v, 0.0, dt, 3, 0)
    S = orc.State(order, m, x, v, 0.0)
    E0f = S.energy()
    worst, worst64 = 0.0, 0.0
    with mp.workdps(45):
        e0 = mp.mpf(E0[0]) + mp.mpf(E0[1])
        for _ in range(20):
            x2, v2, d2 = orc.dd_run(order, m, x2, v2, 0.0, dt, 3, 50, d2=d2)
            E = orc.dd_energy(m, x2, v2, 0.0)
            worst = max(worst, float(abs((mp.mpf(E[0]) + mp.mpf(E[1]) - e0) / e0)))
            S.step(dt, 3, 50)
            worst64 = max(worst64, abs(S.energy() / E0f - 1))
    assert worst < bound, worst
    assert worst64 > 3e-16, worst64          # the FP64 run sits at its round-off level
    assert worst < worst64 / 1000


def test_energy_and_ecc_agree_with_fp64_oracle(orc):
    m, x, v, _ = _planets()
    E2 = orc.dd_energy(m, orc.as_dd(x), orc.as_dd(v), 1e-3)
    assert orc.dd_value(E2) == pytest.approx(orc.energy(m, x, v, 1e-3), rel=1e-14)
    e2 = orc.dd_ecc(m, orc.as_dd(x), orc.as_dd(v), 1.0, 0)
    np.testing.assert_allclose(orc.dd_value(e2), orc.ecc(m, x, v, 1.0, 0), rtol=0, atol=1e-14)


# --------------------------------------------------------------------------- #
# the CUDA library's double-double constants (csrc/hermite_consts_dd.cuh)
# --------------------------------------------------------------------------- #

def _dd_header_values():
    src = r"""
#include <cstdio>
#include "hermite_consts_dd.cuh"
using namespace mh::ddc;
#define DUMP(P, KV, KX, E1, E0)                                                            \
    for (int k = 0; k <= P; ++k) std::printf("kv %d %d %lld %lld\n", P, k, KV(k).num, KV(k).den); \
    for (int b = 0; b < 2; ++b) for (int k = 0; k <= P + 1; ++k)                          \
        std::printf("kx%d %d %d %lld %lld\n", b, P, k, KX(b, k).num, KX(b, k).den);
#define DUMPE(P, E1, E0)                                                                   \
    for (int n = P + 1; n < 2 * P; ++n) for (int k = 0; k <= P; ++k)                      \
        std::printf("e %d %d %d %lld %lld %lld %lld\n", P, n, k, E1(n, k).num, E1(n, k).den, \
                    E0(n, k).num, E0(n, k).den);
int main() {
    DUMP(1, kv1, kx1, 0, 0) DUMP(2, kv2, kx2, 0, 0) DUMP(3, kv3, kx3, 0, 0)
    DUMP(4, kv4, kx4, 0, 0) DUMP(5, kv5, kx5, 0, 0)
    DUMPE(2, e1_2, e0_2) DUMPE(3, e1_3, e0_3) DUMPE(4, e1_4, e0_4) DUMPE(5, e1_5, e0_5)
    return 0;
}
"""
    with tempfile.TemporaryDirectory() as td:
        cpp, exe = os.path.join(td, "dump.cpp"), os.path.join(td, "dump")
        open(cpp, "w").write(src)
        subprocess.run(["g++", "-std=c++17", "-D__host__=", "-D__device__=", "-I", CSRC, cpp, "-o", exe],
                       check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    vals = {}
    for line in out.splitlines():
        t = line.split()
        if t[0] == "e":
            vals[("e", int(t[1]), int(t[2]), int(t[3]))] = (Fraction(int(t[4]), int(t[5])),
                                                           Fraction(int(t[6]), int(t[7])))
        else:
            vals[(t[0], int(t[1]), int(t[2]))] = Fraction(int(t[3]), int(t[4]))
    return vals


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
def test_dd_header_constants_exact(orc, p):
    import shutil
    if shutil.which("g++") is None:
        pytest.skip("no host C++ compiler")
    H = _dd_header_values()
    kv_e, kx_mod_e = C.corrector_dt_power(p, True)
    _, kx_std_e = C.corrector_dt_power(p, False)
    assert [H[("kv", p, k)] for k in range(p + 1)] == kv_e
    assert [H[("kx0", p, k)] for k in range(p + 2)] == kx_mod_e
    assert [H[("kx1", p, k)] for k in range(p + 2)] == kx_std_e
    # end derivatives: the binary128 interpolation (dt = 1) of unit vectors
    for k in range(p + 1):
        for side in (0, 1):
            f0, f1 = np.zeros((p + 1, 3, 2)), np.zeros((p + 1, 3, 2))
            (f1 if side else f0)[k, 0, 0] = 1.0
            out = orc.dd_hermite_interp(p, 1.0, f0, f1, 2 * p)
            for n in range(p + 1, 2 * p):
                got = H[("e", p, n, k)][0 if side else 1]
                want = _frac(out[n, 0])
                assert abs(got - want) <= Fraction(1, 10 ** 20) * max(1, abs(want)), (p, n, k, side)


def test_dd_header_is_the_derivation_scripts_output():
    """The committed hermite_consts_dd.cuh is exactly what
    `derive_constants.py --dd-header` writes."""
    pytest.importorskip("sympy")
    import importlib.util
    spec = importlib.util.spec_from_file_location("derive_constants", os.path.join(CSRC, "derive_constants.py"))
    D = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(D)
    with open(os.path.join(CSRC, "hermite_consts_dd.cuh")) as f:
        assert f.read() == D.dd_header()


@pytest.mark.parametrize("order", [8, 12])
def test_time_symmetric_to_binary128(orc, order):
    """The modified Hermite step with converged iterations is time symmetric
    (Section 2: the corrector's F+ terms are even, the F- terms odd in dt): 100
    steps forward and 100 back return to the start to ~1e-32, the rounding of
    the state to a double-double pair between the two runs."""
    m, x, v = I.kepler_pair(a=1.0, e=0.5, M=1.0, m=1e-3)
    dt = 2.0 ** -6
    x2, v2, d2 = orc.dd_run(order, m, x, v, 0.0, dt, 10, 100)
    xb, vb, _ = orc.dd_run(order, m, x2, v2, 0.0, -dt, 10, 100, d2=d2)
    assert np.abs((xb[..., 0] - x) + xb[..., 1]).max() < 1e-30
    assert np.abs((vb[..., 0] - v) + vb[..., 1]).max() < 1e-30
    # and the run went somewhere: 100 steps are a quarter orbit
    assert np.abs(orc.dd_value(x2) - x).max() > 0.1


def _dd_of(q):
    hi = float(q)
    return [hi, float(q - mp.mpf(hi))]


@pytest.mark.parametrize("e,M_anom", [(0.5, 1.0), (0.1, 2.5), (0.9, 0.3)])
def test_energy_and_ecc_closed_forms(orc, e, M_anom):
    """A two-body state on an exact Kepler orbit (built at 45 digits, rounded to
    double-double pairs): the barycentric energy is -G M m / (2a) and the
    eccentricity vector of the companion is (e, 0, 0) (Appendix A, periapsis on
    the x axis), both to ~1e-30."""
    M, m_, a, G = 1.0, 1e-3, 1.0, 1.0
    with mp.workdps(45):
        mu = mp.mpf(G) * (mp.mpf(M) + mp.mpf(m_))
        E = mp.mpf(M_anom)
        for _ in range(100):
            E -= (E - e * mp.sin(E) - M_anom) / (1 - e * mp.cos(E))
        b = mp.sqrt(1 - mp.mpf(e) ** 2)
        r = [a * (mp.cos(E) - e), a * b * mp.sin(E), mp.mpf(0)]
        w = mp.sqrt(mu / a) / (1 - e * mp.cos(E))
        u = [-w * mp.sin(E), w * b * mp.cos(E), mp.mpf(0)]
        Mt = mp.mpf(M) + mp.mpf(m_)
        f0, f1 = -mp.mpf(m_) / Mt, mp.mpf(M) / Mt
        x2 = np.array([[_dd_of(f0 * q) for q in r], [_dd_of(f1 * q) for q in r]])
        v2 = np.array([[_dd_of(f0 * q) for q in u], [_dd_of(f1 * q) for q in u]])
        E_exact = -mp.mpf(G) * mp.mpf(M) * mp.mpf(m_) / (2 * a)
        E2 = orc.dd_energy(np.array([M, m_]), x2, v2, 0.0, G)
        assert abs((mp.mpf(E2[0]) + mp.mpf(E2[1]) - E_exact) / E_exact) < 1e-30
        e2 = orc.dd_ecc(np.array([M, m_]), x2, v2, G, 0)
        got = [mp.mpf(e2[1, c, 0]) + mp.mpf(e2[1, c, 1]) for c in range(3)]
        assert abs(got[0] - e) < 1e-30 and abs(got[1]) < 1e-30 and got[2] == 0
        assert not e2[0].any()
