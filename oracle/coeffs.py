"""Exact rational Hermite algebra of Dittmann (2020), Section 2 and 2.1.

TEST INFRASTRUCTURE ONLY (part of the oracle): nothing in the product imports it.

Everything here is exact (``fractions.Fraction``), so the printed worked values of
the paper (beta of Eq. 20 evaluated at p = 1, 2, 3 and the position correctors of
Eqs. 21-23) can be compared with equality.

Notation follows the paper: order 2(p+1), h = dt/2, F_n = h^n f^(n)/n! (Eq. 4),
F+-_n = h^n/n! (f^(n)(t+h) +- f^(n)(t-h))/2 (Eq. 5), the even-column Pascal system
[F+_0, F-_1, F+_2, ...] = A [F_0, F_2, ...] with A_nk = C(2k, n) (Eq. 8).
"""
from fractions import Fraction
from math import comb, factorial


def double_factorial(n: int) -> int:
    r = 1
    while n > 1:
        r *= n
        n -= 2
    return r


def beta_optimal(p: int) -> Fraction:
    """Eq. 20: beta = 1 + (-1)^(p+1) (2p+2)!! / (2p+1)!!."""
    return 1 + Fraction((-1) ** (p + 1) * double_factorial(2 * p + 2), double_factorial(2 * p + 1))


def beta_from_integral_ratio(p: int) -> Fraction:
    """Eq. 17 with the ratio of integrals set to 1 (Eqs. 18-19 show the two
    integrals are equal over a Kepler period):
    beta = 1 + (2p+3) 2^(p+1) / (-2)^(p+1) * (2p+2)!! / (2p+3)!!."""
    return 1 + Fraction((2 * p + 3) * 2 ** (p + 1), (-2) ** (p + 1)) * Fraction(
        double_factorial(2 * p + 2), double_factorial(2 * p + 3))


def pascal_even_A(size: int):
    """Eq. 8: A_nk = C(2k, n), n, k = 0 .. size-1."""
    return [[Fraction(comb(2 * k, n)) for k in range(size)] for n in range(size)]


def pascal_odd_A(size: int):
    """Odd-column analogue used for interpolation: A'_nk = C(2k+1, n) mapping
    [F_1, F_3, ...] to [F-_0, F+_1, F-_2, ...] (same construction as Eq. 8
    applied to the odd columns of the Pascal matrix of Eq. 3)."""
    return [[Fraction(comb(2 * k + 1, n)) for k in range(size)] for n in range(size)]


def mat_inverse(M):
    """Exact Gauss-Jordan inverse."""
    n = len(M)
    a = [list(row) + [Fraction(int(i == j)) for j in range(n)] for i, row in enumerate(M)]
    for c in range(n):
        piv = next(r for r in range(c, n) if a[r][c] != 0)
        a[c], a[piv] = a[piv], a[c]
        pv = a[c][c]
        a[c] = [x / pv for x in a[c]]
        for r in range(n):
            if r != c and a[r][c] != 0:
                f = a[r][c]
                a[r] = [x - f * y for x, y in zip(a[r], a[c])]
    return [row[n:] for row in a]


def mat_mul(X, Y):
    return [[sum(X[i][k] * Y[k][j] for k in range(len(Y))) for j in range(len(Y[0]))]
            for i in range(len(X))]


def transpose(M):
    return [list(r) for r in zip(*M)]


def L_inverse_closed(size: int):
    """Eq. 12: L^-1_ij = (-1)^(i+j) C(i, j)."""
    return [[Fraction((-1) ** (i + j) * comb(i, j)) for j in range(size)] for i in range(size)]


def U_inverse_closed(size: int):
    """Eq. 13: U^-1_ij = (-1)^(i+j) / 2^(2j-i) * i/j * C(2j-i-1, j-i) for 1 <= i <= j,
    1 for i = j = 0, else 0."""
    def el(i, j):
        if i == 0 and j == 0:
            return Fraction(1)
        if 1 <= i <= j:
            return Fraction((-1) ** (i + j), 2 ** (2 * j - i)) * Fraction(i, j) * comb(2 * j - i - 1, j - i)
        return Fraction(0)
    return [[el(i, j) for j in range(size)] for i in range(size)]


def quadrature_weights(size: int, beta: Fraction = Fraction(1)):
    """Weights c with Delta/dt = sum_n c_n Fpm_n on [F+_0, F-_1, F+_2, ...]:
    Eqs. 6/7 put 1/(2k+1) on F_2k (beta/(2p+3) on the last term of Eq. 7) and
    Eq. 8 relates F_2k to Fpm; c = w A^-1."""
    w = [Fraction(1, 2 * k + 1) for k in range(size)]
    w[-1] *= beta
    Ai = mat_inverse(pascal_even_A(size))
    return [sum(w[k] * Ai[k][n] for k in range(size)) for n in range(size)]


def corrector_fpm(p: int, modified: bool = True):
    """(cv, cx): velocity weights (p+1 terms, Eq. 6, f = a) and position weights
    (p+2 terms, Eq. 7, f = v) on the Fpm vector."""
    beta = beta_optimal(p) if modified else Fraction(1)
    return quadrature_weights(p + 1), quadrature_weights(p + 2, beta)


def corrector_dt_power(p: int, modified: bool = True):
    """The same correctors written as coefficients of (f1^(n) +- f0^(n)) dt^(n+1),
    the form in which Eqs. 21-23 print them:
      v1 - v0 = sum_n kv_n (a1^(n) +- a0^(n)) dt^(n+1)
      x1 - x0 = sum_n kx_n (v1^(n) +- v0^(n)) dt^(n+1), v^(n) = a^(n-1)
    with + for even n and - for odd n.  Fpm_n = (1/2)(dt/2)^n/n! (...)."""
    cv, cx = corrector_fpm(p, modified)
    conv = lambda c, n: c * Fraction(1, 2) * Fraction(1, 2 ** n) / factorial(n)
    return [conv(c, n) for n, c in enumerate(cv)], [conv(c, n) for n, c in enumerate(cx)]


def truncation_dv(p: int) -> Fraction:
    """Eq. 10: delta v = -1/(-2)^(p+1) (2p+2)!!/(2p+3)!! F+-_(p+1) (coefficient)."""
    return Fraction(-1, (-2) ** (p + 1)) * Fraction(double_factorial(2 * p + 2), double_factorial(2 * p + 3))


def truncation_dx(p: int, beta: Fraction) -> Fraction:
    """Eq. 14: delta x = (beta-1)/((2p+3) 2^(p+1)) F+-_(p+1) (coefficient)."""
    return (beta - 1) / ((2 * p + 3) * 2 ** (p + 1))
