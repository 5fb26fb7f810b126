// Rational constants of the modified Hermite corrector and the end-of-step
// Hermite interpolation, in "dt-power" form, for orders 4 to 12.
// derive_constants.py in this directory reproduces every value below; for
// orders 4, 6, 8 the modified position correctors are the ones printed in
// Dittmann (2020), Section 2.1, Eqs. 21, 22 and 23, which that script checks.
//
// Velocity corrector (Eq. 6, f = a):
//   v1 - v0 = sum_k kv(k) (a1^(k) + (-1)^k a0^(k)) dt^(k+1),   k = 0 .. p
// Position corrector (Eq. 7, f = v, v^(k) = a^(k-1)):
//   x1 - x0 = sum_k kx(b, k) (v1^(k) + (-1)^k v0^(k)) dt^(k+1),   k = 0 .. p+1
// End derivatives (degree 2p+1 Hermite interpolant through a^(0..p) at t0, t1):
//   a^(n)(t1) = sum_k (e1(n, k) a1^(k) + e0(n, k) a0^(k)) dt^(k-n)
#pragma once

namespace mh {

// kv<p>(k), kx<p>(beta_mode, k), e1<p>(n, k), e0<p>(n, k); n counts from p+1.
template <int p> __host__ __device__ constexpr double kv(int k);
template <int p> __host__ __device__ constexpr double kx(int beta_mode, int k);
template <int p> __host__ __device__ constexpr double e1(int n, int k);
template <int p> __host__ __device__ constexpr double e0(int n, int k);

// ---- 4th order (p = 1) ----
template <> __host__ __device__ constexpr double kv<1>(int k)
{
    return k == 0 ? 1.0 / 2.0 : -1.0 / 12.0;
}
template <> __host__ __device__ constexpr double kx<1>(int b, int k)
{
    return b == 0 ? (k == 0 ? 1.0 / 2.0 : k == 1 ? -7.0 / 60.0 : 1.0 / 60.0)       // Eq. 21
                  : (k == 0 ? 1.0 / 2.0 : k == 1 ? -1.0 / 10.0 : 1.0 / 120.0);
}
template <> __host__ __device__ constexpr double e1<1>(int, int) { return 0.0; }
template <> __host__ __device__ constexpr double e0<1>(int, int) { return 0.0; }

// ---- 6th order (p = 2) ----
template <> __host__ __device__ constexpr double kv<2>(int k)
{
    return k == 0 ? 1.0 / 2.0 : k == 1 ? -1.0 / 10.0 : 1.0 / 120.0;
}
template <> __host__ __device__ constexpr double kx<2>(int b, int k)
{
    return b == 0 ? (k == 0 ? 1.0 / 2.0 : k == 1 ? -4.0 / 35.0 : k == 2 ? 13.0 / 840.0 : -1.0 / 840.0)  // Eq. 22
                  : (k == 0 ? 1.0 / 2.0 : k == 1 ? -3.0 / 28.0 : k == 2 ? 1.0 / 84.0 : -1.0 / 1680.0);
}
// a^(3)(t1)
template <> __host__ __device__ constexpr double e1<2>(int, int k)
{
    return k == 0 ? 60.0 : k == 1 ? -36.0 : 9.0;
}
template <> __host__ __device__ constexpr double e0<2>(int, int k)
{
    return k == 0 ? -60.0 : k == 1 ? -24.0 : -3.0;
}

// ---- 8th order (p = 3) ----
template <> __host__ __device__ constexpr double kv<3>(int k)
{
    return k == 0 ? 1.0 / 2.0 : k == 1 ? -3.0 / 28.0 : k == 2 ? 1.0 / 84.0 : -1.0 / 1680.0;
}
template <> __host__ __device__ constexpr double kx<3>(int b, int k)
{
    return b == 0 ? (k == 0 ? 1.0 / 2.0 : k == 1 ? -29.0 / 252.0 : k == 2 ? 1.0 / 63.0
                     : k == 3 ? -1.0 / 720.0 : 1.0 / 15120.0)                        // Eq. 23
                  : (k == 0 ? 1.0 / 2.0 : k == 1 ? -1.0 / 9.0 : k == 2 ? 1.0 / 72.0
                     : k == 3 ? -1.0 / 1008.0 : 1.0 / 30240.0);
}
// a^(4)(t1) (n = 4) and a^(5)(t1) (n = 5)
template <> __host__ __device__ constexpr double e1<3>(int n, int k)
{
    return n == 4 ? (k == 0 ? -840.0 : k == 1 ? 480.0 : k == 2 ? -120.0 : 16.0)
                  : (k == 0 ? -10080.0 : k == 1 ? 5400.0 : k == 2 ? -1200.0 : 120.0);
}
template <> __host__ __device__ constexpr double e0<3>(int n, int k)
{
    return n == 4 ? (k == 0 ? 840.0 : k == 1 ? 360.0 : k == 2 ? 60.0 : 4.0)
                  : (k == 0 ? 10080.0 : k == 1 ? 4680.0 : k == 2 ? 840.0 : 60.0);
}

// ---- 10th order (p = 4): not printed in the paper; the velocity and standard
// position correctors and the end derivatives from the two-point Hermite interpolant,
// the modified position corrector from Eq. 7 with beta = -193/63 (Eq. 20) ----
template <> __host__ __device__ constexpr double kv<4>(int k)
{
    switch (k) {
    case 0: return 1.0 / 2.0;
    case 1: return -1.0 / 9.0;
    case 2: return 1.0 / 72.0;
    case 3: return -1.0 / 1008.0;
    case 4: return 1.0 / 30240.0;
    }
    return 0.0;
}
template <> __host__ __device__ constexpr double kx<4>(int b, int k)
{
    if (b == 0) {
        switch (k) {
        case 0: return 1.0 / 2.0;
        case 1: return -23.0 / 198.0;
        case 2: return 13.0 / 792.0;
        case 3: return -17.0 / 11088.0;
        case 4: return 31.0 / 332640.0;
        case 5: return -1.0 / 332640.0;
        }
        return 0.0;
    }
    switch (k) {
    case 0: return 1.0 / 2.0;
    case 1: return -5.0 / 44.0;
    case 2: return 1.0 / 66.0;
    case 3: return -1.0 / 792.0;
    case 4: return 1.0 / 15840.0;
    case 5: return -1.0 / 665280.0;
    }
    return 0.0;
}
template <> __host__ __device__ constexpr double e1<4>(int n, int k)
{
    switch (n * 16 + k) {
    case 5 * 16 + 0: return 15120.0;
    case 5 * 16 + 1: return -8400.0;
    case 5 * 16 + 2: return 2100.0;
    case 5 * 16 + 3: return -300.0;
    case 5 * 16 + 4: return 25.0;
    case 6 * 16 + 0: return 302400.0;
    case 6 * 16 + 1: return -161280.0;
    case 6 * 16 + 2: return 37800.0;
    case 6 * 16 + 3: return -4800.0;
    case 6 * 16 + 4: return 300.0;
    case 7 * 16 + 0: return 2721600.0;
    case 7 * 16 + 1: return -1411200.0;
    case 7 * 16 + 2: return 317520.0;
    case 7 * 16 + 3: return -37800.0;
    case 7 * 16 + 4: return 2100.0;
    }
    return 0.0;
}
template <> __host__ __device__ constexpr double e0<4>(int n, int k)
{
    switch (n * 16 + k) {
    case 5 * 16 + 0: return -15120.0;
    case 5 * 16 + 1: return -6720.0;
    case 5 * 16 + 2: return -1260.0;
    case 5 * 16 + 3: return -120.0;
    case 5 * 16 + 4: return -5.0;
    case 6 * 16 + 0: return -302400.0;
    case 6 * 16 + 1: return -141120.0;
    case 6 * 16 + 2: return -27720.0;
    case 6 * 16 + 3: return -2760.0;
    case 6 * 16 + 4: return -120.0;
    case 7 * 16 + 0: return -2721600.0;
    case 7 * 16 + 1: return -1310400.0;
    case 7 * 16 + 2: return -267120.0;
    case 7 * 16 + 3: return -27720.0;
    case 7 * 16 + 4: return -1260.0;
    }
    return 0.0;
}

// ---- 12th order (p = 5): not printed in the paper; the velocity and standard
// position correctors and the end derivatives from the two-point Hermite interpolant,
// the modified position corrector from Eq. 7 with beta = 1255/231 (Eq. 20) ----
template <> __host__ __device__ constexpr double kv<5>(int k)
{
    switch (k) {
    case 0: return 1.0 / 2.0;
    case 1: return -5.0 / 44.0;
    case 2: return 1.0 / 66.0;
    case 3: return -1.0 / 792.0;
    case 4: return 1.0 / 15840.0;
    case 5: return -1.0 / 665280.0;
    }
    return 0.0;
}
template <> __host__ __device__ constexpr double kx<5>(int b, int k)
{
    if (b == 0) {
        switch (k) {
        case 0: return 1.0 / 2.0;
        case 1: return -67.0 / 572.0;
        case 2: return 29.0 / 1716.0;
        case 3: return -17.0 / 10296.0;
        case 4: return 23.0 / 205920.0;
        case 5: return -43.0 / 8648640.0;
        case 6: return 1.0 / 8648640.0;
        }
        return 0.0;
    }
    switch (k) {
    case 0: return 1.0 / 2.0;
    case 1: return -3.0 / 26.0;
    case 2: return 5.0 / 312.0;
    case 3: return -5.0 / 3432.0;
    case 4: return 1.0 / 11440.0;
    case 5: return -1.0 / 308880.0;
    case 6: return 1.0 / 17297280.0;
    }
    return 0.0;
}
template <> __host__ __device__ constexpr double e1<5>(int n, int k)
{
    switch (n * 16 + k) {
    case 6 * 16 + 0: return -332640.0;
    case 6 * 16 + 1: return 181440.0;
    case 6 * 16 + 2: return -45360.0;
    case 6 * 16 + 3: return 6720.0;
    case 6 * 16 + 4: return -630.0;
    case 6 * 16 + 5: return 36.0;
    case 7 * 16 + 0: return -9979200.0;
    case 7 * 16 + 1: return 5292000.0;
    case 7 * 16 + 2: return -1270080.0;
    case 7 * 16 + 3: return 176400.0;
    case 7 * 16 + 4: return -14700.0;
    case 7 * 16 + 5: return 630.0;
    case 8 * 16 + 0: return -139708800.0;
    case 8 * 16 + 1: return 72576000.0;
    case 8 * 16 + 2: return -16934400.0;
    case 8 * 16 + 3: return 2257920.0;
    case 8 * 16 + 4: return -176400.0;
    case 8 * 16 + 5: return 6720.0;
    case 9 * 16 + 0: return -1117670400.0;
    case 9 * 16 + 1: return 571536000.0;
    case 9 * 16 + 2: return -130636800.0;
    case 9 * 16 + 3: return 16934400.0;
    case 9 * 16 + 4: return -1270080.0;
    case 9 * 16 + 5: return 45360.0;
    }
    return 0.0;
}
template <> __host__ __device__ constexpr double e0<5>(int n, int k)
{
    switch (n * 16 + k) {
    case 6 * 16 + 0: return 332640.0;
    case 6 * 16 + 1: return 151200.0;
    case 6 * 16 + 2: return 30240.0;
    case 6 * 16 + 3: return 3360.0;
    case 6 * 16 + 4: return 210.0;
    case 6 * 16 + 5: return 6.0;
    case 7 * 16 + 0: return 9979200.0;
    case 7 * 16 + 1: return 4687200.0;
    case 7 * 16 + 2: return 967680.0;
    case 7 * 16 + 3: return 110880.0;
    case 7 * 16 + 4: return 7140.0;
    case 7 * 16 + 5: return 210.0;
    case 8 * 16 + 0: return 139708800.0;
    case 8 * 16 + 1: return 67132800.0;
    case 8 * 16 + 2: return 14212800.0;
    case 8 * 16 + 3: return 1673280.0;
    case 8 * 16 + 4: return 110880.0;
    case 8 * 16 + 5: return 3360.0;
    case 9 * 16 + 0: return 1117670400.0;
    case 9 * 16 + 1: return 546134400.0;
    case 9 * 16 + 2: return 117936000.0;
    case 9 * 16 + 3: return 14212800.0;
    case 9 * 16 + 4: return 967680.0;
    case 9 * 16 + 5: return 30240.0;
    }
    return 0.0;
}

// Binomial coefficient C(n, k) (exact: after step i the product is C(n-k+i, i)).
// Written as a loop, not a recursion: where a call is not folded at compile
// time it must not become a recursive device function, whose stack depth the
// compiler cannot bound.
__host__ __device__ constexpr double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// 1/n!, divided out in the order 1/2, /3, ..., /n.
__host__ __device__ constexpr double inv_fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r /= i;
    return r;
}

}  // namespace mh
