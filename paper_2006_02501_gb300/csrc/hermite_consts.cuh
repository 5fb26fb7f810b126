// Rational constants of the modified Hermite corrector and the end-of-step
// Hermite interpolation, in "dt-power" form.  derive_constants.py in this
// directory reproduces every value below except the modified position
// correctors, which are the ones printed in Dittmann (2020), Section 2.1,
// Eqs. 21 (4th order), 22 (6th) and 23 (8th).
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

// Binomial coefficient as a compile-time constant.
__host__ __device__ constexpr double binom(int n, int k)
{
    return (k < 0 || k > n) ? 0.0 : (k == 0 || k == n) ? 1.0 : binom(n - 1, k - 1) + binom(n - 1, k);
}

__host__ __device__ constexpr double inv_fact(int n)
{
    return n <= 1 ? 1.0 : inv_fact(n - 1) / n;
}

}  // namespace mh
