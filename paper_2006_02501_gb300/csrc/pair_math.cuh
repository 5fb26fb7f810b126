// Pair derivatives of the softened acceleration, shared by the evaluation
// kernels (pair.cu) and the batched integrator (batch.cu).
//
// Pair physics (Dittmann 2020, Section 3, intro): a_ij = G m_j r_ij s^(-3/2),
// s = r_ij^2 + eps^2.  Its time derivatives along the trajectory follow from
// T a = G m r with T = s^(3/2): differentiating n times,
//   A^(n) = G m S r^(n) - sum_{k=1..n} C(n,k) tau_k A^(n-k),   S = s^(-3/2),
//   tau_k = T^(k)/T,  tau_n = 1.5 q_n + sum_{j=1..n-1} (1.5 C(n-1,j-1) - C(n-1,j)) q_j tau_(n-j),
//   q_k = s^(k)/s,    s^(k) = sum_j C(k,j) r^(j).r^(k-j)   (eps enters s^(0) only).
#pragma once

#include "hermite_consts.cuh"

namespace mh {


// q_k = s^(k)/s for k = 1..P from the relative trajectory derivatives r[0..P].
template <int P, typename T>
__device__ __forceinline__ void s_ratios(const T (&r)[P + 1][3], T sinv, T (&q)[P + 1])
{
#pragma unroll
    for (int k = 1; k <= P; ++k) {
        T acc = T(0);
#pragma unroll
        for (int j = 0; 2 * j <= k; ++j) {
            const T w = T((2 * j == k) ? binom(k, j) : 2.0 * binom(k, j));
            const T d = r[j][0] * r[k - j][0] + r[j][1] * r[k - j][1] + r[j][2] * r[k - j][2];
            acc = (j == 0) ? w * d : acc + w * d;
        }
        q[k] = acc * sinv;
    }
}

// A^(0..P) of one pair given mS = G m s^(-3/2), q_k and r^(k); accumulated into acc.
template <int P, typename T>
__device__ __forceinline__ void pair_terms(const T (&r)[P + 1][3], T mS, const T (&q)[P + 1],
                                           T (&acc)[P + 1][3])
{
    T tau[P + 1];
    tau[0] = T(1);
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        T t = T(1.5) * q[n];
#pragma unroll
        for (int j = 1; j <= n - 1; ++j) {
            const T w = T(1.5 * binom(n - 1, j - 1) - binom(n - 1, j));
            t += w * q[j] * tau[n - j];
        }
        tau[n] = t;
    }
    T A[P + 1][3];
#pragma unroll
    for (int n = 0; n <= P; ++n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T a = mS * r[n][c];
#pragma unroll
            for (int k = 1; k <= n; ++k) a -= (T(binom(n, k)) * tau[k]) * A[n - k][c];
            A[n][c] = a;
            acc[n][c] += a;
        }
    }
}

// The same derivatives for P <= 3 written out with alpha = tau_1/3,
// beta = tau_2/3, gamma = tau_3/3 and scaled terms B_k = A^(k) / (G m S):
//   alpha = (r.v)/s,  beta = (v.v + r.a)/s + alpha^2,
//   gamma = (3 v.a + r.adot)/s + alpha (3 beta - 4 alpha^2),
//   B0 = r, B1 = v - 3 alpha B0, B2 = a - 6 alpha B1 - 3 beta B0,
//   B3 = adot - 9 alpha B2 - 9 beta B1 - 3 gamma B0.
// Every B_k is odd under the exchange i <-> j (r^(k) changes sign, alpha, beta,
// gamma and s do not), so one evaluation serves both bodies of a pair.
// sink(k, c, B) receives component c of B_k.
template <int P, typename T, typename Sink>
__device__ __forceinline__ void pair_abg_terms(const T (&r)[P + 1][3], T sinv, Sink &&sink)
{
    static_assert(P >= 1 && P <= 3, "pair_abg handles P = 1, 2, 3");
    const T rv = r[0][0] * r[1][0] + r[0][1] * r[1][1] + r[0][2] * r[1][2];
    const T al = rv * sinv;
    const T a3 = T(3) * al;
    T B1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        B1[c] = r[1][c] - a3 * r[0][c];
        sink(0, c, r[0][c]);
        sink(1, c, B1[c]);
    }
    if constexpr (P >= 2) {
        const T al2 = al * al;
        const T w2 = r[1][0] * r[1][0] + r[1][1] * r[1][1] + r[1][2] * r[1][2]
                   + r[0][0] * r[2][0] + r[0][1] * r[2][1] + r[0][2] * r[2][2];
        const T be = w2 * sinv + al2;
        const T a6 = T(6) * al, b3 = T(3) * be;
        T B2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            B2[c] = r[2][c] - a6 * B1[c] - b3 * r[0][c];
            sink(2, c, B2[c]);
        }
        if constexpr (P >= 3) {
            const T va = r[1][0] * r[2][0] + r[1][1] * r[2][1] + r[1][2] * r[2][2];
            const T w3 = T(3) * va + r[0][0] * r[3][0] + r[0][1] * r[3][1] + r[0][2] * r[3][2];
            const T ga = w3 * sinv + al * (b3 - T(4) * al2);
            const T a9 = T(9) * al, b9 = T(9) * be, g3 = T(3) * ga;
#pragma unroll
            for (int c = 0; c < 3; ++c) sink(3, c, r[3][c] - a9 * B2[c] - b9 * B1[c] - g3 * r[0][c]);
        }
    }
}

// The scaled terms B^(n) = A^(n) / (G m S) of the general recursion, for any P:
// B^(0) = r, B^(n) = r^(n) - sum_{k=1..n} C(n,k) tau_k B^(n-k), with tau_k from
// q_k = s^(k)/s as in pair_terms.  Odd under i <-> j like the P <= 3 form
// (r^(k) changes sign, q_k and tau_k do not).  sink(n, c, B) receives component c of B^(n).
template <int P, typename T, typename Sink>
__device__ __forceinline__ void pair_general_terms(const T (&r)[P + 1][3], T sinv, Sink &&sink)
{
    T q[P + 1];
    s_ratios<P, T>(r, sinv, q);
    T tau[P + 1];
    tau[0] = T(1);
#pragma unroll
    for (int n = 1; n <= P; ++n) {
        T t = T(1.5) * q[n];
#pragma unroll
        for (int j = 1; j <= n - 1; ++j) {
            const T w = T(1.5 * binom(n - 1, j - 1) - binom(n - 1, j));
            t += w * q[j] * tau[n - j];
        }
        tau[n] = t;
    }
    T B[P + 1][3];
#pragma unroll
    for (int n = 0; n <= P; ++n) {
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            T b = r[n][c];
#pragma unroll
            for (int k = 1; k <= n; ++k) b -= (T(binom(n, k)) * tau[k]) * B[n - k][c];
            B[n][c] = b;
            sink(n, c, b);
        }
    }
}

// The odd terms of any supported P: the alpha/beta/gamma form up to P = 3, the
// general recursion above.
template <int P, typename T, typename Sink>
__device__ __forceinline__ void pair_odd_terms(const T (&r)[P + 1][3], T sinv, Sink &&sink)
{
    if constexpr (P <= 3)
        pair_abg_terms<P, T>(r, sinv, sink);
    else
        pair_general_terms<P, T>(r, sinv, sink);
}

// acc_k += (G m S) B_k for one ordered pair.
template <int P, typename T>
__device__ __forceinline__ void pair_abg(const T (&r)[P + 1][3], T mS, T sinv, T (&acc)[P + 1][3])
{
    pair_abg_terms<P, T>(r, sinv, [&](int k, int c, T B) { acc[k][c] += mS * B; });
}

// Pair derivatives for any supported P: the alpha/beta/gamma form up to P = 3,
// the general recursion above it.
template <int P, typename T>
__device__ __forceinline__ void pair_derivs(const T (&r)[P + 1][3], T mS, T sinv, T (&acc)[P + 1][3])
{
    if constexpr (P <= 3) {
        pair_abg<P, T>(r, mS, sinv, acc);
    } else {
        T q[P + 1];
        s_ratios<P, T>(r, sinv, q);
        pair_terms<P, T>(r, mS, q, acc);
    }
}

// Single-precision 1/sqrt(x) of the special-function unit (one instruction;
// x below 2^-126 is flushed to zero).
__device__ __forceinline__ float rsqrt_mufu(float x)
{
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// 1/sqrt(s) in FP64: an FP32 estimate, then one third-order Householder step
// y <- y (1 + e/2 + 3e^2/8), e = 1 - s y^2 (error ~ e0^3, e0 ~ 2^-22).
// The estimate is taken of m in s = 4^k m, m in [1, 4), and scaled by 2^-k, so
// that every positive normal double is in range.  m crosses to single precision
// and the estimate back to double by integer operations on the bit patterns
// (exponent rebiased by 1023 - 127, mantissa truncated to 23 bits going in,
// exact coming back), which keeps both conversions off the FP64 pipe.
// s = 0 (or subnormal) gives +inf, which turns the pair into NaN as the
// softening-free singularity should; an infinite or NaN s gives a non-finite result.
__device__ __forceinline__ double rsqrt_fp64(double s)
{
    constexpr int kRebias = (1023 - 127) << 20;          // exponent shift in the high word
    const long long b = __double_as_longlong(s);
    const int hi = (int)(b >> 32);
    const unsigned lo = (unsigned)b;
    const int de = (hi >> 20) & 0x7ff;                   // biased exponent of s
    const int k = (de - 1023) >> 1;                      // floor(exponent / 2)
    const int mhi = (hi & 0x000fffff) | ((de - 2 * k) << 20);   // m: exponent 1023 or 1024
    const int fb = ((mhi - kRebias) << 3) | (int)(lo >> 29);
    const int yb = __float_as_int(rsqrt_mufu(__int_as_float(fb)));   // 1/sqrt(m) in (0.5, 1]
    const int yhi = de == 0 ? 0x7ff00000 : (yb >> 3) + kRebias - (k << 20);
    const double y = __hiloint2double(yhi, de == 0 ? 0 : (yb & 7) << 29);
    const double e = fma(-s, y * y, 1.0);
    const double t = fma(0.375, e, 0.5);
    return fma(y * e, t, y);
}


}  // namespace mh
