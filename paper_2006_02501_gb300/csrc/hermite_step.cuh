// Per-body pieces of one modified Hermite step (Dittmann 2020, Section 2),
// shared by the per-system kernels (integrator.cu) and the batched
// integrator (batch.cu).
#pragma once

#include "hermite_consts.cuh"

namespace mh {

// Taylor predictor of one component (Section 3 intro): x, v and the
// a-derivatives a^(q), q = 0..p-2, at t0 + dt from x0, v0, d = a^(0..2p-1).
template <int p>
__device__ __forceinline__ void predict_comp(double dt, const double (&d)[2 * p], double x0, double v0,
                                             double &x, double &v, double (&ad)[p > 1 ? p - 1 : 1])
{
    constexpr int K = 2 * p;
    double sx = 0.0, sv = 0.0;
#pragma unroll
    for (int k = K - 1; k >= 0; --k) {
        sx = fma(sx, dt, d[k] * inv_fact(k + 2));
        sv = fma(sv, dt, d[k] * inv_fact(k + 1));
    }
    x = fma(fma(sx, dt, v0), dt, x0);
    v = fma(sv, dt, v0);
#pragma unroll
    for (int q = 0; q + 2 <= p; ++q) {
        double sa = 0.0;
#pragma unroll
        for (int k = K - 1; k >= q; --k) sa = fma(sa, dt, d[k] * inv_fact(k - q));
        ad[q] = sa;
    }
}

// Corrector of one component (velocity, Eq. 6, then position with the new
// velocity, Eq. 7): d0 = a^(0..2p-1) at t0, d1 = a^(0..p) at t1.
template <int p>
__device__ __forceinline__ void correct_comp(double dt, int bm, const double (&d0)[2 * p],
                                             const double (&d1)[p + 1], double x0, double v0,
                                             double &xn, double &vn)
{
    // velocity (Eq. 6): sum_k kv(k) (a1^(k) + (-1)^k a0^(k)) dt^(k+1)
    double sv = 0.0;
#pragma unroll
    for (int k = p; k >= 0; --k) {
        const double f = (k & 1) ? d1[k] - d0[k] : d1[k] + d0[k];
        sv = fma(sv, dt, kv<p>(k) * f);
    }
    vn = fma(sv, dt, v0);
    // position (Eq. 7): kx(0) (v1 + v0) dt + sum_{k>=1} kx(k) (a1^(k-1) +- a0^(k-1)) dt^(k+1)
    double sx = 0.0;
#pragma unroll
    for (int k = p + 1; k >= 1; --k) {
        const double f = (k & 1) ? d1[k - 1] - d0[k - 1] : d1[k - 1] + d0[k - 1];
        sx = fma(sx, dt, (bm == 0 ? kx<p>(0, k) : kx<p>(1, k)) * f);
    }
    sx = fma(sx, dt, (bm == 0 ? kx<p>(0, 0) : kx<p>(1, 0)) * (vn + v0));
    xn = fma(sx, dt, x0);
}

// The corrector with compensated summation of the two updates (Section 3.2,
// after Kahan): cx, cv carry the parts of x, v lost to rounding in earlier
// steps (negated, Kahan's c) and return the new ones.  The increment minus the
// compensation is formed by one fused multiply-add.
template <int p>
__device__ __forceinline__ void correct_comp_kahan(double dt, int bm, const double (&d0)[2 * p],
                                                   const double (&d1)[p + 1], double x0, double v0,
                                                   double &cx, double &cv, double &xn, double &vn)
{
    double sv = 0.0;
#pragma unroll
    for (int k = p; k >= 0; --k) {
        const double f = (k & 1) ? d1[k] - d0[k] : d1[k] + d0[k];
        sv = fma(sv, dt, kv<p>(k) * f);
    }
    const double yv = fma(sv, dt, -cv);
    vn = v0 + yv;
    cv = (vn - v0) - yv;
    double sx = 0.0;
#pragma unroll
    for (int k = p + 1; k >= 1; --k) {
        const double f = (k & 1) ? d1[k - 1] - d0[k - 1] : d1[k - 1] + d0[k - 1];
        sx = fma(sx, dt, (bm == 0 ? kx<p>(0, k) : kx<p>(1, k)) * f);
    }
    sx = fma(sx, dt, (bm == 0 ? kx<p>(0, 0) : kx<p>(1, 0)) * (vn + v0));
    const double yx = fma(sx, dt, -cx);
    xn = x0 + yx;
    cx = (xn - x0) - yx;
}

// a^(p+1..2p-1)(t1) of one component from the degree-(2p+1) Hermite interpolant:
// a^(n)(t1) = sum_k (e1(n,k) a1^(k) + e0(n,k) a0^(k)) dt^(k-n).
template <int p>
__device__ __forceinline__ void interp_comp(double dt, const double (&d0)[2 * p],
                                            const double (&d1)[p + 1],
                                            double (&hi)[2 * p > p + 1 ? p - 1 : 1])
{
    if constexpr (p >= 2) {
        const double rdt = 1.0 / dt;
#pragma unroll
        for (int n = p + 1; n < 2 * p; ++n) {
            double s = 0.0;
#pragma unroll
            for (int k = p; k >= 0; --k) s = fma(s, dt, fma(e1<p>(n, k), d1[k], e0<p>(n, k) * d0[k]));
            double sc = 1.0;
#pragma unroll
            for (int e = 0; e < n; ++e) sc *= rdt;
            hi[n - p - 1] = s * sc;
        }
    }
}

}  // namespace mh
