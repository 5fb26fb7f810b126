// Double-double ("double-word") arithmetic for the extended-precision form.
//
// A value is the unevaluated sum hi + lo of two doubles with |lo| <= ulp(hi)/2,
// 106 significant bits.  The building blocks are the error-free transformations
//   two_sum      a + b = s + t exactly (Knuth, TAOCP vol. 2; Moller 1965),
//   fast_two_sum the same when |a| >= |b| (Dekker 1971),
//   two_prod     a b = p + e exactly, e = fma(a, b, -p),
// and on top of them the double-word algorithms analysed by Joldes, Muller and
// Popescu, "Tight and rigorous error bounds for basic building blocks of
// double-word arithmetic", ACM TOMS 44(2), 2017: the accurate sum of two
// double-words, the double-word x double product, and the double-word x
// double-word product with FMA.  Each has a relative error of a small multiple
// of u^2, u = 2^-53, i.e. ~1e-32.
//
// Every floating-point operation goes through a round-to-nearest intrinsic, so
// the compiler can neither contract a product into a following addition nor
// reorder the error terms.
#pragma once

#include <cuda_runtime.h>

namespace mh {

struct dd {
    double hi, lo;
    dd() = default;
    __host__ __device__ constexpr dd(double h) : hi(h), lo(0.0) {}
    __host__ __device__ constexpr dd(double h, double l) : hi(h), lo(l) {}
};

__device__ __forceinline__ dd two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    const double bv = __dsub_rn(s, a);
    const double av = __dsub_rn(s, bv);
    return dd(s, __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv)));
}

__device__ __forceinline__ dd fast_two_sum(double a, double b)
{
    const double s = __dadd_rn(a, b);
    return dd(s, __dsub_rn(b, __dsub_rn(s, a)));
}

__device__ __forceinline__ dd two_prod(double a, double b)
{
    const double p = __dmul_rn(a, b);
    return dd(p, __fma_rn(a, b, -p));
}

// accurate double-word + double-word
__device__ __forceinline__ dd operator+(dd x, dd y)
{
    const dd s = two_sum(x.hi, y.hi);
    const dd t = two_sum(x.lo, y.lo);
    const dd v = fast_two_sum(s.hi, __dadd_rn(s.lo, t.hi));
    return fast_two_sum(v.hi, __dadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ dd operator-(dd x) { return dd(-x.hi, -x.lo); }
__device__ __forceinline__ dd operator-(dd x, dd y) { return x + (-y); }

// double-word + double
__device__ __forceinline__ dd add_d(dd x, double y)
{
    const dd s = two_sum(x.hi, y);
    return fast_two_sum(s.hi, __dadd_rn(x.lo, s.lo));
}

// double-word x double-word (FMA form)
__device__ __forceinline__ dd operator*(dd x, dd y)
{
    const dd c = two_prod(x.hi, y.hi);
    const double t = __fma_rn(x.hi, y.lo, __dmul_rn(x.lo, y.lo));
    return fast_two_sum(c.hi, __dadd_rn(c.lo, __fma_rn(x.lo, y.hi, t)));
}

// double-word x double
__device__ __forceinline__ dd mul_d(dd x, double y)
{
    const dd c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, __fma_rn(x.lo, y, c.lo));
}

// double-word x double without the closing renormalisation: hi = RN(x.hi y)
// and lo = its exact error plus x.lo y, |lo| up to ~ulp(hi).  For a product that
// goes straight into a double-word sum, which renormalises its result anyway.
__device__ __forceinline__ dd mul_d_raw(dd x, double y)
{
    const double p = __dmul_rn(x.hi, y);
    return dd(p, __fma_rn(x.lo, y, __fma_rn(x.hi, y, -p)));
}

// The sloppy sum of two double-words (Dekker 1971; Joldes, Muller and Popescu
// 2017, the SloppyDWPlusDW algorithm): one two_sum of the high words, the low
// words added in double.  Its error is at most ~2u^2 (|x| + |y|) (no relative
// bound when x and y cancel), the same order as the rounding the summed
// terms already carry, so it serves long sums of pair terms; 11 FP64
// operations against 20 for the accurate sum.
__device__ __forceinline__ dd add_sloppy(dd x, dd y)
{
    const dd s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __dadd_rn(s.lo, __dadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ dd &operator+=(dd &x, dd y) { return x = x + y; }
__device__ __forceinline__ dd &operator-=(dd &x, dd y) { return x = x - y; }

// num / den to double-double, num and den integers of magnitude below 2^53:
// q = RN(num/den) leaves the remainder num - q den exactly representable
// (computed exactly by one fma), and the remainder over den is the low word.
__device__ __forceinline__ dd dd_ratio(long long num, long long den)
{
    const double n = (double)num, d = (double)den;
    const double q = __ddiv_rn(n, d);
    return fast_two_sum(q, __ddiv_rn(__fma_rn(-q, d, n), d));
}

// 1/a for a double a, by the same remainder argument
__device__ __forceinline__ dd dd_recip(double a)
{
    const double q = __drcp_rn(a);
    return fast_two_sum(q, __ddiv_rn(__fma_rn(-q, a, 1.0), a));
}

// 1/sqrt(s): y = rsqrt(s.hi) in double (within an ulp of 1/sqrt(s)), then one
// Newton step y (1 + e/2) with the residual e = 1 - s y^2 formed in double-double.
// For y = (1 + d)/sqrt(s) the step leaves a relative error of 1.5 d^2 + O(d^3),
// ~2^-104 for |d| <= 2^-52.  s <= 0 or non-finite gives a non-finite result.
__device__ __forceinline__ dd rsqrt_dd(dd s)
{
    const double y = rsqrt(s.hi);
    const dd w = s * two_prod(y, y);                       // ~1
    const double e = __dsub_rn(__dsub_rn(1.0, w.hi), w.lo);   // 1 - w.hi is exact near 1
    return fast_two_sum(y, __dmul_rn(__dmul_rn(y, e), 0.5));
}

__device__ __forceinline__ bool dd_isfinite(dd x) { return isfinite(x.hi) && isfinite(x.lo); }

}  // namespace mh
