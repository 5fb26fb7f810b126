// Rational constants of the modified Hermite corrector and end-of-step
// interpolation (the values of hermite_consts.cuh, same meaning: kv(k),
// kx(beta_mode, k), e1(n, k), e0(n, k) with n = p+1 .. 2p-1) as exact
// numerator / denominator pairs, p = 1 .. 5, for the double-double form.
// Written by `python derive_constants.py --dd-header`.
#pragma once

namespace mh {
namespace ddc {

struct Ratio { long long num, den; };

// p = 1 (order 4)
__host__ __device__ constexpr Ratio kv1(int k)
{ constexpr Ratio t[2] = {{1, 2}, {-1, 12}}; return t[k]; }
__host__ __device__ constexpr Ratio kx1(int b, int k)
{ constexpr Ratio t[2][3] = {{{1, 2}, {-7, 60}, {1, 60}}, {{1, 2}, {-1, 10}, {1, 120}}}; return t[b][k]; }

// p = 2 (order 6)
__host__ __device__ constexpr Ratio kv2(int k)
{ constexpr Ratio t[3] = {{1, 2}, {-1, 10}, {1, 120}}; return t[k]; }
__host__ __device__ constexpr Ratio kx2(int b, int k)
{ constexpr Ratio t[2][4] = {{{1, 2}, {-4, 35}, {13, 840}, {-1, 840}}, {{1, 2}, {-3, 28}, {1, 84}, {-1, 1680}}}; return t[b][k]; }
__host__ __device__ constexpr Ratio e1_2(int n, int k)
{ constexpr Ratio t[1][3] = {{{60, 1}, {-36, 1}, {9, 1}}}; return t[n - 3][k]; }
__host__ __device__ constexpr Ratio e0_2(int n, int k)
{ constexpr Ratio t[1][3] = {{{-60, 1}, {-24, 1}, {-3, 1}}}; return t[n - 3][k]; }

// p = 3 (order 8)
__host__ __device__ constexpr Ratio kv3(int k)
{ constexpr Ratio t[4] = {{1, 2}, {-3, 28}, {1, 84}, {-1, 1680}}; return t[k]; }
__host__ __device__ constexpr Ratio kx3(int b, int k)
{ constexpr Ratio t[2][5] = {{{1, 2}, {-29, 252}, {1, 63}, {-1, 720}, {1, 15120}}, {{1, 2}, {-1, 9}, {1, 72}, {-1, 1008}, {1, 30240}}}; return t[b][k]; }
__host__ __device__ constexpr Ratio e1_3(int n, int k)
{ constexpr Ratio t[2][4] = {{{-840, 1}, {480, 1}, {-120, 1}, {16, 1}}, {{-10080, 1}, {5400, 1}, {-1200, 1}, {120, 1}}}; return t[n - 4][k]; }
__host__ __device__ constexpr Ratio e0_3(int n, int k)
{ constexpr Ratio t[2][4] = {{{840, 1}, {360, 1}, {60, 1}, {4, 1}}, {{10080, 1}, {4680, 1}, {840, 1}, {60, 1}}}; return t[n - 4][k]; }

// p = 4 (order 10)
__host__ __device__ constexpr Ratio kv4(int k)
{ constexpr Ratio t[5] = {{1, 2}, {-1, 9}, {1, 72}, {-1, 1008}, {1, 30240}}; return t[k]; }
__host__ __device__ constexpr Ratio kx4(int b, int k)
{ constexpr Ratio t[2][6] = {{{1, 2}, {-23, 198}, {13, 792}, {-17, 11088}, {31, 332640}, {-1, 332640}}, {{1, 2}, {-5, 44}, {1, 66}, {-1, 792}, {1, 15840}, {-1, 665280}}}; return t[b][k]; }
__host__ __device__ constexpr Ratio e1_4(int n, int k)
{ constexpr Ratio t[3][5] = {{{15120, 1}, {-8400, 1}, {2100, 1}, {-300, 1}, {25, 1}}, {{302400, 1}, {-161280, 1}, {37800, 1}, {-4800, 1}, {300, 1}}, {{2721600, 1}, {-1411200, 1}, {317520, 1}, {-37800, 1}, {2100, 1}}}; return t[n - 5][k]; }
__host__ __device__ constexpr Ratio e0_4(int n, int k)
{ constexpr Ratio t[3][5] = {{{-15120, 1}, {-6720, 1}, {-1260, 1}, {-120, 1}, {-5, 1}}, {{-302400, 1}, {-141120, 1}, {-27720, 1}, {-2760, 1}, {-120, 1}}, {{-2721600, 1}, {-1310400, 1}, {-267120, 1}, {-27720, 1}, {-1260, 1}}}; return t[n - 5][k]; }

// p = 5 (order 12)
__host__ __device__ constexpr Ratio kv5(int k)
{ constexpr Ratio t[6] = {{1, 2}, {-5, 44}, {1, 66}, {-1, 792}, {1, 15840}, {-1, 665280}}; return t[k]; }
__host__ __device__ constexpr Ratio kx5(int b, int k)
{ constexpr Ratio t[2][7] = {{{1, 2}, {-67, 572}, {29, 1716}, {-17, 10296}, {23, 205920}, {-43, 8648640}, {1, 8648640}}, {{1, 2}, {-3, 26}, {5, 312}, {-5, 3432}, {1, 11440}, {-1, 308880}, {1, 17297280}}}; return t[b][k]; }
__host__ __device__ constexpr Ratio e1_5(int n, int k)
{ constexpr Ratio t[4][6] = {{{-332640, 1}, {181440, 1}, {-45360, 1}, {6720, 1}, {-630, 1}, {36, 1}}, {{-9979200, 1}, {5292000, 1}, {-1270080, 1}, {176400, 1}, {-14700, 1}, {630, 1}}, {{-139708800, 1}, {72576000, 1}, {-16934400, 1}, {2257920, 1}, {-176400, 1}, {6720, 1}}, {{-1117670400, 1}, {571536000, 1}, {-130636800, 1}, {16934400, 1}, {-1270080, 1}, {45360, 1}}}; return t[n - 6][k]; }
__host__ __device__ constexpr Ratio e0_5(int n, int k)
{ constexpr Ratio t[4][6] = {{{332640, 1}, {151200, 1}, {30240, 1}, {3360, 1}, {210, 1}, {6, 1}}, {{9979200, 1}, {4687200, 1}, {967680, 1}, {110880, 1}, {7140, 1}, {210, 1}}, {{139708800, 1}, {67132800, 1}, {14212800, 1}, {1673280, 1}, {110880, 1}, {3360, 1}}, {{1117670400, 1}, {546134400, 1}, {117936000, 1}, {14212800, 1}, {967680, 1}, {30240, 1}}}; return t[n - 6][k]; }

}  // namespace ddc
}  // namespace mh
