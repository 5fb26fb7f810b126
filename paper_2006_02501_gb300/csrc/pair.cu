// O(N^2) direct-summation evaluation of a^(0..P) (the E of P(EC)^n), every
// ordered pair: the kernels for active lists (block steps), small systems,
// the initialisation passes above P = 3, and mh_pair_eval.  Shared-step
// evaluations of larger systems take the pair-symmetric kernels of
// pair_sym.cu instead.
//
// Pair physics (Dittmann 2020, Section 3, intro): a_ij = G m_j r_ij s^(-3/2),
// s = r_ij^2 + eps^2.  Its time derivatives along the trajectory follow from
// T a = G m r with T = s^(3/2): differentiating n times,
//   A^(n) = G m S r^(n) - sum_{k=1..n} C(n,k) tau_k A^(n-k),   S = s^(-3/2),
//   tau_k = T^(k)/T,  tau_n = 1.5 q_n + sum_{j=1..n-1} (1.5 C(n-1,j-1) - C(n-1,j)) q_j tau_(n-j),
//   q_k = s^(k)/s,    s^(k) = sum_j C(k,j) r^(j).r^(k-j)   (eps enters s^(0) only).
// For P = 3 this is the familiar alpha/beta/gamma form: tau_1 = 3 alpha,
// tau_2 = 3 beta, tau_3 = 3 gamma.
//
// Decomposition: items = (i-tile of `threads` bodies, one or two per thread) x
// (j-chunk); a CTA loops over items with a grid stride; j-records of a chunk
// are staged through shared memory in tiles of `tj` (FP64 evaluations too small
// to fill the GPU use one-warp CTAs and tiles as short as 2: plan_fine64).  Each item writes its own
// partial-sum slot; the corrector (or mh_pair_eval's reduction) adds the
// slots in a fixed order, so the result is deterministic.
//
// Two arithmetic forms:
//   FP64:     every operation in double precision; 1/sqrt(s) from the FP32
//             MUFU estimate refined by one third-order Householder step.
//   FP32PAIR: the pair arithmetic in FP32.  Differences of x and v are taken
//             from a hi/lo split of the FP64 values, (hi_j - hi_i) + (lo_j - lo_i),
//             which is the FP64 difference rounded to FP32 within about one ulp;
//             sums run in FP32 over one shared-memory tile and are added to
//             FP64 accumulators after every tile.
#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "hermite_consts.cuh"
#include "pair_math.cuh"

namespace mh {

namespace {

// ---------------------------------------------------------------------------
// FP64 form
// ---------------------------------------------------------------------------

template <int P>
struct PairArgs64 {
    const double *jrec;   // [3(P+1)][ld]
    const double *m;      // [ld]
    int64_t ld;           // row stride of jrec / length of m
    int64_t n_j;          // bodies j in [0, n_j) (multiple of tj; padding has m = 0)
    int64_t i0, i1;
    double eps2, G;
    double *part;         // [S][(P+1)*3][part_ld], index i - i0
    int64_t part_ld;
    int64_t n_itiles, chunk;
    int split, tj;
    const int *ilist;     // optional: body index of position i (active list); else i itself
    unsigned long long *wmax;   // kH: max over pairs of G (m_i + m_j) s^(-3/2) (bit pattern), raised
};

// kH: also raise wm with w = G (m_i + m_j) s^(-3/2) of the pair (gmi = G m_i), whose
// maximum over pairs gives the time-step criterion of Section 3.3 (Eq. 24).
template <int P, bool kGuard, bool kH>
__device__ __forceinline__ void interact64(const double *sh, int tj, int jj, bool self,
                                           const double (&ri)[P + 1][3], const PairArgs64<P> &a,
                                           double (&acc)[P + 1][3], double gmi, unsigned long long &wm)
{
    constexpr int NF = 3 * (P + 1);
    double r[P + 1][3];
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) r[k][c] = sh[(3 * k + c) * tj + jj] - ri[k][c];
    double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], a.eps2)));
    double mj = sh[NF * tj + jj];
    if (kGuard) {
        s = self ? 1.0 : s;
        mj = self ? 0.0 : mj;
    }
    const double rinv = rsqrt_fp64(s);
    const double sinv = rinv * rinv;
    const double gmj = a.G * mj;
    const double mS = gmj * (rinv * sinv);
    if constexpr (kH) {
        const unsigned long long wb =
            (kGuard && self) ? 0ull : (unsigned long long)__double_as_longlong((gmi + gmj) * (rinv * sinv));
        wm = wb > wm ? wb : wm;
    }
    pair_derivs<P, double>(r, mS, sinv, acc);
}

template <int P, bool kH>
__global__ void __launch_bounds__(128) k_pair_fp64(PairArgs64<P> a)
{
    unsigned long long wm = 0ull;
    constexpr int NF = 3 * (P + 1);
    extern __shared__ double sh[];      // [NF + 1][tj]
    const int tj = a.tj;
    const int64_t items = a.n_itiles * a.split;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t itile = item % a.n_itiles;
        const int jc = (int)(item / a.n_itiles);
        const int64_t i = a.i0 + itile * blockDim.x + threadIdx.x;
        const bool live = i < a.i1;
        const int64_t ipos = live ? i : a.i0;
        const int64_t ic = a.ilist ? (int64_t)a.ilist[ipos] : ipos;
        double ri[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) ri[k][c] = a.jrec[(3 * k + c) * a.ld + ic];
        const double gmi = kH ? a.G * a.m[ic] : 0.0;
        unsigned long long wm_item = 0ull;   // this item's pairs; kept only for a live position
        double acc[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[k][c] = 0.0;

        const int64_t jb = (int64_t)jc * a.chunk;
        const int64_t je = min(jb + a.chunk, a.n_j);
        for (int64_t j0 = jb; j0 < je; j0 += tj) {
            __syncthreads();
            for (int e = threadIdx.x; e < (NF + 1) * tj; e += blockDim.x) {
                const int row = e / tj, col = e - row * tj;
                const int64_t j = j0 + col;
                // bodies past n_j: massless and far away, so they add exactly zero
                sh[e] = j < a.n_j ? (row < NF ? a.jrec[row * a.ld + j] : a.m[j])
                                  : (row < 3 ? kFarAway : 0.0);
            }
            __syncthreads();
            // the i == j pair can only occur when this tile overlaps the CTA's i-range
            // (with an index list any tile may hold it)
            const int64_t ib = a.i0 + itile * blockDim.x;
            if (a.ilist || (j0 < ib + (int64_t)blockDim.x && ib < j0 + tj)) {
                for (int jj = 0; jj < tj; ++jj)
                    interact64<P, true, kH>(sh, tj, jj, j0 + jj == ic, ri, a, acc, gmi, wm_item);
            } else {
                for (int jj = 0; jj < tj; ++jj)
                    interact64<P, false, kH>(sh, tj, jj, false, ri, a, acc, gmi, wm_item);
            }
        }
        // an idle position evaluates body i0 with the guard of its own tile only, so its
        // pairs (possibly i0 with itself) must not enter the maximum
        if (kH && live) wm = wm_item > wm ? wm_item : wm;
        if (live) {
            double *out = a.part + (int64_t)jc * (P + 1) * 3 * a.part_ld + (i - a.i0);
#pragma unroll
            for (int k = 0; k <= P; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) out[(3 * k + c) * a.part_ld] = acc[k][c];
        }
    }
    if constexpr (kH) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xffffffffu, wm, o);
            wm = q > wm ? q : wm;
        }
        if ((threadIdx.x & 31) == 0 && wm) atomicMax(a.wmax, wm);
    }
}

// ---------------------------------------------------------------------------
// FP32-pair form
// ---------------------------------------------------------------------------
// Input rows (jrec32, each of length ld):
//   0-2 x_hi, 3-5 x_lo, 6-8 v_hi, 9-11 v_lo, then a (P >= 2), a-dot (P >= 3), m.
// Shared-memory tile: one record of RS floats per j (x_hi, x_lo, v_hi, v_lo,
// a, a-dot, m, padding), read by every lane of a warp as broadcast float4s.

template <int P>
struct Rec32 {
    static constexpr int NF = nf32(P);                 // input rows
    static constexpr int RS = (NF + 3) / 4 * 4;        // floats per smem record
};

template <int P>
struct PairArgs32 {
    const float *jrec32;  // [NF][ld], the mass row holding G m
    int64_t ld, n_j, i0, i1;
    float eps2;
    double *part;
    int64_t part_ld, n_itiles, chunk;
    int split, tj;
    const int *ilist;     // optional: body index of position i (active list)
};

constexpr int kThreads32 = 256;

// One j-record (already in registers) against one i-body.
template <int P, bool kGuard>
__device__ __forceinline__ void interact32(const float *rec, bool self, const float (&xh)[3],
                                           const float (&xl)[3], const float (&vh)[3], const float (&vl)[3],
                                           const float (&ai)[3], const float (&ji)[3], float eps2,
                                           float (&acc)[P + 1][3])
{
    constexpr int NF = Rec32<P>::NF;
    float r[P + 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r[0][c] = (rec[c] - xh[c]) + (rec[3 + c] - xl[c]);
        r[1][c] = (rec[6 + c] - vh[c]) + (rec[9 + c] - vl[c]);
        if constexpr (P >= 2) r[2][c] = rec[12 + c] - ai[c];
        if constexpr (P >= 3) r[3][c] = rec[15 + c] - ji[c];
    }
    float s = fmaf(r[0][0], r[0][0], fmaf(r[0][1], r[0][1], fmaf(r[0][2], r[0][2], eps2)));
    float gm = rec[NF - 1];
    if (kGuard) {
        s = self ? 1.0f : s;
        gm = self ? 0.0f : gm;
    }
    const float rinv = rsqrt_mufu(s);
    const float sinv = rinv * rinv;
    const float mS = gm * rinv * sinv;
    pair_abg<P, float>(r, mS, sinv, acc);
}

template <int P>
__device__ __forceinline__ void load_rec(const float4 *sh4, int jj, float (&rec)[Rec32<P>::RS])
{
    constexpr int RS = Rec32<P>::RS;
#pragma unroll
    for (int q4 = 0; q4 < RS / 4; ++q4) {
        const float4 t = sh4[jj * (RS / 4) + q4];
        rec[4 * q4 + 0] = t.x; rec[4 * q4 + 1] = t.y;
        rec[4 * q4 + 2] = t.z; rec[4 * q4 + 3] = t.w;
    }
}

// IPT i-bodies per thread (thread t of the CTA owns positions ib + t + k kThreads32).
template <int P, int IPT>
__global__ void __launch_bounds__(kThreads32, 2) k_pair_fp32(PairArgs32<P> a)
{
    constexpr int NF = Rec32<P>::NF;
    constexpr int RS = Rec32<P>::RS;
    constexpr int NR = (P + 1) * 3;
    extern __shared__ float4 sh4[];                   // [tj][RS/4] records, then FP64 accumulators
    float *sh = reinterpret_cast<float *>(sh4);
    const int tj = a.tj;
    // per-position FP64 accumulators across tiles: [NR][IPT * kThreads32]
    double *acc64 = reinterpret_cast<double *>(sh + (size_t)tj * RS);
    constexpr int W = IPT * kThreads32;
    const int64_t items = a.n_itiles * a.split;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t itile = item % a.n_itiles;
        const int jc = (int)(item / a.n_itiles);
        const int64_t ib = a.i0 + itile * W;
        float xh[IPT][3], xl[IPT][3], vh[IPT][3], vl[IPT][3], ai[IPT][3], ji[IPT][3];
        int64_t ic[IPT];
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int64_t i = ib + threadIdx.x + k * kThreads32;
            const int64_t ipos = i < a.i1 ? i : a.i0;
            ic[k] = a.ilist ? (int64_t)a.ilist[ipos] : ipos;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xh[k][c] = a.jrec32[(0 + c) * a.ld + ic[k]];
                xl[k][c] = a.jrec32[(3 + c) * a.ld + ic[k]];
                vh[k][c] = a.jrec32[(6 + c) * a.ld + ic[k]];
                vl[k][c] = a.jrec32[(9 + c) * a.ld + ic[k]];
                ai[k][c] = P >= 2 ? a.jrec32[(12 + c) * a.ld + ic[k]] : 0.0f;
                ji[k][c] = P >= 3 ? a.jrec32[(15 + c) * a.ld + ic[k]] : 0.0f;
            }
#pragma unroll
            for (int q = 0; q < NR; ++q) acc64[q * W + threadIdx.x + k * kThreads32] = 0.0;
        }

        const int64_t jb = (int64_t)jc * a.chunk;
        const int64_t je = min(jb + a.chunk, a.n_j);
        for (int64_t j0 = jb; j0 < je; j0 += tj) {
            __syncthreads();
            for (int e = threadIdx.x; e < NF * tj; e += kThreads32) {
                const int row = e / tj, col = e - row * tj;
                const int64_t j = j0 + col;
                sh[col * RS + row] = j < a.n_j ? a.jrec32[row * a.ld + j] : (row < 3 ? (float)kFarAway : 0.0f);
            }
            __syncthreads();
            float acc[IPT][P + 1][3];
#pragma unroll
            for (int k = 0; k < IPT; ++k)
#pragma unroll
                for (int n = 0; n <= P; ++n)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[k][n][c] = 0.0f;
            if (a.ilist || (j0 < ib + W && ib < j0 + tj)) {
                // the tile may hold this thread's own bodies: guard the i == j pairs
#pragma unroll 2
                for (int jj = 0; jj < tj; ++jj) {
                    float rec[RS];
                    load_rec<P>(sh4, jj, rec);
#pragma unroll
                    for (int k = 0; k < IPT; ++k)
                        interact32<P, true>(rec, j0 + jj == ic[k], xh[k], xl[k], vh[k], vl[k], ai[k], ji[k],
                                            a.eps2, acc[k]);
                }
            } else {
#pragma unroll 2
                for (int jj = 0; jj < tj; ++jj) {
                    float rec[RS];
                    load_rec<P>(sh4, jj, rec);
#pragma unroll
                    for (int k = 0; k < IPT; ++k)
                        interact32<P, false>(rec, false, xh[k], xl[k], vh[k], vl[k], ai[k], ji[k], a.eps2, acc[k]);
                }
            }
#pragma unroll
            for (int k = 0; k < IPT; ++k)
#pragma unroll
                for (int n = 0; n <= P; ++n)
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        acc64[(3 * n + c) * W + threadIdx.x + k * kThreads32] += (double)acc[k][n][c];
        }
#pragma unroll
        for (int k = 0; k < IPT; ++k) {
            const int64_t i = ib + threadIdx.x + k * kThreads32;
            if (i < a.i1) {
                double *out = a.part + (int64_t)jc * NR * a.part_ld + (i - a.i0);
#pragma unroll
                for (int q = 0; q < NR; ++q) out[q * a.part_ld] = acc64[q * W + threadIdx.x + k * kThreads32];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP32-pair form, packed: two i-bodies per thread in the two lanes of
// Blackwell's paired FP32 instructions (FFMA2/FMUL2/FADD2), so that one issue
// slot advances both pairs.  Same arithmetic as interact32 per lane, with the
// multiply-adds written out explicitly; results differ from the scalar kernels
// only by the rounding of those contractions.  The shared-memory tile stores
// every j value twice ({v, v}), so a 16-byte load yields two packed operands.
// ---------------------------------------------------------------------------

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// B_k of pair_abg_terms for two pairs at once; acc_k += mS B_k.
template <int P>
__device__ __forceinline__ void pair_abg_x2(const float2 (&r)[P + 1][3], float2 mS, float2 sinv,
                                            float2 (&acc)[P + 1][3])
{
    const float2 rv = fma2(r[0][2], r[1][2], fma2(r[0][1], r[1][1], mul2(r[0][0], r[1][0])));
    const float2 al = mul2(rv, sinv);
    const float2 na3 = mul2(f2(-3.0f), al);
    float2 B1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        B1[c] = fma2(na3, r[0][c], r[1][c]);
        acc[0][c] = fma2(mS, r[0][c], acc[0][c]);
        acc[1][c] = fma2(mS, B1[c], acc[1][c]);
    }
    if constexpr (P >= 2) {
        const float2 al2 = mul2(al, al);
        float2 w2 = mul2(r[1][0], r[1][0]);
        w2 = fma2(r[1][1], r[1][1], w2);
        w2 = fma2(r[1][2], r[1][2], w2);
        w2 = fma2(r[0][0], r[2][0], w2);
        w2 = fma2(r[0][1], r[2][1], w2);
        w2 = fma2(r[0][2], r[2][2], w2);
        const float2 be = fma2(w2, sinv, al2);
        const float2 na6 = mul2(f2(-6.0f), al), nb3 = mul2(f2(-3.0f), be);
        float2 B2[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            B2[c] = fma2(nb3, r[0][c], fma2(na6, B1[c], r[2][c]));
            acc[2][c] = fma2(mS, B2[c], acc[2][c]);
        }
        if constexpr (P >= 3) {
            const float2 va = fma2(r[1][2], r[2][2], fma2(r[1][1], r[2][1], mul2(r[1][0], r[2][0])));
            const float2 rj = fma2(r[0][2], r[3][2], fma2(r[0][1], r[3][1], mul2(r[0][0], r[3][0])));
            const float2 w3 = fma2(f2(3.0f), va, rj);
            // gamma = w3/s + alpha (3 beta - 4 alpha^2), with 3 beta - 4 alpha^2 = -(nb3 + 4 alpha^2)
            const float2 u = fma2(f2(4.0f), al2, nb3);
            const float2 ga = fma2(w3, sinv, mul2(mul2(f2(-1.0f), al), u));
            const float2 na9 = mul2(f2(-9.0f), al), nb9 = mul2(f2(-9.0f), be), ng3 = mul2(f2(-3.0f), ga);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float2 B3 = fma2(ng3, r[0][c], fma2(nb9, B1[c], fma2(na9, B2[c], r[3][c])));
                acc[3][c] = fma2(mS, B3, acc[3][c]);
            }
        }
    }
}

// One j-record (packed duplicates in shared memory) against this thread's two
// i-bodies, whose x, v hi/lo and a, a-dot are held negated (ni*).
template <int P, bool kGuard>
__device__ __forceinline__ void interact32x2(const float2 *rec, bool self0, bool self1,
                                             const float2 (&nxh)[3], const float2 (&nxl)[3],
                                             const float2 (&nvh)[3], const float2 (&nvl)[3],
                                             const float2 (&nai)[3], const float2 (&nji)[3], float2 eps2,
                                             float2 (&acc)[P + 1][3])
{
    constexpr int NF = Rec32<P>::NF;
    float2 r[P + 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r[0][c] = add2(add2(rec[c], nxh[c]), add2(rec[3 + c], nxl[c]));
        r[1][c] = add2(add2(rec[6 + c], nvh[c]), add2(rec[9 + c], nvl[c]));
        if constexpr (P >= 2) r[2][c] = add2(rec[12 + c], nai[c]);
        if constexpr (P >= 3) r[3][c] = add2(rec[15 + c], nji[c]);
    }
    float2 s = fma2(r[0][0], r[0][0], fma2(r[0][1], r[0][1], fma2(r[0][2], r[0][2], eps2)));
    float2 gm = rec[NF - 1];
    if (kGuard) {
        s.x = self0 ? 1.0f : s.x;
        s.y = self1 ? 1.0f : s.y;
        gm.x = self0 ? 0.0f : gm.x;
        gm.y = self1 ? 0.0f : gm.y;
    }
    const float2 rinv = make_float2(rsqrt_mufu(s.x), rsqrt_mufu(s.y));
    const float2 sinv = mul2(rinv, rinv);
    const float2 mS = mul2(mul2(gm, rinv), sinv);
    pair_abg_x2<P>(r, mS, sinv, acc);
}

// Thread t of the CTA owns positions ib + t and ib + t + kThreads32 (the layout
// of k_pair_fp32<P, 2>, so both write the same partial-sum slots).
template <int P>
__global__ void __launch_bounds__(kThreads32, 2) k_pair_fp32x2(PairArgs32<P> a)
{
    constexpr int NF = Rec32<P>::NF;
    constexpr int RS = Rec32<P>::RS;
    constexpr int NR = (P + 1) * 3;
    constexpr int W = 2 * kThreads32;
    extern __shared__ float4 sh4[];                   // [tj][RS] packed records, then FP64 accumulators
    float2 *sh2 = reinterpret_cast<float2 *>(sh4);
    const int tj = a.tj;
    double *acc64 = reinterpret_cast<double *>(sh2 + (size_t)tj * RS);   // [NR][W]
    const float2 eps2 = f2(a.eps2);
    const int64_t items = a.n_itiles * a.split;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int64_t itile = item % a.n_itiles;
        const int jc = (int)(item / a.n_itiles);
        const int64_t ib = a.i0 + itile * W;
        int64_t ic[2];
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int64_t i = ib + threadIdx.x + k * kThreads32;
            const int64_t ipos = i < a.i1 ? i : a.i0;
            ic[k] = a.ilist ? (int64_t)a.ilist[ipos] : ipos;
#pragma unroll
            for (int q = 0; q < NR; ++q) acc64[q * W + threadIdx.x + k * kThreads32] = 0.0;
        }
        auto ld2n = [&](int row) {
            return make_float2(-a.jrec32[row * a.ld + ic[0]], -a.jrec32[row * a.ld + ic[1]]);
        };
        float2 nxh[3], nxl[3], nvh[3], nvl[3], nai[3], nji[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            nxh[c] = ld2n(0 + c);
            nxl[c] = ld2n(3 + c);
            nvh[c] = ld2n(6 + c);
            nvl[c] = ld2n(9 + c);
            nai[c] = P >= 2 ? ld2n(12 + c) : f2(0.0f);
            nji[c] = P >= 3 ? ld2n(15 + c) : f2(0.0f);
        }

        const int64_t jb = (int64_t)jc * a.chunk;
        const int64_t je = min(jb + a.chunk, a.n_j);
        for (int64_t j0 = jb; j0 < je; j0 += tj) {
            __syncthreads();
            for (int e = threadIdx.x; e < NF * tj; e += kThreads32) {
                const int row = e / tj, col = e - row * tj;
                const int64_t j = j0 + col;
                sh2[col * RS + row] = f2(j < a.n_j ? a.jrec32[row * a.ld + j] : (row < 3 ? (float)kFarAway : 0.0f));
            }
            __syncthreads();
            float2 acc[P + 1][3];
#pragma unroll
            for (int n = 0; n <= P; ++n)
#pragma unroll
                for (int c = 0; c < 3; ++c) acc[n][c] = f2(0.0f);
            if (a.ilist || (j0 < ib + W && ib < j0 + tj)) {
#pragma unroll 2
                for (int jj = 0; jj < tj; ++jj)
                    interact32x2<P, true>(sh2 + jj * RS, j0 + jj == ic[0], j0 + jj == ic[1], nxh, nxl, nvh, nvl,
                                          nai, nji, eps2, acc);
            } else {
#pragma unroll 2
                for (int jj = 0; jj < tj; ++jj)
                    interact32x2<P, false>(sh2 + jj * RS, false, false, nxh, nxl, nvh, nvl, nai, nji, eps2, acc);
            }
#pragma unroll
            for (int n = 0; n <= P; ++n)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    acc64[(3 * n + c) * W + threadIdx.x] += (double)acc[n][c].x;
                    acc64[(3 * n + c) * W + threadIdx.x + kThreads32] += (double)acc[n][c].y;
                }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int64_t i = ib + threadIdx.x + k * kThreads32;
            if (i < a.i1) {
                double *out = a.part + (int64_t)jc * NR * a.part_ld + (i - a.i0);
#pragma unroll
                for (int q = 0; q < NR; ++q) out[q * a.part_ld] = acc64[q * W + threadIdx.x + k * kThreads32];
            }
        }
    }
}

// FP64 contributions of a short list of heavy source bodies (precision form):
// one thread per body i, the heavy records read through the read-only cache.
template <int P>
__global__ void k_pair_heavy(int64_t N, int64_t ld, const double *__restrict__ m,
                             const double *__restrict__ jrec, const int *__restrict__ heavy,
                             int n_heavy, double eps2, double G, double *__restrict__ out,
                             int64_t out_ld, const int *__restrict__ ilist)
{
    const int64_t pos = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (pos >= N) return;                       // N: number of positions (bodies or active list)
    const int64_t i = ilist ? (int64_t)ilist[pos] : pos;
    double ri[P + 1][3], acc[P + 1][3];
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            ri[k][c] = jrec[(3 * k + c) * ld + i];
            acc[k][c] = 0.0;
        }
    for (int h = 0; h < n_heavy; ++h) {
        const int j = __ldg(heavy + h);
        if (j == i) continue;
        double r[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[k][c] = __ldg(jrec + (3 * k + c) * ld + j) - ri[k][c];
        const double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], eps2)));
        const double rinv = rsqrt_fp64(s);
        const double sinv = rinv * rinv;
        const double mS = G * __ldg(m + j) * (rinv * sinv);
        pair_derivs<P, double>(r, mS, sinv, acc);
    }
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) out[(3 * k + c) * out_ld + pos] = acc[k][c];
}

template <int P>
int launch_fp64(const double *jrec, const double *m, int64_t ld, int64_t n_j, double eps,
                double G, int64_t i0, int64_t i1, double *part, int64_t part_ld,
                const PairPlan &pl, const int *ilist, cudaStream_t st, unsigned long long *wmax)
{
    PairArgs64<P> a{jrec, m, ld, n_j, i0, i1, eps * eps, G, part, part_ld,
                    pl.n_itiles, pl.chunk, pl.split, pl.tj, ilist, wmax};
    const size_t smem = sizeof(double) * (3 * (P + 1) + 1) * pl.tj;
    if (wmax)
        k_pair_fp64<P, true><<<pl.grid, pl.threads, smem, st>>>(a);
    else
        k_pair_fp64<P, false><<<pl.grid, pl.threads, smem, st>>>(a);
    MH_LAUNCHED("k_pair_fp64");
    return MH_OK;
}

template <int P, int IPT>
int launch_fp32_ipt(const PairArgs32<P> &a, const PairPlan &pl, cudaStream_t st)
{
    const size_t smem = sizeof(float) * Rec32<P>::RS * pl.tj + sizeof(double) * (P + 1) * 3 * IPT * kThreads32;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        MH_CUDA(cudaFuncSetAttribute(k_pair_fp32<P, IPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set[dev] = true;
    }
    k_pair_fp32<P, IPT><<<pl.grid, pl.threads, smem, st>>>(a);
    MH_LAUNCHED("k_pair_fp32");
    return MH_OK;
}

template <int P>
int launch_fp32_packed(const PairArgs32<P> &a, const PairPlan &pl, cudaStream_t st)
{
    const size_t smem = sizeof(float2) * Rec32<P>::RS * pl.tj + sizeof(double) * (P + 1) * 3 * 2 * kThreads32;
    static bool attr_set[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        MH_CUDA(cudaFuncSetAttribute(k_pair_fp32x2<P>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024));
        attr_set[dev] = true;
    }
    k_pair_fp32x2<P><<<pl.grid, pl.threads, smem, st>>>(a);
    MH_LAUNCHED("k_pair_fp32x2");
    return MH_OK;
}

template <int P>
int launch_fp32(const float *jrec32, int64_t ld, int64_t n_j, double eps, int64_t i0,
                int64_t i1, double *part, int64_t part_ld, const PairPlan &pl, const int *ilist,
                cudaStream_t st)
{
    PairArgs32<P> a{jrec32, ld, n_j, i0, i1, (float)(eps * eps), part, part_ld,
                    pl.n_itiles, pl.chunk, pl.split, pl.tj, ilist};
    if (pl.packed) return launch_fp32_packed<P>(a, pl, st);
    return pl.ipt == 2 ? launch_fp32_ipt<P, 2>(a, pl, st) : launch_fp32_ipt<P, 1>(a, pl, st);
}

}  // namespace

int launch_pair_heavy(int P, int64_t N, int64_t ld, const double *m, const double *jrec,
                      const int *heavy, int n_heavy, double eps, double G, double *part, int slot,
                      cudaStream_t st, const int *ilist, int64_t part_ld)
{
    const int64_t pld = part_ld > 0 ? part_ld : ld;
    double *out = part + (int64_t)slot * (P + 1) * 3 * pld;
    const unsigned g = (unsigned)((N + 127) / 128);
    const double e2 = eps * eps;
    switch (P) {
    case 1: k_pair_heavy<1><<<g, 128, 0, st>>>(N, ld, m, jrec, heavy, n_heavy, e2, G, out, pld, ilist); break;
    case 2: k_pair_heavy<2><<<g, 128, 0, st>>>(N, ld, m, jrec, heavy, n_heavy, e2, G, out, pld, ilist); break;
    case 3: k_pair_heavy<3><<<g, 128, 0, st>>>(N, ld, m, jrec, heavy, n_heavy, e2, G, out, pld, ilist); break;
    default: set_error("launch_pair_heavy: P must be 1..3"); return MH_EINVAL;
    }
    MH_LAUNCHED("k_pair_heavy");
    return MH_OK;
}

// ---------------------------------------------------------------------------
// Short active lists (block steps at which only a few bodies are due): one warp
// per (active body, j-chunk), the lanes over the chunk's sources in strides of
// 32, so that every lane evaluates useful pairs; the lanes' sums meet in a
// fixed shuffle tree (deterministic), and each (body, chunk) writes its own
// partial-sum slot.  FP32-pair: the precision form's pair arithmetic with FP32
// sums over at most 64 pairs per lane, added to FP64; the heavy bodies (mass 0
// in the FP32 rows) are added by k_pair_heavy.  FP64: the plain form.
// ---------------------------------------------------------------------------

template <int P>
struct ShortArgs {
    const double *jrec;   // FP64 rows [3(P+1)][ld] (FP64 form)
    const double *m;      // masses (FP64 form)
    const float *jrec32;  // FP32 rows [nf32(P)][ld] (precision form)
    int64_t ld, n_j, n_i;
    double eps2, G;
    double *part;         // [S][(P+1)*3][part_ld], by active position
    int64_t part_ld, chunk;
    int split;
    const int *ilist;     // active position -> body
};

template <int P, bool kF32>
__global__ void __launch_bounds__(128) k_pair_short(ShortArgs<P> a)
{
    constexpr int NR = (P + 1) * 3;
    const int lane = threadIdx.x & 31;
    const int64_t items = a.n_i * a.split;
    for (int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; item < items;
         item += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t pos = item % a.n_i;
        const int jc = (int)(item / a.n_i);
        const int64_t i = a.ilist[pos];
        const int64_t jb = (int64_t)jc * a.chunk;
        const int64_t je = min(jb + a.chunk, a.n_j);
        double acc64[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) acc64[k][c] = 0.0;
        if constexpr (kF32) {
            constexpr int NF = Rec32<P>::NF;
            float xh[3], xl[3], vh[3], vl[3], ai[3], ji[3];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                xh[c] = a.jrec32[(0 + c) * a.ld + i];
                xl[c] = a.jrec32[(3 + c) * a.ld + i];
                vh[c] = a.jrec32[(6 + c) * a.ld + i];
                vl[c] = a.jrec32[(9 + c) * a.ld + i];
                ai[c] = P >= 2 ? a.jrec32[(12 + c) * a.ld + i] : 0.0f;
                ji[c] = P >= 3 ? a.jrec32[(15 + c) * a.ld + i] : 0.0f;
            }
            const float eps2 = (float)a.eps2;
            for (int64_t j0 = jb; j0 < je; j0 += 64 * 32) {
                float acc[P + 1][3];
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc[k][c] = 0.0f;
                const int64_t j1 = min(j0 + 64 * 32, je);
                for (int64_t j = j0 + lane; j < j1; j += 32) {
                    float rec[NF];
#pragma unroll
                    for (int q = 0; q < NF; ++q) rec[q] = a.jrec32[q * a.ld + j];
                    interact32<P, true>(rec, j == i, xh, xl, vh, vl, ai, ji, eps2, acc);
                }
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) acc64[k][c] += (double)acc[k][c];
            }
        } else {
            double ri[P + 1][3];
#pragma unroll
            for (int k = 0; k <= P; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) ri[k][c] = a.jrec[(3 * k + c) * a.ld + i];
            for (int64_t j = jb + lane; j < je; j += 32) {
                double r[P + 1][3];
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) r[k][c] = a.jrec[(3 * k + c) * a.ld + j] - ri[k][c];
                double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], a.eps2)));
                const bool self = j == i;
                s = self ? 1.0 : s;
                const double rinv = rsqrt_fp64(s);
                const double sinv = rinv * rinv;
                const double mS = self ? 0.0 : a.G * a.m[j] * (rinv * sinv);
                pair_derivs<P, double>(r, mS, sinv, acc64);
            }
        }
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                double v = acc64[k][c];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
                acc64[k][c] = v;
            }
        if (lane == 0) {
            double *out = a.part + (int64_t)jc * NR * a.part_ld + pos;
#pragma unroll
            for (int k = 0; k <= P; ++k)
#pragma unroll
                for (int c = 0; c < 3; ++c) out[(3 * k + c) * a.part_ld] = acc64[k][c];
        }
    }
}

// FP64 plan for evaluations too small to fill the GPU with 128-body i-tiles
// (few bodies, or a short active list): one warp per CTA, 32-body i-tiles and
// j-tiles as short as 2, so that the pairs spread over every SM (GB300 has two
// FP64 lanes per SM, so an SM left idle is a large loss).
static PairPlan plan_fine64(int64_t n_i, int64_t n_j, int split_hint, int n_sm)
{
    PairPlan pl{};
    pl.threads = 32;
    pl.i_per_cta = 32;
    pl.n_itiles = (n_i + 31) / 32;
    const int slots = n_sm * 16;                          // resident one-warp CTAs per device
    pl.tj = 64;
    while (pl.tj > 2 && pl.n_itiles * std::min<int64_t>(64, (n_j + pl.tj - 1) / pl.tj) < 4 * (int64_t)n_sm)
        pl.tj /= 2;
    const int64_t n_jt = (n_j + pl.tj - 1) / pl.tj;
    int best_S = 1;
    double best_cost = 1e300;
    // up to 64 j-chunks, more when few i-tiles would leave SMs idle (active lists
    // of a few bodies under block steps: the callers size the partial sums by
    // the evaluated bodies, so the extra slots are small)
    const int s_cap = (int)std::max<int64_t>(64, std::min<int64_t>(slots / std::max<int64_t>(pl.n_itiles, 1), 512));
    const int s_max = (int)std::min<int64_t>(s_cap, n_jt);
    // a split hint takes the largest split <= hint that cuts the j-tiles into
    // chunks of equal length (the hint itself when it does)
    int hinted = 0;
    if (split_hint > 0)
        for (int S = std::min(split_hint, s_max); S >= 1 && !hinted; --S)
            if ((n_jt + (n_jt + S - 1) / S - 1) / ((n_jt + S - 1) / S) == S) hinted = S;
    for (int S = 1; S <= s_max; ++S) {
        if (hinted && S != hinted) continue;
        const int64_t tiles_per_chunk = (n_jt + S - 1) / S;
        if ((n_jt + tiles_per_chunk - 1) / tiles_per_chunk != S) continue;
        const int64_t waves = (pl.n_itiles * S + slots - 1) / slots;
        const double cost = (double)waves * tiles_per_chunk * (1.0 + 0.002 * S);
        if (cost < best_cost) { best_cost = cost; best_S = S; }
    }
    pl.split = best_S;
    pl.chunk = (n_jt + best_S - 1) / best_S * pl.tj;
    pl.grid = (int)std::min<int64_t>(pl.n_itiles * pl.split, slots);
    return pl;
}

PairPlan plan_pair(int P, int precision, int64_t n_i, int64_t n_j, int split_hint, int device, int variant)
{
    const int ipt = variant;
    static int n_sm_cache[64] = {0};
    int n_sm = device >= 0 && device < 64 ? n_sm_cache[device] : 0;
    if (n_sm == 0) {
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
        if (n_sm <= 0) n_sm = 148;
        if (device >= 0 && device < 64) n_sm_cache[device] = n_sm;
    }
    PairPlan pl{};
    pl.threads = precision == MH_PREC_FP64 ? 128 : kThreads32;
    pl.ipt = precision == MH_PREC_FP64 ? 1 : (ipt >= 2 ? 2 : 1);
    pl.packed = precision != MH_PREC_FP64 && ipt == 3;
    pl.i_per_cta = pl.threads * pl.ipt;
    pl.tj = precision == MH_PREC_FP64 ? 64 : 128;
    const int occ = precision == MH_PREC_FP64 ? 4 : 2;     // resident CTAs per SM
    const int slots = n_sm * occ;
    pl.n_itiles = (n_i + pl.i_per_cta - 1) / pl.i_per_cta;
    const int64_t n_jt = (n_j + pl.tj - 1) / pl.tj;        // j-tiles
    int best_S = 1;
    double best_cost = 1e300;
    // up to 64 j-chunks, more when few i-tiles would leave SMs idle (active lists
    // of a few bodies under block steps: the callers size the partial sums by
    // the evaluated bodies, so the extra slots are small)
    const int s_cap = (int)std::max<int64_t>(64, std::min<int64_t>(slots / std::max<int64_t>(pl.n_itiles, 1), 512));
    const int s_max = (int)std::min<int64_t>(s_cap, n_jt);
    // a split hint takes the largest split <= hint that cuts the j-tiles into
    // chunks of equal length (the hint itself when it does)
    int hinted = 0;
    if (split_hint > 0)
        for (int S = std::min(split_hint, s_max); S >= 1 && !hinted; --S)
            if ((n_jt + (n_jt + S - 1) / S - 1) / ((n_jt + S - 1) / S) == S) hinted = S;
    for (int S = 1; S <= s_max; ++S) {
        if (hinted && S != hinted) continue;
        const int64_t tiles_per_chunk = (n_jt + S - 1) / S;
        const int64_t S_eff = (n_jt + tiles_per_chunk - 1) / tiles_per_chunk;
        if (S_eff != S) continue;
        const int64_t items = pl.n_itiles * S;
        const int64_t waves = (items + slots - 1) / slots;
        // time ~ waves x tiles per item; small penalty per chunk for the partial-sum traffic
        const double cost = (double)waves * tiles_per_chunk * (1.0 + 0.002 * S);
        if (cost < best_cost) { best_cost = cost; best_S = S; }
    }
    pl.split = best_S;
    const int64_t tiles_per_chunk = (n_jt + best_S - 1) / best_S;
    pl.chunk = tiles_per_chunk * pl.tj;
    const int64_t items = pl.n_itiles * pl.split;
    pl.grid = (int)std::min<int64_t>(items, slots);
    if (precision == MH_PREC_FP64 && items < 2 * (int64_t)n_sm) return plan_fine64(n_i, n_j, split_hint, n_sm);
    return pl;
}

int plan_short(int64_t n_i, int64_t n_j, int device)
{
    static int n_sm_cache[64] = {0};
    int n_sm = device >= 0 && device < 64 ? n_sm_cache[device] : 0;
    if (n_sm == 0) {
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
        if (n_sm <= 0) n_sm = 148;
        if (device >= 0 && device < 64) n_sm_cache[device] = n_sm;
    }
    // about 16 warps per SM in all, and at least 64 sources per warp
    const int64_t want = (16 * (int64_t)n_sm + n_i - 1) / std::max<int64_t>(n_i, 1);
    const int64_t cap = std::max<int64_t>(1, n_j / 64);
    return (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(want, cap), 4096));
}

int launch_pair_short(int P, int precision, int64_t n_i, int64_t n_j, int64_t ld, const double *m,
                      const double *jrec, const float *jrec32, double eps, double G, double *part,
                      int64_t part_ld, int split, const int *ilist, cudaStream_t st)
{
    if (P < 1 || P > 3 || split < 1 || n_i < 1) {
        set_error("launch_pair_short: P must be 1..3, split and n_i positive");
        return MH_EINVAL;
    }
    const int64_t chunk = (n_j + split - 1) / split;
    const int64_t warps = n_i * split;
    const unsigned grid = (unsigned)std::min<int64_t>((warps + 3) / 4, 65535);
    const bool f32 = precision == MH_PREC_FP32PAIR;
    auto go = [&](auto tag) -> int {
        constexpr int PP = decltype(tag)::value;
        ShortArgs<PP> a{jrec, m, jrec32, ld, n_j, n_i, eps * eps, G, part, part_ld, chunk, split, ilist};
        if (f32)
            k_pair_short<PP, true><<<grid, 128, 0, st>>>(a);
        else
            k_pair_short<PP, false><<<grid, 128, 0, st>>>(a);
        MH_LAUNCHED("k_pair_short");
        return MH_OK;
    };
    switch (P) {
    case 1: return go(std::integral_constant<int, 1>{});
    case 2: return go(std::integral_constant<int, 2>{});
    default: return go(std::integral_constant<int, 3>{});
    }
}

int launch_pair(int P, int precision, int64_t n_j, int64_t ld, const double *m, const double *jrec,
                const float *jrec32, double eps, double G, int64_t i0, int64_t i1, double *part,
                int64_t part_ld, const PairPlan &pl, cudaStream_t st, const int *ilist,
                unsigned long long *wmax)
{
    if (precision == MH_PREC_FP64) {
        if (wmax && P > 5) {
            set_error("launch_pair: the Eq. 24 maximum is tracked for P <= 5 only");
            return MH_EINVAL;
        }
        switch (P) {
        case 1: return launch_fp64<1>(jrec, m, ld, n_j, eps, G, i0, i1, part, part_ld, pl, ilist, st, wmax);
        case 2: return launch_fp64<2>(jrec, m, ld, n_j, eps, G, i0, i1, part, part_ld, pl, ilist, st, wmax);
        case 3: return launch_fp64<3>(jrec, m, ld, n_j, eps, G, i0, i1, part, part_ld, pl, ilist, st, wmax);
        // P = 4, 5: the 10th- and 12th-order steps; P = 5, 7, 9: initialisation passes
        case 4: return launch_fp64<4>(jrec, m, ld, n_j, eps, G, i0, i1, part, part_ld, pl, ilist, st, wmax);
        case 5: return launch_fp64<5>(jrec, m, ld, n_j, eps, G, i0, i1, part, part_ld, pl, ilist, st, wmax);
        case 7: return launch_fp64<7>(jrec, m, ld, n_j, eps, G, i0, i1, part, part_ld, pl, ilist, st, nullptr);
        case 9: return launch_fp64<9>(jrec, m, ld, n_j, eps, G, i0, i1, part, part_ld, pl, ilist, st, nullptr);
        }
    } else {
        switch (P) {
        // the FP32 input rows carry G m: G is applied when they are written
        case 1: return launch_fp32<1>(jrec32, ld, n_j, eps, i0, i1, part, part_ld, pl, ilist, st);
        case 2: return launch_fp32<2>(jrec32, ld, n_j, eps, i0, i1, part, part_ld, pl, ilist, st);
        case 3: return launch_fp32<3>(jrec32, ld, n_j, eps, i0, i1, part, part_ld, pl, ilist, st);
        }
    }
    set_error("launch_pair: unsupported P/precision");
    return MH_EINVAL;
}

}  // namespace mh
