// FP64 all-pairs evaluation of a^(0..P) that computes every unordered pair once
// (the E of P(EC)^n under shared steps, and the initialisation passes P <= 5).
//
// Pair physics (Dittmann 2020, Section 3, intro): a_ij = G m_j r_ij s^(-3/2).
// With the scaled terms B_k of pair_math.cuh, body i receives G m_j S B_k(i,j)
// and body j receives G m_i S B_k(j,i) = -G m_i S B_k(i,j): the terms are odd
// under i <-> j and S, alpha, beta, gamma are even.  One evaluation of the pair
// therefore serves both bodies, and an interaction costs about 96 FP64
// operations per unordered pair instead of 2 x 83 for two ordered pairs.  On a
// part with two FP64 lanes per SM this halves the time of the FP64 form; the
// extra data movement (shuffles, shared memory) runs on otherwise idle pipes.
//
// Decomposition.  Bodies are cut into blocks of R = 128 (the padded count Np is
// a multiple of R; nB blocks).  Block row I handles the diagonal block (I, I)
// and the blocks J = I + d (mod nB), d = 1 .. D with D = floor(nB/2); when nB
// is even (always, for the simulation's padding to 256) the block pair at
// d = nB/2 is done by the rows I < nB/2 only.  Every unordered block pair is
// then done exactly once and every row has the same amount of work, to one block.  A row is cut into C chunks of blocks; an item is one
// (row, chunk) and CTAs loop over items with a grid stride.
//
// Inside a CTA (4 warps) warp w holds the 32 i-bodies I*R + 32w + lane.  For
// an off-diagonal block the warps take the block's four 32-body j-subtiles in
// a rotation (warp w takes subtile (w + jt) mod 4 at stage jt); a warp runs the
// 32 x 32 pairs of a subtile as a ring: each lane holds one j-body with its
// j-side accumulator and passes both one lane on after every pair.  The j-side
// sums of a subtile move between warps through shared memory at the stage
// barriers.  The diagonal block is evaluated as ordered pairs (i-side only,
// the i == j pair guarded).
//
// Output: the partial-sum slots of the other evaluation kernels, S = C + D of
// them: slot c < C holds row chunk c's sums for its own bodies, slot C + d - 1
// the sums that the block at distance d wrote into its j-bodies (zero where no
// such block exists).  The corrector adds the S slots in a fixed order, so the
// result is deterministic and independent of which CTA ran which item.
#include <algorithm>

#include "common.cuh"
#include "pair_math.cuh"

namespace mh {

namespace {

constexpr int kSymWarps = 4;
constexpr int kSymR = 32 * kSymWarps;     // bodies per block

template <int P>
struct SymArgs {
    const double *jrec;   // [3(P+1)][ld]
    const double *m;      // [ld]
    int64_t ld;           // row stride (the padded body count, a multiple of kSymR)
    int64_t N;            // bodies; positions N .. ld-1 are padding
    int nB, D, C, Bc;     // blocks, distances, row chunks, blocks per chunk
    double eps2, G;
    double *part;         // [C + D][(P+1)*3][ld]
    unsigned long long *wmax;   // kH: max over pairs of G (m_i + m_j) s^(-3/2) (bit pattern), raised
};

// Record of body b.  Padding bodies get mass 0 and distinct far-away positions,
// so that no pair has r = 0 (their own sums are never read).
template <int P>
__device__ __forceinline__ void load_body(const SymArgs<P> &a, int64_t b, double (&r)[P + 1][3], double &gm)
{
    if (b < a.N) {
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[k][c] = a.jrec[(3 * k + c) * a.ld + b];
        gm = a.G * a.m[b];
    } else {
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) r[k][c] = 0.0;
        r[0][0] = kFarAway + (double)(b - a.N);
        gm = 0.0;
    }
}

template <int P>
__device__ __forceinline__ void rotate(double (&r)[P + 1][3], double &gm, int src)
{
#pragma unroll
    for (int k = 0; k <= P; ++k)
#pragma unroll
        for (int c = 0; c < 3; ++c) r[k][c] = __shfl_sync(0xffffffffu, r[k][c], src);
    gm = __shfl_sync(0xffffffffu, gm, src);
}

// kH: also track w = G (m_i + m_j) s^(-3/2) over all pairs i != j, whose maximum
// gives the time-step criterion of Section 3.3 (Eq. 24: H = eta w_max^(-1/2)).
// Non-negative doubles order as their bit patterns, so the maximum is an
// integer maximum (off the FP64 pipe) and the result does not depend on the
// order of the pairs.
template <int P, bool kH>
__global__ void __launch_bounds__(kSymR, 2) k_pair_fp64_sym(SymArgs<P> a)
{
    constexpr int NR = 3 * (P + 1);
    unsigned long long wm = 0ull;
    __shared__ double accs[NR][kSymR];    // j-side sums of the current block, by column
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int src = (lane + 1) & 31;      // ring: after t passes lane l holds j-lane (l + t) mod 32
    const bool even = (a.nB & 1) == 0;
    const int64_t items = (int64_t)a.nB * a.C;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int I = (int)(item % a.nB);
        const int ch = (int)(item / a.nB);
        const int64_t ib = (int64_t)I * kSymR + threadIdx.x;
        double ri[P + 1][3], gmi;
        load_body<P>(a, ib, ri, gmi);
        double acci[P + 1][3];
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) acci[k][c] = 0.0;

        const int dmax = (even && I >= a.nB / 2) ? a.D - 1 : a.D;
        const int b0 = ch * a.Bc;
        const int b1 = min(b0 + a.Bc, dmax + 1);
        for (int b = b0; b < b1; ++b) {
            if (b == 0) {
                // diagonal block: ordered pairs into the i-side only
                for (int js = 0; js < kSymWarps; ++js) {
                    double rj[P + 1][3], gmj;
                    load_body<P>(a, (int64_t)I * kSymR + js * 32 + lane, rj, gmj);
                    for (int t = 0; t < 32; ++t) {
                        const bool self = js == w && t == 0;
                        double r[P + 1][3];
#pragma unroll
                        for (int k = 0; k <= P; ++k)
#pragma unroll
                            for (int c = 0; c < 3; ++c) r[k][c] = rj[k][c] - ri[k][c];
                        double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], a.eps2)));
                        s = self ? 1.0 : s;
                        const double wi = self ? 0.0 : gmj;
                        const double rinv = rsqrt_fp64(s);
                        const double sinv = rinv * rinv;
                        const double S = rinv * sinv;
                        const double mS = wi * S;
                        if constexpr (kH) {
                            const unsigned long long wb = self ? 0ull : (unsigned long long)__double_as_longlong((gmi + gmj) * S);
                            wm = wb > wm ? wb : wm;
                        }
                        pair_odd_terms<P, double>(r, sinv, [&](int k, int c, double B) {
                            acci[k][c] = fma(mS, B, acci[k][c]);
                        });
                        rotate<P>(rj, gmj, src);
                    }
                }
                continue;
            }
            const int J = (I + b) % a.nB;
            for (int jt = 0; jt < kSymWarps; ++jt) {
                const int js = (w + jt) % kSymWarps;
                double rj[P + 1][3], gmj, accj[P + 1][3];
                load_body<P>(a, (int64_t)J * kSymR + js * 32 + lane, rj, gmj);
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) accj[k][c] = jt == 0 ? 0.0 : accs[3 * k + c][js * 32 + lane];
                for (int t = 0; t < 32; ++t) {
                    double r[P + 1][3];
#pragma unroll
                    for (int k = 0; k <= P; ++k)
#pragma unroll
                        for (int c = 0; c < 3; ++c) r[k][c] = rj[k][c] - ri[k][c];
                    const double s = fma(r[0][0], r[0][0], fma(r[0][1], r[0][1], fma(r[0][2], r[0][2], a.eps2)));
                    const double rinv = rsqrt_fp64(s);
                    const double sinv = rinv * rinv;
                    const double S = rinv * sinv;
                    const double wi = gmj * S, wj = gmi * S;
                    if constexpr (kH) {
                        const unsigned long long wb = (unsigned long long)__double_as_longlong(wi + wj);
                        wm = wb > wm ? wb : wm;
                    }
                    pair_odd_terms<P, double>(r, sinv, [&](int k, int c, double B) {
                        acci[k][c] = fma(wi, B, acci[k][c]);
                        accj[k][c] = fma(-wj, B, accj[k][c]);
                    });
                    rotate<P>(rj, gmj, src);
#pragma unroll
                    for (int k = 0; k <= P; ++k)
#pragma unroll
                        for (int c = 0; c < 3; ++c) accj[k][c] = __shfl_sync(0xffffffffu, accj[k][c], src);
                }
#pragma unroll
                for (int k = 0; k <= P; ++k)
#pragma unroll
                    for (int c = 0; c < 3; ++c) accs[3 * k + c][js * 32 + lane] = accj[k][c];
                __syncthreads();
            }
            double *out = a.part + (int64_t)(a.C + b - 1) * NR * a.ld + (int64_t)J * kSymR + threadIdx.x;
#pragma unroll
            for (int q = 0; q < NR; ++q) out[q * a.ld] = accs[q][threadIdx.x];
            __syncthreads();
        }
        if (even && I >= a.nB / 2 && ch == a.C - 1) {
            // this row has no block at d = D: its slot in block I + D stays zero
            const int J = (I + a.D) % a.nB;
            double *out = a.part + (int64_t)(a.C + a.D - 1) * NR * a.ld + (int64_t)J * kSymR + threadIdx.x;
#pragma unroll
            for (int q = 0; q < NR; ++q) out[q * a.ld] = 0.0;
        }
        double *out = a.part + (int64_t)ch * NR * a.ld + ib;
#pragma unroll
        for (int k = 0; k <= P; ++k)
#pragma unroll
            for (int c = 0; c < 3; ++c) out[(3 * k + c) * a.ld] = acci[k][c];
    }
    if constexpr (kH) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long q = __shfl_xor_sync(0xffffffffu, wm, o);
            wm = q > wm ? q : wm;
        }
        if (lane == 0 && wm) atomicMax(a.wmax, wm);
    }
}

template <int P>
int launch_sym(const SymPlan &pl, const double *jrec, const double *m, int64_t ld, int64_t N, double eps,
               double G, double *part, unsigned long long *wmax, cudaStream_t st)
{
    SymArgs<P> a{jrec, m, ld, N, pl.nB, pl.D, pl.C, pl.Bc, eps * eps, G, part, wmax};
    if (wmax)
        k_pair_fp64_sym<P, true><<<pl.grid, kSymR, 0, st>>>(a);
    else
        k_pair_fp64_sym<P, false><<<pl.grid, kSymR, 0, st>>>(a);
    MH_LAUNCHED("k_pair_fp64_sym");
    return MH_OK;
}

// ---------------------------------------------------------------------------
// FP32-pair form, each unordered pair once.  Same block schedule, ring and
// partial-sum slots as the FP64 kernel above; the pair arithmetic is the
// precision form's: x and v differences from the hi/lo split, (hi_j - hi_i) +
// (lo_j - lo_i), everything else of the pair in FP32.  The FP32 sums cover one
// 32-step ring and are then added to FP64 accumulators: registers for the
// i-side, the shared-memory column sums for the j-side.
// ---------------------------------------------------------------------------

template <int P>
struct SymArgs32 {
    const float *jrec32;  // [nf32(P)][ld]: x_hi, x_lo, v_hi, v_lo, a, a-dot, G m
    int64_t ld, N;
    int nB, D, C, Bc;
    float eps2;
    double *part;         // [C + D][(P+1)*3][ld]
};

template <int P>
struct Rec32s {
    static constexpr int NF = nf32(P);
};

// Record of body b; padding bodies massless at distinct far-away positions.
template <int P>
__device__ __forceinline__ void load_body32(const SymArgs32<P> &a, int64_t b, float (&r)[Rec32s<P>::NF])
{
    constexpr int NF = Rec32s<P>::NF;
    if (b < a.N) {
#pragma unroll
        for (int q = 0; q < NF; ++q) r[q] = a.jrec32[q * a.ld + b];
    } else {
#pragma unroll
        for (int q = 0; q < NF; ++q) r[q] = 0.0f;
        r[0] = (float)kFarAway + (float)(b - a.N);
    }
}

// Relative trajectory derivatives of the pair (j - i) from two records.
template <int P>
__device__ __forceinline__ void rel32(const float (&ri)[Rec32s<P>::NF], const float (&rj)[Rec32s<P>::NF],
                                      float (&r)[P + 1][3])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        r[0][c] = (rj[c] - ri[c]) + (rj[3 + c] - ri[3 + c]);
        r[1][c] = (rj[6 + c] - ri[6 + c]) + (rj[9 + c] - ri[9 + c]);
        if constexpr (P >= 2) r[2][c] = rj[12 + c] - ri[12 + c];
        if constexpr (P >= 3) r[3][c] = rj[15 + c] - ri[15 + c];
    }
}

// Two warps per CTA, two i-bodies per lane: lane l of warp w holds the bodies
// of i-subtiles 2w and 2w + 1 in the two lanes of Blackwell's paired FP32
// instructions (FFMA2/FMUL2/FADD2), so every j-record passed around the ring
// serves two pairs and one issue slot advances both.  The i-side sums are
// packed too; the j-side sum of a ring lane adds both pairs' terms in FP32.
// FP32 sums cover one 128-body block (as the tiles of the ordered kernels) and
// are added to FP64 once per block.
constexpr int kSym32Warps = 2;

__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }

// The scaled terms B_k of pair_abg_terms for two pairs at once (negated
// coefficients so that every update is one multiply-add); sink(k, c, B).
template <int P, typename Sink>
__device__ __forceinline__ void pair_abg_terms_x2(const float2 (&r)[P + 1][3], float2 sinv, Sink &&sink)
{
    const float2 rv = fma2(r[0][2], r[1][2], fma2(r[0][1], r[1][1], mul2(r[0][0], r[1][0])));
    const float2 al = mul2(rv, sinv);
    const float2 na3 = mul2(f2(-3.0f), al);
    float2 B1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        B1[c] = fma2(na3, r[0][c], r[1][c]);
        sink(0, c, r[0][c]);
        sink(1, c, B1[c]);
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
            sink(2, c, B2[c]);
        }
        if constexpr (P >= 3) {
            const float2 va = fma2(r[1][2], r[2][2], fma2(r[1][1], r[2][1], mul2(r[1][0], r[2][0])));
            const float2 rj = fma2(r[0][2], r[3][2], fma2(r[0][1], r[3][1], mul2(r[0][0], r[3][0])));
            const float2 w3 = fma2(f2(3.0f), va, rj);
            // gamma = w3/s + alpha (3 beta - 4 alpha^2), 3 beta - 4 alpha^2 = -(nb3 + 4 alpha^2)
            const float2 u = fma2(f2(4.0f), al2, nb3);
            const float2 ga = fma2(w3, sinv, mul2(mul2(f2(-1.0f), al), u));
            const float2 na9 = mul2(f2(-9.0f), al), nb9 = mul2(f2(-9.0f), be), ng3 = mul2(f2(-3.0f), ga);
#pragma unroll
            for (int c = 0; c < 3; ++c) sink(3, c, fma2(ng3, r[0][c], fma2(nb9, B1[c], fma2(na9, B2[c], r[3][c]))));
        }
    }
}

template <int P>
__global__ void __launch_bounds__(32 * kSym32Warps, 4) k_pair_fp32_sym(SymArgs32<P> a)
{
    constexpr int NF = Rec32s<P>::NF;
    constexpr int NR = 3 * (P + 1);
    __shared__ float accs[NR][kSymR];     // j-side FP32 sums of the current block, by column
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int src = (lane + 1) & 31;
    const bool even = (a.nB & 1) == 0;
    const float2 eps2 = f2(a.eps2);
    const int64_t items = (int64_t)a.nB * a.C;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int I = (int)(item % a.nB);
        const int ch = (int)(item / a.nB);
        // the lane's two i-bodies, negated (differences become additions), packed
        float2 ni[NF - 1], gmi;
        {
            float r0[NF], r1[NF];
            load_body32<P>(a, (int64_t)I * kSymR + (2 * w) * 32 + lane, r0);
            load_body32<P>(a, (int64_t)I * kSymR + (2 * w + 1) * 32 + lane, r1);
#pragma unroll
            for (int q = 0; q < NF - 1; ++q) ni[q] = make_float2(-r0[q], -r1[q]);
            gmi = make_float2(r0[NF - 1], r1[NF - 1]);
        }
        double acc64[2][NR];
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int q = 0; q < NR; ++q) acc64[k][q] = 0.0;

        const int dmax = (even && I >= a.nB / 2) ? a.D - 1 : a.D;
        const int b0 = ch * a.Bc;
        const int b1 = min(b0 + a.Bc, dmax + 1);
        for (int b = b0; b < b1; ++b) {
            const bool diag = b == 0;
            const int J = (I + b) % a.nB;
            float2 acci[P + 1][3];
#pragma unroll
            for (int n = 0; n <= P; ++n)
#pragma unroll
                for (int c = 0; c < 3; ++c) acci[n][c] = f2(0.0f);
            for (int jt = 0; jt < 4; ++jt) {
                // off-diagonal: at stage jt warp w takes j-subtile (2w + jt) mod 4 (the two
                // warps never share one); diagonal block: every warp takes every subtile
                const int js = diag ? jt : (2 * w + jt) & 3;
                float rj[NF];
                load_body32<P>(a, (int64_t)J * kSymR + js * 32 + lane, rj);
                float accj[P + 1][3];
#pragma unroll
                for (int n = 0; n <= P; ++n)
#pragma unroll
                    for (int c = 0; c < 3; ++c) accj[n][c] = 0.0f;
                for (int t = 0; t < 32; ++t) {
                    float2 r[P + 1][3];
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        r[0][c] = add2(add2(f2(rj[c]), ni[c]), add2(f2(rj[3 + c]), ni[3 + c]));
                        r[1][c] = add2(add2(f2(rj[6 + c]), ni[6 + c]), add2(f2(rj[9 + c]), ni[9 + c]));
                        if constexpr (P >= 2) r[2][c] = add2(f2(rj[12 + c]), ni[12 + c]);
                        if constexpr (P >= 3) r[3][c] = add2(f2(rj[15 + c]), ni[15 + c]);
                    }
                    float2 s = fma2(r[0][0], r[0][0], fma2(r[0][1], r[0][1], fma2(r[0][2], r[0][2], eps2)));
                    const bool self0 = diag && js == 2 * w && t == 0;
                    const bool self1 = diag && js == 2 * w + 1 && t == 0;
                    s.x = self0 ? 1.0f : s.x;
                    s.y = self1 ? 1.0f : s.y;
                    const float2 rinv = make_float2(rsqrt_mufu(s.x), rsqrt_mufu(s.y));
                    const float2 sinv = mul2(rinv, rinv);
                    const float2 S = mul2(rinv, sinv);
                    float2 wi = mul2(f2(rj[NF - 1]), S);
                    wi.x = self0 ? 0.0f : wi.x;
                    wi.y = self1 ? 0.0f : wi.y;
                    const float2 wj = diag ? f2(0.0f) : mul2(gmi, S);
                    pair_abg_terms_x2<P>(r, sinv, [&](int n, int c, float2 B) {
                        acci[n][c] = fma2(wi, B, acci[n][c]);
                        accj[n][c] = fmaf(-wj.y, B.y, fmaf(-wj.x, B.x, accj[n][c]));
                    });
#pragma unroll
                    for (int q = 0; q < NF; ++q) rj[q] = __shfl_sync(0xffffffffu, rj[q], src);
                    if (!diag) {
#pragma unroll
                        for (int n = 0; n <= P; ++n)
#pragma unroll
                            for (int c = 0; c < 3; ++c) accj[n][c] = __shfl_sync(0xffffffffu, accj[n][c], src);
                    }
                }
                if (!diag) {
                    // each column is visited twice, by warp 0 and by warp 1: first at stage
                    // 0 (columns 0, 2) or 1 (columns 1, 3), second at stage 2 or 3
#pragma unroll
                    for (int n = 0; n <= P; ++n)
#pragma unroll
                        for (int c = 0; c < 3; ++c) {
                            float &cell = accs[3 * n + c][js * 32 + lane];
                            cell = (jt < 2 ? 0.0f : cell) + accj[n][c];
                        }
                    __syncthreads();
                }
            }
#pragma unroll
            for (int n = 0; n <= P; ++n)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    acc64[0][3 * n + c] += (double)acci[n][c].x;
                    acc64[1][3 * n + c] += (double)acci[n][c].y;
                }
            if (!diag) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const int col = threadIdx.x + k * 64;
                    double *out = a.part + (int64_t)(a.C + b - 1) * NR * a.ld + (int64_t)J * kSymR + col;
#pragma unroll
                    for (int q = 0; q < NR; ++q) out[q * a.ld] = (double)accs[q][col];
                }
                __syncthreads();
            }
        }
        if (even && I >= a.nB / 2 && ch == a.C - 1) {
            const int J = (I + a.D) % a.nB;
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                double *out = a.part + (int64_t)(a.C + a.D - 1) * NR * a.ld + (int64_t)J * kSymR + threadIdx.x + k * 64;
#pragma unroll
                for (int q = 0; q < NR; ++q) out[q * a.ld] = 0.0;
            }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            double *out = a.part + (int64_t)ch * NR * a.ld + (int64_t)I * kSymR + (2 * w + k) * 32 + lane;
#pragma unroll
            for (int q = 0; q < NR; ++q) out[q * a.ld] = acc64[k][q];
        }
    }
}

template <int P>
int launch_sym32(const SymPlan &pl, const float *jrec32, int64_t ld, int64_t N, double eps, double *part,
                 cudaStream_t st)
{
    SymArgs32<P> a{jrec32, ld, N, pl.nB, pl.D, pl.C, pl.Bc, (float)(eps * eps), part};
    k_pair_fp32_sym<P><<<pl.grid, 32 * kSym32Warps, 0, st>>>(a);
    MH_LAUNCHED("k_pair_fp32_sym");
    return MH_OK;
}

}  // namespace

SymPlan plan_sym(int P, int64_t ld, int device, bool fp32)
{
    SymPlan pl{};
    if (ld % kSymR != 0 || ld < kSymR || P < 1 || P > (fp32 ? 3 : 5)) return pl;
    // resident CTAs per device, cached per (device, P, form)
    static int slot_cache[64][16] = {{0}};
    const int ci = P + (fp32 ? 8 : 0);
    int slots = device >= 0 && device < 64 ? slot_cache[device][ci] : 0;
    if (slots == 0) {
        int n_sm = 0, occ = 0;
        cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, device);
        if (fp32) {
            const void *fn = P == 1 ? (const void *)k_pair_fp32_sym<1>
                           : P == 2 ? (const void *)k_pair_fp32_sym<2> : (const void *)k_pair_fp32_sym<3>;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 32 * kSym32Warps, 0);
        } else {
            const void *fn = P == 1 ? (const void *)k_pair_fp64_sym<1, false>
                           : P == 2 ? (const void *)k_pair_fp64_sym<2, false>
                           : P == 3 ? (const void *)k_pair_fp64_sym<3, false>
                           : P == 4 ? (const void *)k_pair_fp64_sym<4, false> : (const void *)k_pair_fp64_sym<5, false>;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kSymR, 0);
        }
        slots = std::max(n_sm, 1) * std::max(occ, 1);
        if (device >= 0 && device < 64) slot_cache[device][ci] = slots;
    }
    pl.nB = (int)(ld / kSymR);
    pl.D = pl.nB / 2;
    const int nb = pl.D + 1;                        // blocks of the longest row
    // items of equal size; pick the chunk count with the fewest block-times on the
    // busiest CTA (the diagonal block counts about twice, it runs ordered pairs)
    double best = 1e300;
    for (int C = 1; C <= nb; ++C) {
        const int Bc = (nb + C - 1) / C;
        if ((nb + Bc - 1) / Bc != C) continue;
        const int64_t items = (int64_t)pl.nB * C;
        const int64_t waves = (items + slots - 1) / slots;
        const double cost = (double)waves * (Bc + 1.0) * (1.0 + 0.001 * C);
        if (cost < best) {
            best = cost;
            pl.C = C;
            pl.Bc = Bc;
        }
    }
    pl.grid = (int)std::min<int64_t>((int64_t)pl.nB * pl.C, slots);
    pl.slots = pl.C + pl.D;
    return pl;
}

int launch_pair_sym32(int P, const SymPlan &pl, const float *jrec32, int64_t ld, int64_t N, double eps,
                      double *part, cudaStream_t st)
{
    switch (P) {
    case 1: return launch_sym32<1>(pl, jrec32, ld, N, eps, part, st);
    case 2: return launch_sym32<2>(pl, jrec32, ld, N, eps, part, st);
    case 3: return launch_sym32<3>(pl, jrec32, ld, N, eps, part, st);
    }
    set_error("launch_pair_sym32: P must be 1..3");
    return MH_EINVAL;
}

int launch_pair_sym(int P, const SymPlan &pl, const double *jrec, const double *m, int64_t ld, int64_t N,
                    double eps, double G, double *part, cudaStream_t st, unsigned long long *wmax)
{
    switch (P) {
    case 1: return launch_sym<1>(pl, jrec, m, ld, N, eps, G, part, wmax, st);
    case 2: return launch_sym<2>(pl, jrec, m, ld, N, eps, G, part, wmax, st);
    case 3: return launch_sym<3>(pl, jrec, m, ld, N, eps, G, part, wmax, st);
    case 4: return launch_sym<4>(pl, jrec, m, ld, N, eps, G, part, wmax, st);
    case 5: return launch_sym<5>(pl, jrec, m, ld, N, eps, G, part, wmax, st);
    }
    set_error("launch_pair_sym: P must be 1..5");
    return MH_EINVAL;
}

}  // namespace mh
