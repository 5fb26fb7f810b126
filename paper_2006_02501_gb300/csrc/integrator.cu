// O(N) kernels of one P(EC)^n step (Dittmann 2020, Section 2 and Section 3 intro):
//   k_predict   Taylor predictor of x, v and the a-derivatives the evaluation
//               needs; writes the evaluation input (FP64 rows or the FP32
//               hi/lo rows of the precision form).
//   k_correct   adds the split-j partial sums of the evaluation, applies the
//               corrector (velocity first, Eq. 6, then position with the new
//               velocity, Eq. 7 with beta of Eq. 20 or beta = 1), writes the
//               next evaluation input; after the last pass also the Hermite
//               interpolation of a^(p+1..2p-1) at t1 and the commit t0 <- t1.
//   k_init_rows / k_init_reduce   plumbing of the explicit initial derivatives.
// One thread per body; arrays are SoA rows of length ld (coalesced).
#include "common.cuh"
#include "hermite_consts.cuh"
#include "hermite_step.cuh"

namespace mh {

namespace {

struct StepArgs {
    int64_t N, ld;
    double dt;
    const double *m;
    double *x0, *v0, *d0;     // committed state at t0 (d0: [2p][3][ld])
    double *x1, *v1;          // estimate at t1
    double *jrec;             // FP64 evaluation input [3(p+1)][ld] (x, v, a, a-dot)
    float *jrec32;            // FP32 evaluation input [nf32(p)][ld]
    const double *part;       // [S][(p+1)*3][ld]
    int split;
    int precision;
    int beta_mode;
    int *flag;
    const unsigned long long *bound_rd;   // [x, v] grid bounds read by this kernel
    unsigned long long *bound_wr;         // [x, v] raised with this kernel's values
    unsigned long long *conv = nullptr;   // optional [max |x_new - x_old|, max |x_new|] (double bits)
    TimeSymArgs ts{};                     // time-symmetric variable step (ts.w != null), else dt above
    double *comp = nullptr;               // optional [6][ld]: compensation of x, v (Kahan), committed by the last pass
};

// H of Eq. 24 from a word holding the maximum over pairs of G (m_i + m_j) s^(-3/2).
__device__ __forceinline__ double eq24_H(const TimeSymArgs &ts, int idx)
{
    return ts.eta * rsqrt(__longlong_as_double((long long)ts.w[idx]));
}

// Step of the predictor: dir H- (Section 3.3; the first estimate of dt).
__device__ __forceinline__ double predictor_dt(const StepArgs &a)
{
    return a.ts.w ? a.ts.dir * eq24_H(a.ts, a.ts.prev) : a.dt;
}

// Time-symmetric steps (Section 3.3, reading R15): pass k corrects with the dt
// its evaluation was made at -- dir H- for the first pass, dir (H- + H+_(k-1))/2
// after -- and, unless it is the last pass, moves the corrected end state to the
// next dt = dir (H- + H+_k)/2, H+_k being Eq. 24 at the positions pass k evaluated.
__device__ __forceinline__ double timesym_dt(const StepArgs &a, int after_pass)
{
    const double Hm = eq24_H(a.ts, a.ts.prev);
    return after_pass < 0 ? a.ts.dir * Hm
                          : a.ts.dir * 0.5 * (Hm + eq24_H(a.ts, a.ts.bank * kTsMaxIter + after_pass));
}

__device__ __forceinline__ double corrector_dt(const StepArgs &a)
{
    return a.ts.w ? timesym_dt(a, a.ts.pass - 1) : a.dt;
}

__device__ __forceinline__ void raise_bound(unsigned long long *slot, double val)
{
    // warp-wide max of non-negative doubles through their bit patterns, one atomic per warp
    unsigned long long b = __double_as_longlong(val);
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, b, o);
        b = q > b ? q : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(slot, b);
}

// Evaluation input of body i (FP64 rows 3k+c: x, v, a, a-dot as needed by P = p).
template <int p>
__device__ __forceinline__ void write_input(const StepArgs &a, int64_t i, const double (&x)[3],
                                            const double (&v)[3], const double (&ad)[p > 1 ? p - 1 : 1][3])
{
    // FP64 rows: the input of the FP64 form, and of the heavy-body pairs of the precision form
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        a.jrec[(0 + c) * a.ld + i] = x[c];
        a.jrec[(3 + c) * a.ld + i] = v[c];
#pragma unroll
        for (int q = 0; q + 2 <= p; ++q) a.jrec[(6 + 3 * q + c) * a.ld + i] = ad[q][c];
    }
    if (a.precision != MH_PREC_FP64) {
        const double gx = split_grid(__longlong_as_double(a.bound_rd[0]));
        const double gv = split_grid(__longlong_as_double(a.bound_rd[1]));
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float h, l;
            split_hi_lo(x[c], gx, 1.0 / gx, h, l);
            a.jrec32[(0 + c) * a.ld + i] = h;
            a.jrec32[(3 + c) * a.ld + i] = l;
            split_hi_lo(v[c], gv, 1.0 / gv, h, l);
            a.jrec32[(6 + c) * a.ld + i] = h;
            a.jrec32[(9 + c) * a.ld + i] = l;
#pragma unroll
            for (int q = 0; q + 2 <= p; ++q) a.jrec32[(12 + 3 * q + c) * a.ld + i] = (float)ad[q][c];
        }
    }
}

// Raise the grid bounds with this thread's |x|, |v| (every lane of the warp calls it).
__device__ __forceinline__ void track_bounds(const StepArgs &a, bool live, const double (&x)[3],
                                             const double (&v)[3])
{
    if (a.precision == MH_PREC_FP64) return;
    double bx = 0.0, bv = 0.0;
    if (live) {
        bx = fmax(fabs(x[0]), fmax(fabs(x[1]), fabs(x[2])));
        bv = fmax(fabs(v[0]), fmax(fabs(v[1]), fabs(v[2])));
        if (!(bx <= 1e300)) bx = 0.0;      // non-finite values are reported by the flag, not tracked
        if (!(bv <= 1e300)) bv = 0.0;
    }
    raise_bound(a.bound_wr + 0, bx);
    raise_bound(a.bound_wr + 1, bv);
}

template <int p>
__global__ void k_predict(StepArgs a)
{
    constexpr int K = 2 * p;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < a.N;
    const int64_t i = live ? i0 : a.N - 1;      // idle lanes recompute the last body, store nothing
    const double dt = predictor_dt(a);
    if (a.ts.w && i0 == 0)                                // this step's words (other bank than prev)
        for (int k = 0; k < a.ts.n_iter; ++k) a.ts.w[a.ts.bank * kTsMaxIter + k] = 0ull;
    double x[3], v[3], ad[p > 1 ? p - 1 : 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d[K];
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = a.d0[(3 * k + c) * a.ld + i];
        // Horner: x + dt (v + dt (d0/2! + dt (d1/3! + ...)))
        double sx = 0.0, sv = 0.0;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            sx = fma(sx, dt, d[k] * inv_fact(k + 2));
            sv = fma(sv, dt, d[k] * inv_fact(k + 1));
        }
        const double x0 = a.x0[c * a.ld + i], v0 = a.v0[c * a.ld + i];
        x[c] = fma(fma(sx, dt, v0), dt, x0);
        v[c] = fma(sv, dt, v0);
#pragma unroll
        for (int q = 0; q + 2 <= p; ++q) {
            double sa = 0.0;
#pragma unroll
            for (int k = K - 1; k >= q; --k) sa = fma(sa, dt, d[k] * inv_fact(k - q));
            ad[q][c] = sa;
        }
        if (live) {
            a.x1[c * a.ld + i] = x[c];
            a.v1[c * a.ld + i] = v[c];
        }
    }
    track_bounds(a, live, x, v);
    if (live) write_input<p>(a, i, x, v, ad);
}

template <int p, bool kLast>
__global__ void k_correct(StepArgs a)
{
    constexpr int K = 2 * p;
    constexpr int NR = (p + 1) * 3;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < a.N;
    const int64_t i = live ? i0 : a.N - 1;      // idle lanes recompute the last body, store nothing
    const double dt = corrector_dt(a);
    if (kLast && a.ts.t && i0 == 0) *a.ts.t += dt;    // the device clock (read and written by this thread only)
    // time-symmetric steps, all passes but the last: shift of the end time for the next pass
    const double shift = (!kLast && a.ts.w) ? timesym_dt(a, a.ts.pass) - dt : 0.0;
    double x[3], v[3], ad[p > 1 ? p - 1 : 1][3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d1[p + 1], d0[K];
        if (a.split == 1) {
            // one slot (small systems pre-add theirs): straight-line loads that overlap
#pragma unroll
            for (int k = 0; k <= p; ++k) d1[k] = 0.0 + a.part[(int64_t)(3 * k + c) * a.ld + i];
        } else {
#pragma unroll
            for (int k = 0; k <= p; ++k) {
                double s = 0.0;
                for (int q = 0; q < a.split; ++q) s += a.part[((int64_t)q * NR + 3 * k + c) * a.ld + i];
                d1[k] = s;
            }
        }
#pragma unroll
        for (int k = 0; k < K; ++k) d0[k] = a.d0[(3 * k + c) * a.ld + i];
        double xn, vn;
        if (a.comp) {
            // compensated summation of the updates (Section 3.2): the new compensation
            // is committed with the step, every pass starts from the committed one
            double cx = a.comp[c * a.ld + i], cv = a.comp[(3 + c) * a.ld + i];
            correct_comp_kahan<p>(dt, a.beta_mode, d0, d1, a.x0[c * a.ld + i], a.v0[c * a.ld + i], cx, cv, xn, vn);
            if (kLast && live) {
                a.comp[c * a.ld + i] = cx;
                a.comp[(3 + c) * a.ld + i] = cv;
            }
        } else {
            correct_comp<p>(dt, a.beta_mode, d0, d1, a.x0[c * a.ld + i], a.v0[c * a.ld + i], xn, vn);
        }
#pragma unroll
        for (int q = 0; q + 2 <= p; ++q) ad[q][c] = d1[q];
        if (!kLast && a.ts.w) {
            // Taylor series of the end state over the change of dt, with a^(0..p) just evaluated
            double sx = 0.0, sv = 0.0;
#pragma unroll
            for (int k = p; k >= 0; --k) {
                sx = fma(sx, shift, d1[k] * inv_fact(k + 2));
                sv = fma(sv, shift, d1[k] * inv_fact(k + 1));
            }
            xn = fma(fma(sx, shift, vn), shift, xn);
            vn = fma(sv, shift, vn);
#pragma unroll
            for (int q = 0; q + 2 <= p; ++q) {
                double sa = 0.0;
#pragma unroll
                for (int k = p; k >= q; --k) sa = fma(sa, shift, d1[k] * inv_fact(k - q));
                ad[q][c] = sa;
            }
        }
        x[c] = xn;
        v[c] = vn;
        finite = finite && isfinite(xn) && isfinite(vn);
        if (!live) continue;
        if (kLast) {
            a.x0[c * a.ld + i] = xn;
            a.v0[c * a.ld + i] = vn;
            double hi[K > p + 1 ? p - 1 : 1];
            interp_comp<p>(dt, d0, d1, hi);
#pragma unroll
            for (int k = 0; k < K; ++k)
                a.d0[(3 * k + c) * a.ld + i] = k <= p ? d1[k] : hi[k - p - 1];
        }
    }
    if (live && !finite) atomicOr(a.flag, 1);
    if (!kLast) {
        if (a.conv) {
            // convergence of P(EC)^n: largest change of a position component, and the scale
            double dx = 0.0, xm = 0.0;
            if (live)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    dx = fmax(dx, fabs(x[c] - a.x1[c * a.ld + i]));
                    xm = fmax(xm, fabs(x[c]));
                }
            if (!(dx <= 1e300)) dx = 1e300;
            raise_bound(a.conv + 0, dx);
            raise_bound(a.conv + 1, xm);
        }
        if (live)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                a.x1[c * a.ld + i] = x[c];
                a.v1[c * a.ld + i] = v[c];
            }
        track_bounds(a, live, x, v);
        if (live) write_input<p>(a, i, x, v, ad);
    }
}

// ---------------------------------------------------------------------------
// Learned residual on the Taylor predictor (reading R13 of the design notes).
// Frame: e1 = a/|a|, e2 along the part of a-dot normal to a, e3 = e1 x e2.
// Features u_k = R^T F_k / (|a| sigma^k), F_k = h^k a^(k)/k!, then 1 + log10(sigma),
// sigma = max_{1<=k<2p} (|F_k|/|F_0|)^(1/k) (the shortest time scale of the stack, so |u_k| <= 1);
// targets/outputs y = (R^T dx / (|a| h^2 sigma^6), R^T dv / (|a| h sigma^6)).
// ---------------------------------------------------------------------------

constexpr double kSigmaMax = 0.5;

struct Frame {
    double R[3][3];   // R[i][c]: component c of e_i
    double na, sigma;
    bool ok;
};

// Frame and scales of body i from its derivative stack at t0.
template <int p>
__device__ Frame make_frame(const double *d0, int64_t ld, int64_t i, double h)
{
    Frame f{};
    double a[3], j[3];
    for (int c = 0; c < 3; ++c) {
        a[c] = d0[(0 * 3 + c) * ld + i];
        j[c] = d0[(1 * 3 + c) * ld + i];
    }
    f.na = sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
    f.sigma = 0.0;
    if (f.na > 0.0) {
        double hk = h;
#pragma unroll
        for (int k = 1; k < 2 * p; ++k) {
            const double dx = d0[(3 * k) * ld + i], dy = d0[(3 * k + 1) * ld + i], dz = d0[(3 * k + 2) * ld + i];
            const double r = sqrt(dx * dx + dy * dy + dz * dz) * hk * inv_fact(k) / f.na;
            f.sigma = fmax(f.sigma, pow(r, 1.0 / k));
            hk *= h;
        }
    }
    f.ok = f.na > 0.0 && f.sigma > 0.0 && f.sigma <= kSigmaMax;
    if (!f.ok) return f;
    double e1[3] = {a[0] / f.na, a[1] / f.na, a[2] / f.na};
    const double pj = j[0] * e1[0] + j[1] * e1[1] + j[2] * e1[2];
    double u[3] = {j[0] - pj * e1[0], j[1] - pj * e1[1], j[2] - pj * e1[2]};
    double nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    if (!(nu > 1e-300)) {
        const double alt[3] = {fabs(e1[0]) < 0.9 ? 1.0 : 0.0, fabs(e1[0]) < 0.9 ? 0.0 : 1.0, 0.0};
        const double pa = alt[0] * e1[0] + alt[1] * e1[1];
        for (int c = 0; c < 3; ++c) u[c] = alt[c] - pa * e1[c];
        nu = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
    double e2[3] = {u[0] / nu, u[1] / nu, u[2] / nu};
    double e3[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    for (int c = 0; c < 3; ++c) {
        f.R[0][c] = e1[c];
        f.R[1][c] = e2[c];
        f.R[2][c] = e3[c];
    }
    return f;
}

template <int p>
__device__ void write_features(const Frame &f, const double *d0, int64_t ld, int64_t i, double h, float *out)
{
    constexpr int K = 2 * p;
    double hk = 1.0, sk = 1.0;
    for (int k = 0; k < K; ++k) {
        double F[3];
        for (int c = 0; c < 3; ++c) F[c] = d0[(3 * k + c) * ld + i] * hk * inv_fact(k);
        for (int e = 0; e < 3; ++e) {
            const double r = f.R[e][0] * F[0] + f.R[e][1] * F[1] + f.R[e][2] * F[2];
            out[3 * k + e] = f.ok ? (float)(r / (f.na * sk)) : 0.0f;
        }
        hk *= h;
        sk *= f.ok ? f.sigma : 1.0;
    }
    out[3 * K] = f.ok ? (float)(1.0 + log10(f.sigma)) : 0.0f;
}

// Training samples: features at t0 and the scaled converged-minus-predicted residual.
template <int p>
__global__ void k_collect(int64_t N, int64_t ld, double dt, const double *x0s, const double *v0s,
                          const double *d0s, const double *x1, const double *v1, float *feats, float *targ)
{
    constexpr int K = 2 * p;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double h = 0.5 * dt;
    const Frame f = make_frame<p>(d0s, ld, i, h);
    write_features<p>(f, d0s, ld, i, h, feats + i * (3 * K + 1));
    double dx[3], dv[3];
    for (int c = 0; c < 3; ++c) {
        double dk[K], xp, vp, ad[p > 1 ? p - 1 : 1];
        for (int k = 0; k < K; ++k) dk[k] = d0s[(3 * k + c) * ld + i];
        predict_comp<p>(dt, dk, x0s[c * ld + i], v0s[c * ld + i], xp, vp, ad);
        dx[c] = x1[c * ld + i] - xp;
        dv[c] = v1[c * ld + i] - vp;
    }
    double s6 = f.sigma * f.sigma * f.sigma;
    s6 *= s6;
    const double den = f.na * s6;
    for (int e = 0; e < 3; ++e) {
        const double rx = f.R[e][0] * dx[0] + f.R[e][1] * dx[1] + f.R[e][2] * dx[2];
        const double rv = f.R[e][0] * dv[0] + f.R[e][1] * dv[1] + f.R[e][2] * dv[2];
        targ[i * 6 + e] = f.ok ? (float)(rx / (den * h * h)) : 0.0f;
        targ[i * 6 + 3 + e] = f.ok ? (float)(rv / (den * h)) : 0.0f;
    }
}

// Features of every body for the predictor (written to feats [N x 3K]).
template <int p>
__global__ void k_learned_features(int64_t N, int64_t ld, double dt, const double *d0, float *feats)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double h = 0.5 * dt;
    const Frame f = make_frame<p>(d0, ld, i, h);
    write_features<p>(f, d0, ld, i, h, feats + i * (6 * p + 1));
}

// Adds the network's residual to the prediction (bodies whose frame is defined;
// the plain prediction otherwise) and rewrites every evaluation input.  The
// residual (dx, dv) is read as the two next Taylor terms: the derivatives
// a^(2p), a^(2p+1) that produce exactly (dx, dv) at t0 + dt, which then extend
// the predicted a^(q) (q <= p-2) too, so the predicted x, v, a, a-dot stay one
// consistent polynomial.
template <int p>
__global__ void k_learned_apply(StepArgs a, const float *y, float clamp)
{
    constexpr int K = 2 * p;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < a.N;
    const int64_t i = live ? i0 : a.N - 1;
    const double dt = a.dt, h = 0.5 * dt;
    const Frame f = make_frame<p>(a.d0, a.ld, i, h);
    double x[3], v[3], ad[p > 1 ? p - 1 : 1][3];
    for (int c = 0; c < 3; ++c) {
        x[c] = a.jrec[(0 + c) * a.ld + i];
        v[c] = a.jrec[(3 + c) * a.ld + i];
        for (int q = 0; q + 2 <= p; ++q) ad[q][c] = a.jrec[(6 + 3 * q + c) * a.ld + i];
    }
    if (f.ok) {
        double s6 = f.sigma * f.sigma * f.sigma;
        s6 *= s6;
        const double den = f.na * s6;
        double yx[3], yv[3];
        const double cl = (double)clamp;
        for (int e = 0; e < 3; ++e) {
            yx[e] = fmin(fmax((double)y[i * 6 + e], -cl), cl);
            yv[e] = fmin(fmax((double)y[i * 6 + 3 + e], -cl), cl);
        }
        // Taylor weights t_n = dt^n / n! of the two next terms
        double tw[K + 4];
        tw[0] = 1.0;
        for (int n = 1; n < K + 4; ++n) tw[n] = tw[n - 1] * dt / n;
        // dx = t_{K+2} A + t_{K+3} B,  dv = t_{K+1} A + t_{K+2} B
        const double det = tw[K + 2] * tw[K + 2] - tw[K + 3] * tw[K + 1];
        for (int c = 0; c < 3; ++c) {
            const double dx = (f.R[0][c] * yx[0] + f.R[1][c] * yx[1] + f.R[2][c] * yx[2]) * den * h * h;
            const double dv = (f.R[0][c] * yv[0] + f.R[1][c] * yv[1] + f.R[2][c] * yv[2]) * den * h;
            const double A = (dx * tw[K + 2] - dv * tw[K + 3]) / det;
            const double B = (dv * tw[K + 2] - dx * tw[K + 1]) / det;
            x[c] += dx;
            v[c] += dv;
            for (int q = 0; q + 2 <= p; ++q) ad[q][c] += tw[K - q] * A + tw[K + 1 - q] * B;
        }
    }
    if (live)
        for (int c = 0; c < 3; ++c) {
            a.x1[c * a.ld + i] = x[c];
            a.v1[c * a.ld + i] = v[c];
        }
    track_bounds(a, live, x, v);
    if (live) write_input<p>(a, i, x, v, ad);
}

// ---------------------------------------------------------------------------
// Block time steps.  Every body i has a tick T[i] (units of dt_max 2^-k_max)
// and a level (step dt_max 2^-level).  The next block time is the minimum of
// T[i] + 2^(k_max - level[i]); the bodies reaching it form the active list.
// ---------------------------------------------------------------------------

struct BlockArgs {
    long long *T;
    int *level;
    int *act;                   // active list (positions -> bodies)
    unsigned long long *blk;    // [0] next block tick, [1] active count
    int k_max;
    double dt_max, tick, eta;
    long long T_next;           // host copy for the kernels that follow the readback
    int64_t n_act;
    int64_t part_ld;
};

__device__ __forceinline__ double norm3(double a, double b, double c)
{
    // no contraction: the same operation order as a plain C evaluation
    return sqrt(__dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c)));
}

// Aarseth-type estimate dt = eta sqrt((|a||a2| + |a1|^2) / (|a1||a3| + |a2|^2)) and
// the level rule: shrink freely, grow by one level only when T is a multiple of it.
__device__ int block_level(const double (&n)[4], double eta, double dt_max, int k_max, int k_old,
                           long long T)
{
    const double num = __dadd_rn(__dmul_rn(n[0], n[2]), __dmul_rn(n[1], n[1]));
    const double den = __dadd_rn(__dmul_rn(n[1], n[3]), __dmul_rn(n[2], n[2]));
    const double dtc = __dmul_rn(eta, sqrt(__ddiv_rn(num, den)));
    int k = 0;
    while (k < k_max && dt_max * ldexp(1.0, -k) > dtc) ++k;
    if (k_old < 0 || k >= k_old) return k;
    const int kg = k_old - 1;
    const long long span = 1LL << (k_max - kg);
    return (T % span == 0) ? kg : k_old;
}

__global__ void k_block_init_levels(int64_t N, int64_t ld, const double *d0, BlockArgs b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double n[4];
    for (int k = 0; k < 4; ++k)
        n[k] = norm3(d0[(3 * k) * ld + i], d0[(3 * k + 1) * ld + i], d0[(3 * k + 2) * ld + i]);
    b.level[i] = block_level(n, b.eta, b.dt_max, b.k_max, -1, 0);
    b.T[i] = 0;
}

__global__ void k_block_reset(unsigned long long *blk)
{
    blk[0] = ~0ull;
    blk[1] = 0ull;
}

__global__ void k_block_next(int64_t N, BlockArgs b)
{
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long t = ~0ull;
    if (i0 < N) t = (unsigned long long)(b.T[i0] + (1LL << (b.k_max - b.level[i0])));
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long q = __shfl_xor_sync(0xffffffffu, t, o);
        t = q < t ? q : t;
    }
    if ((threadIdx.x & 31) == 0) atomicMin(b.blk, t);
}

__global__ void k_block_active(int64_t N, BlockArgs b)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const unsigned long long tn = b.blk[0];
    if ((unsigned long long)(b.T[i] + (1LL << (b.k_max - b.level[i]))) == tn) {
        const unsigned long long pos = atomicAdd(b.blk + 1, 1ull);
        b.act[pos] = (int)i;
    }
}

// Prediction of every body to the next block time (its own dt).
template <int p>
__global__ void k_block_predict(StepArgs a, BlockArgs b)
{
    constexpr int K = 2 * p;
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < a.N;
    const int64_t i = live ? i0 : a.N - 1;
    const double dt = (double)(b.T_next - b.T[i]) * b.tick;
    double x[3], v[3], ad[p > 1 ? p - 1 : 1][3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d[K];
#pragma unroll
        for (int k = 0; k < K; ++k) d[k] = a.d0[(3 * k + c) * a.ld + i];
        double sx = 0.0, sv = 0.0;
#pragma unroll
        for (int k = K - 1; k >= 0; --k) {
            sx = fma(sx, dt, d[k] * inv_fact(k + 2));
            sv = fma(sv, dt, d[k] * inv_fact(k + 1));
        }
        const double x0 = a.x0[c * a.ld + i], v0 = a.v0[c * a.ld + i];
        x[c] = fma(fma(sx, dt, v0), dt, x0);
        v[c] = fma(sv, dt, v0);
#pragma unroll
        for (int q = 0; q + 2 <= p; ++q) {
            double sa = 0.0;
#pragma unroll
            for (int k = K - 1; k >= q; --k) sa = fma(sa, dt, d[k] * inv_fact(k - q));
            ad[q][c] = sa;
        }
    }
    track_bounds(a, live, x, v);
    if (live) write_input<p>(a, i, x, v, ad);
}

// Correction of the active bodies (position pos -> body act[pos]) with their own dt.
template <int p, bool kLast>
__global__ void k_block_correct(StepArgs a, BlockArgs b)
{
    constexpr int K = 2 * p;
    constexpr int NR = (p + 1) * 3;
    const int64_t pos0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = pos0 < b.n_act;
    const int64_t pos = live ? pos0 : 0;
    const int64_t i = b.act[pos];
    const double dt = (double)(b.T_next - b.T[i]) * b.tick;
    double x[3], v[3], ad[p > 1 ? p - 1 : 1][3];
    double nrm[4][3];
    bool finite = true;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double d1[p + 1], d0[K];
#pragma unroll
        for (int k = 0; k <= p; ++k) {
            double s = 0.0;
            for (int q = 0; q < a.split; ++q) s += a.part[((int64_t)q * NR + 3 * k + c) * b.part_ld + pos];
            d1[k] = s;
        }
#pragma unroll
        for (int k = 0; k < K; ++k) d0[k] = a.d0[(3 * k + c) * a.ld + i];
        double xn, vn;
        correct_comp<p>(dt, a.beta_mode, d0, d1, a.x0[c * a.ld + i], a.v0[c * a.ld + i], xn, vn);
        x[c] = xn;
        v[c] = vn;
#pragma unroll
        for (int q = 0; q + 2 <= p; ++q) ad[q][c] = d1[q];
        finite = finite && isfinite(xn) && isfinite(vn);
        if (kLast) {
            double hi[K > p + 1 ? p - 1 : 1];
            interp_comp<p>(dt, d0, d1, hi);
#pragma unroll
            for (int k = 0; k < 4; ++k) nrm[k][c] = k <= p ? d1[k] : hi[k - p - 1];
            if (live) {
                a.x0[c * a.ld + i] = xn;
                a.v0[c * a.ld + i] = vn;
#pragma unroll
                for (int k = 0; k < K; ++k)
                    a.d0[(3 * k + c) * a.ld + i] = k <= p ? d1[k] : hi[k - p - 1];
            }
        }
    }
    if (live && !finite) atomicOr(a.flag, 1);
    if (kLast) {
        if (live) {
            double n[4];
            for (int k = 0; k < 4; ++k) n[k] = norm3(nrm[k][0], nrm[k][1], nrm[k][2]);
            b.level[i] = block_level(n, b.eta, b.dt_max, b.k_max, b.level[i], b.T_next);
            b.T[i] = b.T_next;
        }
    } else {
        track_bounds(a, live, x, v);
        if (live) write_input<p>(a, i, x, v, ad);
    }
}

// Initialisation pass with P = have+1: rows 3k+c of jrec hold x, v, a^(0..have-1).
__global__ void k_init_rows(int64_t N, int64_t ld, int have, const double *x0, const double *v0,
                            const double *d0, double *jrec)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int c = 0; c < 3; ++c) {
        jrec[(0 + c) * ld + i] = x0[c * ld + i];
        jrec[(3 + c) * ld + i] = v0[c * ld + i];
        for (int k = 0; k < have; ++k) jrec[(6 + 3 * k + c) * ld + i] = d0[(3 * k + c) * ld + i];
    }
}

// Slot 0 of part <- the sum of slots 0 .. split-1, one thread per (row, body), in
// the order the corrector adds them (so the corrector, given split = 1, gives
// the same bits).  For small systems, whose many j-chunk slots would otherwise be
// added serially by one thread per body.
__global__ void k_reduce_slots(int64_t N, int64_t ld, int nr, int split, double *part)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)nr * N) return;
    const int r = (int)(e / N);
    const int64_t i = e - (int64_t)r * N;
    // loads issued in independent batches of 8 (a latency-bound kernel), added in slot order
    double s = 0.0;
    for (int q0 = 0; q0 < split; q0 += 8) {
        double b[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) b[u] = q0 + u < split ? part[((int64_t)(q0 + u) * nr + r) * ld + i] : 0.0;
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (q0 + u < split) s += b[u];
    }
    part[(int64_t)r * ld + i] = s;
}

// Slot 0 <- the sum of `split` slots, one warp per (row, position): lane l adds
// slots l, l + 32, ... in order, then the lanes' sums meet in a fixed tree, so
// the result does not depend on scheduling.  For short active lists with many
// j-chunks, where one thread per (row, position) would add hundreds of slots
// one after another.
__global__ void k_reduce_slots_warp(int64_t n, int64_t ld, int nr, int split, double *part)
{
    const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (e >= (int64_t)nr * n) return;            // whole warps leave together
    const int r = (int)(e / n);
    const int64_t i = e - (int64_t)r * n;
    double s = 0.0;
    for (int q = lane; q < split; q += 32) s += part[((int64_t)q * nr + r) * ld + i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) part[(int64_t)r * ld + i] = s;
}

// Block step evaluated for all bodies (slots by body index, rows of Np): the
// active bodies' sums, out[r][a] = sum over the slots q, in slot order, of
// part[q][r][act[a]], rows of ld_out (the active count padded), one thread per
// (row, active body).
__global__ void k_gather_active(int64_t n_act, int64_t Np, int nr, int split, const double *__restrict__ part,
                                const int *__restrict__ act, int64_t ld_out, double *__restrict__ out)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)nr * n_act) return;
    const int r = (int)(t / n_act);
    const int64_t a = t - (int64_t)r * n_act;
    const int64_t i = act[a];
    double s = 0.0;
    for (int q = 0; q < split; ++q) s += part[((int64_t)q * nr + r) * Np + i];
    out[(int64_t)r * ld_out + a] = s;
}

// d0 rows [lo, hi) <- sum over S partial slots of rows [lo, hi) (slot row count nr).
__global__ void k_init_reduce(int64_t N, int64_t ld, int nr, int lo, int hi, int split,
                              const double *part, double *d0)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    for (int k = lo; k < hi; ++k)
        for (int c = 0; c < 3; ++c) {
            double s = 0.0;
            for (int q = 0; q < split; ++q) s += part[((int64_t)q * nr + 3 * k + c) * ld + i];
            d0[(3 * k + c) * ld + i] = s;
        }
}

// out rows [0, nr) <- sum over S slots (mh_pair_eval's reduction).
__global__ void k_reduce_out(int64_t n, int64_t ld_part, int nr, int split, const double *part,
                             double *out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int r = 0; r < nr; ++r) {
        double s = 0.0;
        for (int q = 0; q < split; ++q) s += part[((int64_t)q * nr + r) * ld_part + i];
        out[r * n + i] = s;
    }
}

// max |x| and max |v| over the bodies of FP64 SoA rows (stride N) into bound[0..1]
// (bound must be zero on entry).
__global__ void k_absmax(int64_t N, const double *traj, unsigned long long *bound)
{
    const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = i0 < N;
    const int64_t i = live ? i0 : 0;
    double bx = 0.0, bv = 0.0;
    for (int c = 0; c < 3; ++c) {
        bx = fmax(bx, fabs(traj[c * N + i]));
        bv = fmax(bv, fabs(traj[(3 + c) * N + i]));
    }
    if (!live || !(bx <= 1e300)) bx = 0.0;
    if (!live || !(bv <= 1e300)) bv = 0.0;
    raise_bound(bound + 0, bx);
    raise_bound(bound + 1, bv);
}

// Precision-form input rows (x hi/lo, v hi/lo, a, a-dot, G m) from FP64 SoA rows
// (stride N) of x, v, a, a-dot, with the hi parts on the grid of bound[0..1].
__global__ void k_split32(int64_t N, int P, const double *traj, const double *m, double G, float *rows,
                          const unsigned long long *bound)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double gx = split_grid(__longlong_as_double(bound[0]));
    const double gv = split_grid(__longlong_as_double(bound[1]));
    for (int c = 0; c < 3; ++c) {
        float h, l;
        split_hi_lo(traj[(0 + c) * N + i], gx, 1.0 / gx, h, l);
        rows[(0 + c) * N + i] = h;
        rows[(3 + c) * N + i] = l;
        split_hi_lo(traj[(3 + c) * N + i], gv, 1.0 / gv, h, l);
        rows[(6 + c) * N + i] = h;
        rows[(9 + c) * N + i] = l;
        for (int q = 0; q + 2 <= P; ++q) rows[(12 + 3 * q + c) * N + i] = (float)traj[(6 + 3 * q + c) * N + i];
    }
    rows[(int64_t)(nf32(P) - 1) * N + i] = (float)(G * m[i]);
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

template <int p>
int launch_step_kernels(const StepArgs &a, int phase, bool last, cudaStream_t st)
{
    // one warp per block for small systems: the FP64 work of a body then spreads
    // over N/32 SMs instead of N/128 (two FP64 lanes per SM)
    const int T = a.N < kSmallN ? 32 : 128;
    const unsigned g = blocks_for(a.N, T);
    if (phase == 0) {
        k_predict<p><<<g, T, 0, st>>>(a);
        MH_LAUNCHED("k_predict");
    } else if (last) {
        k_correct<p, true><<<g, T, 0, st>>>(a);
        MH_LAUNCHED("k_correct(last)");
    } else {
        k_correct<p, false><<<g, T, 0, st>>>(a);
        MH_LAUNCHED("k_correct");
    }
    return MH_OK;
}

}  // namespace

template <int p>
int launch_block_kernels(const StepArgs &a, const BlockArgs &b, int phase, bool last, cudaStream_t st)
{
    const int T = 128;
    if (phase == 0) {
        k_block_predict<p><<<blocks_for(a.N, T), T, 0, st>>>(a, b);
        MH_LAUNCHED("k_block_predict");
    } else if (last) {
        k_block_correct<p, true><<<blocks_for(b.n_act, T), T, 0, st>>>(a, b);
        MH_LAUNCHED("k_block_correct(last)");
    } else {
        k_block_correct<p, false><<<blocks_for(b.n_act, T), T, 0, st>>>(a, b);
        MH_LAUNCHED("k_block_correct");
    }
    return MH_OK;
}

static BlockArgs block_args(const DeviceState &s, const mh_config &cfg, long long T_next, int64_t n_act,
                            int64_t part_ld)
{
    BlockArgs b{s.T, s.level, s.act, s.blk, cfg.k_max, cfg.dt_max, ldexp(cfg.dt_max, -cfg.k_max),
                cfg.eta, T_next, n_act, part_ld};
    return b;
}

int launch_collect(const DeviceState &s, double dt, const double *x0s, const double *v0s, const double *d0s,
                   float *feats, float *targ, cudaStream_t st)
{
    const unsigned g = blocks_for(s.N, 128);
    switch (s.p) {
    case 1: k_collect<1><<<g, 128, 0, st>>>(s.N, s.Np, dt, x0s, v0s, d0s, s.x0, s.v0, feats, targ); break;
    case 2: k_collect<2><<<g, 128, 0, st>>>(s.N, s.Np, dt, x0s, v0s, d0s, s.x0, s.v0, feats, targ); break;
    case 3: k_collect<3><<<g, 128, 0, st>>>(s.N, s.Np, dt, x0s, v0s, d0s, s.x0, s.v0, feats, targ); break;
    }
    MH_LAUNCHED("k_collect");
    return MH_OK;
}

int launch_learned_features(const DeviceState &s, double dt, float *feats, cudaStream_t st)
{
    const unsigned g = blocks_for(s.N, 128);
    switch (s.p) {
    case 1: k_learned_features<1><<<g, 128, 0, st>>>(s.N, s.Np, dt, s.d0, feats); break;
    case 2: k_learned_features<2><<<g, 128, 0, st>>>(s.N, s.Np, dt, s.d0, feats); break;
    case 3: k_learned_features<3><<<g, 128, 0, st>>>(s.N, s.Np, dt, s.d0, feats); break;
    }
    MH_LAUNCHED("k_learned_features");
    return MH_OK;
}

int launch_learned_apply(const DeviceState &s, const mh_config &cfg, double dt, const float *y, float clamp,
                         cudaStream_t st)
{
    StepArgs a{s.N, s.Np, dt, s.m, s.x0, s.v0, s.d0, s.x1, s.v1, s.jrec, s.jrec32, s.part,
               0, cfg.precision, cfg.beta_mode, s.flag,
               s.bound ? s.bound + 2 * s.flip : nullptr, s.bound ? s.bound + 2 * (1 - s.flip) : nullptr};
    const unsigned g = blocks_for(s.N, 128);
    switch (s.p) {
    case 1: k_learned_apply<1><<<g, 128, 0, st>>>(a, y, clamp); break;
    case 2: k_learned_apply<2><<<g, 128, 0, st>>>(a, y, clamp); break;
    case 3: k_learned_apply<3><<<g, 128, 0, st>>>(a, y, clamp); break;
    }
    MH_LAUNCHED("k_learned_apply");
    return MH_OK;
}

int launch_block_init(const DeviceState &s, const mh_config &cfg, cudaStream_t st)
{
    k_block_init_levels<<<blocks_for(s.N, 128), 128, 0, st>>>(s.N, s.Np, s.d0, block_args(s, cfg, 0, 0, s.Np));
    MH_LAUNCHED("k_block_init_levels");
    return MH_OK;
}

int launch_block_schedule(const DeviceState &s, const mh_config &cfg, cudaStream_t st)
{
    const BlockArgs b = block_args(s, cfg, 0, 0, s.Np);
    k_block_reset<<<1, 1, 0, st>>>(s.blk);
    MH_LAUNCHED("k_block_reset");
    k_block_next<<<blocks_for(s.N, 128), 128, 0, st>>>(s.N, b);
    MH_LAUNCHED("k_block_next");
    k_block_active<<<blocks_for(s.N, 128), 128, 0, st>>>(s.N, b);
    MH_LAUNCHED("k_block_active");
    return MH_OK;
}

// phase 0: predict all bodies to T_next; phase 1: correct the active list.
int launch_block_phase(const DeviceState &s, const mh_config &cfg, long long T_next, int64_t n_act,
                       int phase, bool last, int split, cudaStream_t st, int64_t part_ld)
{
    StepArgs a{s.N, s.Np, 0.0, s.m, s.x0, s.v0, s.d0, s.x1, s.v1, s.jrec, s.jrec32, s.part,
               split, cfg.precision, cfg.beta_mode, s.flag,
               s.bound ? s.bound + 2 * s.flip : nullptr, s.bound ? s.bound + 2 * (1 - s.flip) : nullptr};
    const BlockArgs b = block_args(s, cfg, T_next, n_act, part_ld > 0 ? part_ld : s.Np);
    switch (s.p) {
    case 2: return launch_block_kernels<2>(a, b, phase, last, st);
    case 3: return launch_block_kernels<3>(a, b, phase, last, st);
    }
    set_error("block steps need order 6 or 8");
    return MH_EINVAL;
}

// phase 0: predict; phase 1: correct (last = final pass of the step).
int launch_step_phase(const DeviceState &s, const mh_config &cfg, double dt, int phase, bool last,
                      int split, cudaStream_t st, unsigned long long *conv, const TimeSymArgs *ts)
{
    StepArgs a{s.N, s.Np, dt, s.m, s.x0, s.v0, s.d0, s.x1, s.v1, s.jrec, s.jrec32, s.part,
               split, cfg.precision, cfg.beta_mode, s.flag,
               s.bound ? s.bound + 2 * s.flip : nullptr, s.bound ? s.bound + 2 * (1 - s.flip) : nullptr,
               conv};
    if (ts) a.ts = *ts;
    a.comp = s.comp;
    switch (s.p) {
    case 1: return launch_step_kernels<1>(a, phase, last, st);
    case 2: return launch_step_kernels<2>(a, phase, last, st);
    case 3: return launch_step_kernels<3>(a, phase, last, st);
    case 4: return launch_step_kernels<4>(a, phase, last, st);
    case 5: return launch_step_kernels<5>(a, phase, last, st);
    }
    set_error("unsupported p");
    return MH_EINVAL;
}

int launch_init_rows(const DeviceState &s, int have, cudaStream_t st)
{
    k_init_rows<<<blocks_for(s.N, 128), 128, 0, st>>>(s.N, s.Np, have, s.x0, s.v0, s.d0, s.jrec);
    MH_LAUNCHED("k_init_rows");
    return MH_OK;
}

int launch_reduce_slots(const DeviceState &s, int nr, int split, cudaStream_t st)
{
    const int64_t n = (int64_t)nr * s.N;
    k_reduce_slots<<<blocks_for(n, 32), 32, 0, st>>>(s.N, s.Np, nr, split, s.part);
    MH_LAUNCHED("k_reduce_slots");
    return MH_OK;
}

int launch_gather_active(int64_t n_act, int64_t Np, int nr, int split, const double *part, const int *act,
                         int64_t ld_out, double *out, cudaStream_t st)
{
    const int64_t n = (int64_t)nr * n_act;
    k_gather_active<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n_act, Np, nr, split, part, act, ld_out, out);
    MH_LAUNCHED("k_gather_active");
    return MH_OK;
}

int launch_reduce_slots_warp(int64_t n, int64_t ld, int nr, int split, double *part, cudaStream_t st)
{
    const int64_t warps = (int64_t)nr * n;
    k_reduce_slots_warp<<<(unsigned)((warps + 3) / 4), 128, 0, st>>>(n, ld, nr, split, part);
    MH_LAUNCHED("k_reduce_slots_warp");
    return MH_OK;
}

int launch_init_reduce(const DeviceState &s, int nr, int lo, int hi, int split, cudaStream_t st)
{
    k_init_reduce<<<blocks_for(s.N, 128), 128, 0, st>>>(s.N, s.Np, nr, lo, hi, split, s.part, s.d0);
    MH_LAUNCHED("k_init_reduce");
    return MH_OK;
}

int launch_split32(int64_t N, int P, const double *traj, const double *m, double G, float *rows,
                   unsigned long long *bound, cudaStream_t st)
{
    MH_CUDA(cudaMemsetAsync(bound, 0, 2 * sizeof(unsigned long long), st));
    k_absmax<<<blocks_for(N, 128), 128, 0, st>>>(N, traj, bound);
    MH_LAUNCHED("k_absmax");
    k_split32<<<blocks_for(N, 128), 128, 0, st>>>(N, P, traj, m, G, rows, bound);
    MH_LAUNCHED("k_split32");
    return MH_OK;
}

int launch_reduce_out(int64_t n, int64_t ld_part, int nr, int split, const double *part, double *out,
                      cudaStream_t st)
{
    k_reduce_out<<<blocks_for(n, 128), 128, 0, st>>>(n, ld_part, nr, split, part, out);
    MH_LAUNCHED("k_reduce_out");
    return MH_OK;
}

}  // namespace mh
