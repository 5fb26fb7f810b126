/*
 * Plain FP64 CPU oracle for the modified Hermite integrators of Dittmann (2020),
 * "Modified Hermite Integrators of Arbitrary Order", MNRAS.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference
 * that the CUDA path is checked against.  Only the test suite, the smoke check
 * and the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, constant or table with the CUDA library.
 *
 * Every routine follows the paper's steps in the paper's notation:
 *   - scaled stack F, F_n and F+-_n ........................ Section 2, Eqs. 1, 4, 5
 *   - even-column Pascal system A, A_nk = C(2k, n) ......... Section 2, Eq. 8
 *   - velocity / position quadrature with beta ............. Section 2, Eqs. 6, 7
 *   - optimal beta ......................................... Section 2.1, Eq. 20
 *   - Taylor predictor, explicit initial derivatives ........ Section 3 (intro)
 *   - softened pair acceleration ............................ Section 3 (intro)
 *   - P(EC)^n iteration ..................................... Section 2.1 (end), Section 3
 *   - time-step criterion H and the symmetric step .......... Section 3.3, Eq. 24
 *   - Laplace-Runge-Lenz vector ............................. Appendix A, Eq. A1
 *
 * Readings where the paper is silent (listed in the design notes as well):
 *   R1  Taylor predictor depth: x, v and the a-derivatives used by the
 *       evaluation are predicted with every derivative the step holds,
 *       a^(0) .. a^(2p-1).
 *   R2  In evaluation k >= 2 of one step, the relative a and a-dot that enter the
 *       higher pair derivatives come from evaluation k-1 of the same step
 *       (the predicted values in evaluation 1).
 *   R3  a^(p+1) .. a^(2p-1) at the end of a step come from the degree-(2p+1)
 *       Hermite interpolant through a^(0..p) at both ends (Eqs. 2-5), shifted to
 *       t+h with the Pascal matrix (Eq. 3).
 *   R4  Energy uses the softened pair potential -G m_i m_j / sqrt(r^2+eps^2),
 *       the potential whose gradient is the Section 3 pair acceleration.
 *
 * Layout: positions/velocities are N x 3 row-major; a derivative stack holds
 * K vectors per particle, d[(i*K + k)*3 + c] = k-th time derivative of the
 * acceleration of particle i, component c.
 *
 * Compiled with -ffp-contract=off so no fused multiply-adds are formed.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <limits.h>

#define ORC_MAXP 9           /* highest acceleration derivative supported in a pair (a^(9): 12th-order initialisation) */
#define ORC_MAXSYS 8         /* largest Pascal sub-system (p+2 for p <= 6) */

/* ------------------------------------------------------------------------- */
/* small helpers                                                              */
/* ------------------------------------------------------------------------- */

static double binom(int n, int k)
{
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

static double fact(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= (double)i;
    return r;
}

static double dot3(const double *a, const double *b)
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Solve M y = b for an n x n matrix by Gaussian elimination with partial
 * pivoting (M and b are overwritten). */
static void gauss_solve(int n, double M[ORC_MAXSYS][ORC_MAXSYS], double *b)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
            double t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = M[r][c] / M[c][c];
            for (int k = c; k < n; ++k) M[r][k] -= f * M[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int k = r + 1; k < n; ++k) s -= M[r][k] * b[k];
        b[r] = s / M[r][r];
    }
}

/* ------------------------------------------------------------------------- */
/* Section 2: Hermite algebra                                                 */
/* ------------------------------------------------------------------------- */

/* Optimal beta for order 2(p+1) (Section 2.1, Eq. 20):
 *   beta = 1 + (-1)^(p+1) (2p+2)!! / (2p+1)!!                                */
double orc_beta(int p)
{
    double even = 1.0, odd = 1.0;
    for (int k = 2 * p + 2; k > 1; k -= 2) even *= (double)k;
    for (int k = 2 * p + 1; k > 1; k -= 2) odd *= (double)k;
    return 1.0 + ((p + 1) % 2 ? -1.0 : 1.0) * even / odd;
}

/* Quadrature weights on [F+_0, F-_1, F+_2, ...] (length nsys).
 * Eq. 8 gives [F+_0, F-_1, F+_2, ...]^T = A [F_0, F_2, F_4, ...]^T with
 * A_nk = C(2k, n); Eqs. 6/7 integrate with weights 1/(2k+1) on F_2k, the last
 * one multiplied by wlast_scale (beta for the position, Eq. 7).
 * The result c satisfies  Delta/Delta t = sum_n c_n Fpm_n,  i.e. c = w A^-1.
 * Computed by solving A^T c = w. */
static void quad_weights(int nsys, double wlast_scale, double *c)
{
    double M[ORC_MAXSYS][ORC_MAXSYS];
    for (int n = 0; n < nsys; ++n)
        for (int k = 0; k < nsys; ++k)
            M[k][n] = binom(2 * k, n);          /* M = A^T */
    for (int k = 0; k < nsys; ++k) c[k] = 1.0 / (double)(2 * k + 1);
    c[nsys - 1] *= wlast_scale;
    gauss_solve(nsys, M, c);
}

/* Velocity weights (p+1 terms, Eq. 6, f = a) and position weights (p+2 terms,
 * Eq. 7, f = v).  beta_mode 0: the optimal beta of Eq. 20; 1: beta = 1 (the
 * exact-polynomial corrector the paper compares against). */
void orc_corrector_weights(int p, int beta_mode, double *cv, double *cx)
{
    quad_weights(p + 1, 1.0, cv);
    quad_weights(p + 2, beta_mode == 0 ? orc_beta(p) : 1.0, cx);
}

/* Degree-(2p+1) Hermite interpolation of f from f^(0..p) at t-h and t+h,
 * returning f^(n)(t+h) for n = 0 .. nout-1 (R3).
 * Steps: F+-_n (Eq. 5) -> even system A (Eq. 8) for F_0, F_2, ... and the odd
 * analogue A'_nk = C(2k+1, n) on [F-_0, F+_1, F-_2, ...] for F_1, F_3, ...
 * -> Pascal shift F(t+h) = P F(t) (Eq. 3) -> unscale by n!/h^n (Eq. 1).
 * f0, f1: (p+1) x 3 arrays; out: nout x 3.                                  */
void orc_hermite_interp(int p, double dt, const double *f0, const double *f1,
                        int nout, double *out)
{
    const double h = 0.5 * dt;
    const int ns = p + 1;
    for (int c = 0; c < 3; ++c) {
        double Fev[ORC_MAXSYS], Fod[ORC_MAXSYS];
        double Me[ORC_MAXSYS][ORC_MAXSYS], Mo[ORC_MAXSYS][ORC_MAXSYS];
        for (int n = 0; n < ns; ++n) {
            double sc = 0.5 * pow(h, n) / fact(n);
            double plus = sc * (f1[n * 3 + c] + f0[n * 3 + c]);
            double minus = sc * (f1[n * 3 + c] - f0[n * 3 + c]);
            Fev[n] = (n % 2 == 0) ? plus : minus;   /* [F+_0, F-_1, F+_2, ...] */
            Fod[n] = (n % 2 == 0) ? minus : plus;   /* [F-_0, F+_1, F-_2, ...] */
            for (int k = 0; k < ns; ++k) {
                Me[n][k] = binom(2 * k, n);
                Mo[n][k] = binom(2 * k + 1, n);
            }
        }
        gauss_solve(ns, Me, Fev);      /* Fev[k] = F_2k  at the midpoint */
        gauss_solve(ns, Mo, Fod);      /* Fod[k] = F_2k+1 at the midpoint */
        double F[2 * ORC_MAXSYS];
        for (int k = 0; k < ns; ++k) { F[2 * k] = Fev[k]; F[2 * k + 1] = Fod[k]; }
        for (int n = 0; n < nout; ++n) {
            double s = 0.0;
            for (int k = n; k < 2 * ns; ++k) s += binom(k, n) * F[k];
            out[n * 3 + c] = s * fact(n) / pow(h, n);
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Section 3: softened pair acceleration and its time derivatives             */
/* ------------------------------------------------------------------------- */

/* Time derivatives 0..P of a = G m r (r.r + eps^2)^(-3/2) (Section 3, intro)
 * along a trajectory whose relative derivatives are r[k], k = 0..P
 * (r = x_j - x_i, v_j - v_i, a_j - a_i, ...).
 * Generic Leibniz form:
 *   s     = r.r + eps^2,  s^(n) = sum_k C(n,k) r^(k).r^(n-k)
 *   S     = s^(-3/2);     s S' = -(3/2) s' S, differentiated n-1 times
 *   a^(n) = G m sum_k C(n,k) r^(k) S^(n-k)                                   */
void orc_pair_derivs(int P, const double *r, double eps2, double Gm, double *out)
{
    double s[ORC_MAXP + 1], S[ORC_MAXP + 1];
    for (int n = 0; n <= P; ++n) {
        double acc = 0.0;
        for (int k = 0; k <= n; ++k) acc += binom(n, k) * dot3(r + 3 * k, r + 3 * (n - k));
        s[n] = acc;
    }
    s[0] += eps2;
    S[0] = 1.0 / (s[0] * sqrt(s[0]));
    for (int n = 1; n <= P; ++n) {
        double rhs = 0.0;
        for (int k = 0; k <= n - 1; ++k) rhs += binom(n - 1, k) * s[k + 1] * S[n - 1 - k];
        rhs *= -1.5;
        for (int k = 1; k <= n - 1; ++k) rhs -= binom(n - 1, k) * s[k] * S[n - k];
        S[n] = rhs / s[0];
    }
    for (int n = 0; n <= P; ++n)
        for (int c = 0; c < 3; ++c) {
            double acc = 0.0;
            for (int k = 0; k <= n; ++k) acc += binom(n, k) * r[3 * k + c] * S[n - k];
            out[3 * n + c] = Gm * acc;
        }
}

/* Direct summation (the O(N^2) evaluation): for i in [i0, i1),
 *   out_i^(n) = sum_{j != i} pair_derivs(r_ij^(0..P)), n = 0..P.
 * tr: N x (P+1) x 3 trajectory derivatives per particle: x, v, a, a-dot, ...
 * (only tr[.][0..P] used).  out: (i1-i0) x (P+1) x 3.                         */
void orc_evaluate(int N, int P, const double *m, const double *tr, double eps,
                  double G, int i0, int i1, double *out)
{
    const int K = P + 1;
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(static)
    for (int i = i0; i < i1; ++i) {
        double acc[(ORC_MAXP + 1) * 3];
        double r[(ORC_MAXP + 1) * 3], d[(ORC_MAXP + 1) * 3];
        for (int q = 0; q < K * 3; ++q) acc[q] = 0.0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int q = 0; q < K * 3; ++q) r[q] = tr[(size_t)j * K * 3 + q] - tr[(size_t)i * K * 3 + q];
            orc_pair_derivs(P, r, eps2, G * m[j], d);
            for (int q = 0; q < K * 3; ++q) acc[q] += d[q];
        }
        for (int q = 0; q < K * 3; ++q) out[(size_t)(i - i0) * K * 3 + q] = acc[q];
    }
}

/* ------------------------------------------------------------------------- */
/* Section 3 (intro): explicit initial derivatives                            */
/* ------------------------------------------------------------------------- */

/* a^(0) .. a^(2p-1) at t = 0, computed analytically in passes of two orders:
 * pass 1 gives a, a-dot from x, v; pass 2 gives a^(2), a^(3) using everyone's
 * a, a-dot; pass 3 gives a^(4), a^(5) using a^(2), a^(3).  For the 8th-order
 * scheme this reaches the 5th derivative, as Section 3 describes.
 * derivs: N x (2p) x 3 output.                                               */
void orc_initialise(int N, int p, const double *m, const double *x, const double *v,
                    double eps, double G, double *derivs)
{
    const int K = 2 * p;                 /* stored derivatives a^(0..2p-1) */
    const int T = K + 2;                 /* trajectory derivatives x, v, a .. a^(2p-1) */
    double *tr = (double *)calloc((size_t)N * T * 3, sizeof(double));
    double *out = (double *)malloc((size_t)N * T * 3 * sizeof(double));
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) {
            tr[((size_t)i * T + 0) * 3 + c] = x[i * 3 + c];
            tr[((size_t)i * T + 1) * 3 + c] = v[i * 3 + c];
        }
    for (int have = 0; have < K; have += 2) {
        /* known: x, v, a^(0..have-1); compute pair derivatives up to order have+1 */
        const int P = have + 1;
        /* the evaluator wants exactly P+1 trajectory entries per particle */
        double *trP = (double *)malloc((size_t)N * (P + 1) * 3 * sizeof(double));
        for (int i = 0; i < N; ++i)
            memcpy(trP + (size_t)i * (P + 1) * 3, tr + (size_t)i * T * 3, (size_t)(P + 1) * 3 * sizeof(double));
        orc_evaluate(N, P, m, trP, eps, G, 0, N, out);
        for (int i = 0; i < N; ++i)
            for (int n = have; n <= P && n < K; ++n)
                for (int c = 0; c < 3; ++c)
                    tr[((size_t)i * T + 2 + n) * 3 + c] = out[((size_t)i * (P + 1) + n) * 3 + c];
        free(trP);
    }
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c)
                derivs[((size_t)i * K + k) * 3 + c] = tr[((size_t)i * T + 2 + k) * 3 + c];
    free(tr);
    free(out);
}

/* ------------------------------------------------------------------------- */
/* Section 3 (intro): Taylor predictor                                        */
/* ------------------------------------------------------------------------- */

/* Predict particle i by the Taylor series of its trajectory to dt (R1).
 * xp, vp: 3 each; ap: (p-1) x 3 predicted a^(0..p-2) (the relative
 * accelerations the higher pair derivatives need).                          */
static void predict_one(int p, double dt, const double *x, const double *v,
                        const double *d, double *xp, double *vp, double *ap)
{
    const int K = 2 * p;
    for (int c = 0; c < 3; ++c) {
        double sx = x[c] + v[c] * dt, sv = v[c];
        for (int k = 0; k < K; ++k) {
            sx += d[k * 3 + c] * pow(dt, k + 2) / fact(k + 2);
            sv += d[k * 3 + c] * pow(dt, k + 1) / fact(k + 1);
        }
        xp[c] = sx;
        vp[c] = sv;
        for (int q = 0; q + 2 <= p; ++q) {
            double sa = 0.0;
            for (int k = q; k < K; ++k) sa += d[k * 3 + c] * pow(dt, k - q) / fact(k - q);
            ap[q * 3 + c] = sa;
        }
    }
}

void orc_predict(int N, int p, double dt, const double *x, const double *v,
                 const double *derivs, double *xp, double *vp, double *ap)
{
    const int K = 2 * p;
    for (int i = 0; i < N; ++i)
        predict_one(p, dt, x + 3 * i, v + 3 * i, derivs + (size_t)i * K * 3,
                    xp + 3 * i, vp + 3 * i, ap + (size_t)i * (p > 1 ? p - 1 : 1) * 3);
}

/* ------------------------------------------------------------------------- */
/* Section 2 (Eqs. 5-7): the corrector                                        */
/* ------------------------------------------------------------------------- */

/* One correction of particle i.  d0, d1: a^(0..p) at t and t+dt.
 * Velocity first (Eq. 6, f = a), then position (Eq. 7, f = v) with the new
 * v1, as Section 2 prescribes.
 * comp (optional): compensated summation of the updates over the steps
 * (Section 3.2, after Kahan): comp[0..2] and comp[3..5] hold the parts of x and
 * v lost to rounding so far (negated, as Kahan's c); the update y = inc - c is
 * added to x0, and comp_out receives the new c = ((x0 + y) - x0) - y.          */
static void correct_one_c(int p, double dt, const double *cv, const double *cx,
                          const double *x0, const double *v0,
                          const double *d0, const double *d1, double *x1, double *v1,
                          const double *comp, double *comp_out)
{
    const double h = 0.5 * dt;
    for (int c = 0; c < 3; ++c) {
        /* F+-_n of f = a: [F+_0, F-_1, F+_2, ...] */
        double dv = 0.0;
        for (int n = 0; n <= p; ++n) {
            double sc = 0.5 * pow(h, n) / fact(n);
            double fpm = (n % 2 == 0) ? sc * (d1[n * 3 + c] + d0[n * 3 + c])
                                      : sc * (d1[n * 3 + c] - d0[n * 3 + c]);
            dv += cv[n] * fpm;
        }
        if (comp) {
            const double y = dv * dt - comp[3 + c];
            const double t = v0[c] + y;
            comp_out[3 + c] = (t - v0[c]) - y;
            v1[c] = t;
        } else {
            v1[c] = v0[c] + dv * dt;
        }
    }
    for (int c = 0; c < 3; ++c) {
        /* f = v: f^(0) = v, f^(n) = a^(n-1) */
        double dx = 0.0;
        for (int n = 0; n <= p + 1; ++n) {
            double f1 = (n == 0) ? v1[c] : d1[(n - 1) * 3 + c];
            double f0 = (n == 0) ? v0[c] : d0[(n - 1) * 3 + c];
            double sc = 0.5 * pow(h, n) / fact(n);
            double fpm = (n % 2 == 0) ? sc * (f1 + f0) : sc * (f1 - f0);
            dx += cx[n] * fpm;
        }
        if (comp) {
            const double y = dx * dt - comp[c];
            const double t = x0[c] + y;
            comp_out[c] = (t - x0[c]) - y;
            x1[c] = t;
        } else {
            x1[c] = x0[c] + dx * dt;
        }
    }
}

static void correct_one(int p, double dt, const double *cv, const double *cx,
                        const double *x0, const double *v0,
                        const double *d0, const double *d1, double *x1, double *v1)
{
    correct_one_c(p, dt, cv, cx, x0, v0, d0, d1, x1, v1, NULL, NULL);
}

/* ------------------------------------------------------------------------- */
/* One shared P(EC)^n step (Section 2.1 end, Section 3)                       */
/* ------------------------------------------------------------------------- */

double orc_timestep_H(int N, const double *m, const double *x, double eps, double eta, double G);

/* Advance x, v, derivs (N x 2p x 3, a^(0..2p-1)) by one step in place.
 * P: Taylor predictor.  Then n_iter times: E (direct summation of a^(0..p) at
 * the current estimate of t+dt) and C (corrector).  No evaluation follows the
 * last correction; the next step starts from the derivatives of the n-th E.
 * Finally a^(p+1..2p-1) at t+dt by interpolation (R3).
 *
 * Constant step (eta <= 0): dt as given.
 * Time-symmetric variable step (eta > 0, Section 3.3): dt = dir (H- + H+)/2,
 * with dir = +1 or -1 the sign of the dt argument, H- = *H (Eq. 24 at the
 * start of the step) and H+ = Eq. 24 at the positions of the latest
 * evaluation, so that dt is re-chosen as the iteration proceeds (R15):
 *   the prediction uses dt = dir H-;
 *   every pass corrects with the dt its evaluation was made at, so the
 *   derivatives and the end time of each correction agree;
 *   after every pass but the last, dt <- dir (H- + H+)/2 and the corrected
 *   end state (x, v and the a-derivatives the next evaluation takes, R2) is
 *   moved to the new end time by its Taylor series with the derivatives just
 *   evaluated, over the small change of dt.
 * At convergence dt = dir (H(start) + H(end))/2, symmetric in time.  On return
 * *H holds H+ of the last evaluation, the next step's H-.  Returns the dt of
 * the final correction.                                                        */
static double step_impl(int N, int p, int beta_mode, int n_iter, double dt, double eta, double *H,
                        const double *m, double eps, double G, double *x, double *v, double *derivs,
                        double *comp)
{
    const int K = 2 * p;
    const int P = p;                          /* pair derivatives evaluated */
    const int na = (p > 1 ? p - 1 : 1);
    const double dir = dt < 0 ? -1.0 : 1.0;
    double cv[ORC_MAXSYS], cx[ORC_MAXSYS];
    orc_corrector_weights(p, beta_mode, cv, cx);

    double *xp = (double *)malloc((size_t)N * 3 * sizeof(double));
    double *vp = (double *)malloc((size_t)N * 3 * sizeof(double));
    double *ap = (double *)malloc((size_t)N * na * 3 * sizeof(double));
    double *tr = (double *)malloc((size_t)N * (P + 1) * 3 * sizeof(double));
    double *d1 = (double *)malloc((size_t)N * (P + 1) * 3 * sizeof(double));
    double *x1 = (double *)malloc((size_t)N * 3 * sizeof(double));
    double *v1 = (double *)malloc((size_t)N * 3 * sizeof(double));
    double *cnew = comp ? (double *)malloc((size_t)N * 6 * sizeof(double)) : NULL;

    const double H_minus = eta > 0 ? *H : 0.0;
    if (eta > 0) dt = dir * H_minus;
    orc_predict(N, p, dt, x, v, derivs, xp, vp, ap);
    memcpy(x1, xp, (size_t)N * 3 * sizeof(double));
    memcpy(v1, vp, (size_t)N * 3 * sizeof(double));

    for (int it = 0; it < n_iter; ++it) {
        /* evaluation inputs: latest x, v; relative a^(0..P-2) predicted in the
         * first evaluation, else from the previous evaluation (R2) */
        for (int i = 0; i < N; ++i) {
            double *t = tr + (size_t)i * (P + 1) * 3;
            for (int c = 0; c < 3; ++c) { t[c] = x1[i * 3 + c]; t[3 + c] = v1[i * 3 + c]; }
            for (int q = 0; q + 2 <= P; ++q)
                for (int c = 0; c < 3; ++c)
                    t[(q + 2) * 3 + c] = (it == 0) ? ap[((size_t)i * na + q) * 3 + c]
                                                   : d1[((size_t)i * (P + 1) + q) * 3 + c];
        }
        orc_evaluate(N, P, m, tr, eps, G, 0, N, d1);
        double H_plus = 0.0;
        if (eta > 0) {
            /* H+ at the positions just evaluated (x1 before this correction) */
            H_plus = orc_timestep_H(N, m, x1, eps, eta, G);
            *H = H_plus;
        }
        for (int i = 0; i < N; ++i) {
            double d0[(ORC_MAXP + 1) * 3];
            for (int q = 0; q <= P; ++q)
                for (int c = 0; c < 3; ++c) d0[q * 3 + c] = derivs[((size_t)i * K + q) * 3 + c];
            correct_one_c(p, dt, cv, cx, x + 3 * i, v + 3 * i, d0,
                          d1 + (size_t)i * (P + 1) * 3, x1 + 3 * i, v1 + 3 * i,
                          comp ? comp + 6 * i : NULL, comp ? cnew + 6 * i : NULL);
        }
        if (eta > 0 && it < n_iter - 1) {
            const double dt_new = dir * 0.5 * (H_minus + H_plus);
            const double delta = dt_new - dt;
            /* move the end state by delta: x, v and a^(0..P) by their Taylor
             * series with a^(0..P) at the old end time */
            for (int i = 0; i < N; ++i) {
                double *e = d1 + (size_t)i * (P + 1) * 3;
                for (int c = 0; c < 3; ++c) {
                    double a[ORC_MAXP + 1];
                    for (int q = 0; q <= P; ++q) a[q] = e[q * 3 + c];
                    double sx = x1[i * 3 + c] + v1[i * 3 + c] * delta, sv = v1[i * 3 + c];
                    for (int q = 0; q <= P; ++q) {
                        sx += a[q] * pow(delta, q + 2) / fact(q + 2);
                        sv += a[q] * pow(delta, q + 1) / fact(q + 1);
                    }
                    x1[i * 3 + c] = sx;
                    v1[i * 3 + c] = sv;
                    for (int q = 0; q <= P; ++q) {
                        double sq = 0.0;
                        for (int j = q; j <= P; ++j) sq += a[j] * pow(delta, j - q) / fact(j - q);
                        e[q * 3 + c] = sq;
                    }
                }
            }
            dt = dt_new;
        }
    }

    for (int i = 0; i < N; ++i) {
        double d0[(ORC_MAXP + 1) * 3], hi[2 * ORC_MAXSYS * 3];
        const double *e1 = d1 + (size_t)i * (P + 1) * 3;
        for (int q = 0; q <= P; ++q)
            for (int c = 0; c < 3; ++c) d0[q * 3 + c] = derivs[((size_t)i * K + q) * 3 + c];
        if (K > P + 1) orc_hermite_interp(p, dt, d0, e1, K, hi);
        for (int q = 0; q < K; ++q)
            for (int c = 0; c < 3; ++c)
                derivs[((size_t)i * K + q) * 3 + c] = (q <= P) ? e1[q * 3 + c] : hi[q * 3 + c];
        for (int c = 0; c < 3; ++c) { x[i * 3 + c] = x1[i * 3 + c]; v[i * 3 + c] = v1[i * 3 + c]; }
    }
    if (comp) memcpy(comp, cnew, (size_t)N * 6 * sizeof(double));   /* the committed step's compensation */
    free(xp); free(vp); free(ap); free(tr); free(d1); free(x1); free(v1); free(cnew);
    return dt;
}

/* One shared P(EC)^n step of constant dt (Section 2.1 end, Section 3). */
void orc_step(int N, int p, int beta_mode, int n_iter, double dt, const double *m,
              double eps, double G, double *x, double *v, double *derivs)
{
    step_impl(N, p, beta_mode, n_iter, dt, 0.0, NULL, m, eps, G, x, v, derivs, NULL);
}

/* nsteps constant steps with compensated summation of the x, v updates
 * (Section 3.2); comp: N x 6 carried compensation (zero at the start). */
void orc_run_comp(int N, int p, int beta_mode, int n_iter, double dt, int nsteps,
                  const double *m, double eps, double G, double *x, double *v, double *derivs,
                  double *comp)
{
    for (int s = 0; s < nsteps; ++s)
        step_impl(N, p, beta_mode, n_iter, dt, 0.0, NULL, m, eps, G, x, v, derivs, comp);
}

/* nsteps time-symmetric variable steps (Section 3.3) forward (dir > 0) or
 * backward (dir < 0).  *H: in, Eq. 24 at the start; out, the next step's H-.
 * dts (may be NULL): the nsteps step sizes taken.  Returns the time advanced. */
double orc_run_timesym(int N, int p, int beta_mode, int n_iter, int dir, double eta, int nsteps,
                       const double *m, double eps, double G, double *x, double *v, double *derivs,
                       double *H, double *dts)
{
    double t = 0.0;
    for (int s = 0; s < nsteps; ++s) {
        const double dt = step_impl(N, p, beta_mode, n_iter, dir < 0 ? -1.0 : 1.0, eta, H, m, eps, G,
                                    x, v, derivs, NULL);
        if (dts) dts[s] = dt;
        t += dt;
    }
    return t;
}

/* Corrector alone for N particles (exposed for tests): d0, d1 are N x (p+1) x 3. */
void orc_correct(int N, int p, int beta_mode, double dt, const double *x0, const double *v0,
                 const double *d0, const double *d1, double *x1, double *v1)
{
    double cv[ORC_MAXSYS], cx[ORC_MAXSYS];
    orc_corrector_weights(p, beta_mode, cv, cx);
    for (int i = 0; i < N; ++i)
        correct_one(p, dt, cv, cx, x0 + 3 * i, v0 + 3 * i, d0 + (size_t)i * (p + 1) * 3,
                    d1 + (size_t)i * (p + 1) * 3, x1 + 3 * i, v1 + 3 * i);
}

/* nsteps shared steps of constant dt. */
void orc_run(int N, int p, int beta_mode, int n_iter, double dt, int nsteps,
             const double *m, double eps, double G, double *x, double *v, double *derivs)
{
    for (int s = 0; s < nsteps; ++s)
        orc_step(N, p, beta_mode, n_iter, dt, m, eps, G, x, v, derivs);
}

/* ------------------------------------------------------------------------- */
/* Diagnostics: energy and Laplace-Runge-Lenz / eccentricity vectors          */
/* ------------------------------------------------------------------------- */

/* E = sum_i m_i |v_i|^2 / 2 - sum_{i<j} G m_i m_j / sqrt(r_ij^2 + eps^2)  (R4) */
double orc_energy(int N, const double *m, const double *x, const double *v,
                  double eps, double G)
{
    double kin = 0.0, pot = 0.0;
    for (int i = 0; i < N; ++i) kin += 0.5 * m[i] * dot3(v + 3 * i, v + 3 * i);
    for (int i = 0; i < N; ++i) {
        double pi = 0.0;
        for (int j = i + 1; j < N; ++j) {
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            pi += m[j] / sqrt(dot3(d, d) + eps * eps);
        }
        pot += G * m[i] * pi;
    }
    return kin - pot;
}

/* Eccentricity vector of each body about the central body (Appendix A, Eq. A1):
 *   mu e = (|v|^2 - mu/|r|) r - (r.v) v,  r, v relative to the central body,
 *   mu = G (m_c + m_i).  The central body's own entry is set to zero.        */
void orc_ecc(int N, const double *m, const double *x, const double *v, double G,
             int central, double *e)
{
    for (int i = 0; i < N; ++i) {
        if (i == central) { e[3 * i] = e[3 * i + 1] = e[3 * i + 2] = 0.0; continue; }
        double r[3], u[3];
        for (int c = 0; c < 3; ++c) {
            r[c] = x[3 * i + c] - x[3 * central + c];
            u[c] = v[3 * i + c] - v[3 * central + c];
        }
        double mu = G * (m[central] + m[i]);
        double rn = sqrt(dot3(r, r)), v2 = dot3(u, u), rv = dot3(r, u);
        for (int c = 0; c < 3; ++c) e[3 * i + c] = ((v2 - mu / rn) * r[c] - rv * u[c]) / mu;
    }
}

/* ------------------------------------------------------------------------- */
/* Section 3.3: time-step criterion                                           */
/* ------------------------------------------------------------------------- */

/* H = eta min_{i != j} ((r_ij^2 + eps^2)^(3/2) / (G (m_i + m_j)))^(1/2)  (Eq. 24,
 * written there for G = 1: the two-body Kepler time scale of the closest pair) */
double orc_timestep_H(int N, const double *m, const double *x, double eps, double eta, double G)
{
    double best = INFINITY;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            double d[3] = {x[3 * j] - x[3 * i], x[3 * j + 1] - x[3 * i + 1], x[3 * j + 2] - x[3 * i + 2]};
            double s = dot3(d, d) + eps * eps;
            double q = sqrt(s * sqrt(s) / (G * (m[i] + m[j])));   /* (s^(3/2) / G M)^(1/2) */
            if (q < best) best = q;
        }
    return eta * best;
}

/* ------------------------------------------------------------------------- */
/* Block time steps (Section 4 names the option; the scheme below is the     */
/* reading recorded in the design notes, R12)                                 */
/* ------------------------------------------------------------------------- */

/* Aarseth-type step estimate from a, a-dot, a^(2), a^(3) of one body:
 *   dt = eta sqrt((|a||a2| + |a1|^2) / (|a1||a3| + |a2|^2)).                 */
double orc_aarseth_dt(const double *d, double eta)
{
    const double a0 = sqrt(dot3(d, d)), a1 = sqrt(dot3(d + 3, d + 3));
    const double a2 = sqrt(dot3(d + 6, d + 6)), a3 = sqrt(dot3(d + 9, d + 9));
    return eta * sqrt((a0 * a2 + a1 * a1) / (a1 * a3 + a2 * a2));
}

/* Level for a body with estimate dt_c: the smallest k in [0, k_max] with
 * dt_max 2^-k <= dt_c (k_max if none).  From level k_old at tick T (ticks of
 * dt_max 2^-k_max) the step may shrink freely but grows by at most one level,
 * and only when T is a multiple of the grown step.  k_old < 0: no constraint. */
int orc_block_level(double dt_c, double dt_max, int k_max, int k_old, long long T)
{
    int k = 0;
    while (k < k_max && dt_max * ldexp(1.0, -k) > dt_c) ++k;
    if (k_old < 0 || k >= k_old) return k;
    const int kg = k_old - 1;                      /* grow by one level at most */
    const long long span = 1LL << (k_max - kg);
    return (T % span == 0) ? kg : k_old;
}

/* Initial levels at T = 0 from the initial derivatives (N x K x 3, K = 2p >= 4). */
void orc_block_init_levels(int N, int p, const double *derivs, double eta, double dt_max,
                           int k_max, int *level)
{
    const int K = 2 * p;
    for (int i = 0; i < N; ++i)
        level[i] = orc_block_level(orc_aarseth_dt(derivs + (size_t)i * K * 3, eta), dt_max, k_max, -1, 0);
}

/* One block step (p >= 2).  Every body i lives at its own tick T[i] with level
 * level[i] (step dt_max 2^-level).  The next block time is
 * T_next = min_i (T[i] + 2^(k_max - level[i])); the bodies reaching it are
 * active.  All bodies are predicted to T_next by their Taylor series; the
 * active ones then take n_iter evaluate-correct passes with their own step
 * (inactive sources keep their predicted values, active sources their latest
 * corrected x, v and, from the second pass on, the a, a-dot of the previous
 * evaluation), followed by the interpolation of their higher derivatives, the
 * commit T[i] = T_next and a new level.  Returns the number of active bodies;
 * *T_out receives T_next.                                                    */
int orc_block_step(int N, int p, int beta_mode, int n_iter, double dt_max, int k_max,
                   double eta, const double *m, double eps, double G, double *x, double *v,
                   double *derivs, long long *T, int *level, long long *T_out)
{
    const int K = 2 * p;
    const int P = p;
    const int na = p - 1;
    const double tick = dt_max * ldexp(1.0, -k_max);
    double cv[ORC_MAXSYS], cx[ORC_MAXSYS];
    orc_corrector_weights(p, beta_mode, cv, cx);

    long long Tn = LLONG_MAX;
    for (int i = 0; i < N; ++i) {
        const long long t = T[i] + (1LL << (k_max - level[i]));
        if (t < Tn) Tn = t;
    }
    int *act = (int *)malloc((size_t)N * sizeof(int));
    int n_act = 0;
    for (int i = 0; i < N; ++i)
        if (T[i] + (1LL << (k_max - level[i])) == Tn) act[n_act++] = i;

    /* prediction of every body to T_next */
    double *tr = (double *)malloc((size_t)N * (P + 1) * 3 * sizeof(double));
    double *ap = (double *)malloc((size_t)(na > 0 ? na : 1) * 3 * sizeof(double));
    for (int i = 0; i < N; ++i) {
        double *t = tr + (size_t)i * (P + 1) * 3;
        predict_one(p, (double)(Tn - T[i]) * tick, x + 3 * i, v + 3 * i, derivs + (size_t)i * K * 3,
                    t, t + 3, ap);
        for (int q = 0; q < na; ++q)
            for (int c = 0; c < 3; ++c) t[(q + 2) * 3 + c] = ap[q * 3 + c];
    }
    double *d1 = (double *)malloc((size_t)n_act * (P + 1) * 3 * sizeof(double));
    double *one = (double *)malloc((size_t)(P + 1) * 3 * sizeof(double));
    double *x1 = (double *)malloc((size_t)n_act * 3 * sizeof(double));
    double *v1 = (double *)malloc((size_t)n_act * 3 * sizeof(double));
    for (int it = 0; it < n_iter; ++it) {
        for (int q = 0; q < n_act; ++q) {
            orc_evaluate(N, P, m, tr, eps, G, act[q], act[q] + 1, one);
            memcpy(d1 + (size_t)q * (P + 1) * 3, one, (size_t)(P + 1) * 3 * sizeof(double));
        }
        for (int q = 0; q < n_act; ++q) {
            const int i = act[q];
            const double dt = (double)(Tn - T[i]) * tick;
            double d0[(ORC_MAXP + 1) * 3];
            for (int k = 0; k <= P; ++k)
                for (int c = 0; c < 3; ++c) d0[k * 3 + c] = derivs[((size_t)i * K + k) * 3 + c];
            correct_one(p, dt, cv, cx, x + 3 * i, v + 3 * i, d0, d1 + (size_t)q * (P + 1) * 3,
                        x1 + 3 * q, v1 + 3 * q);
        }
        /* the active bodies' new estimates become the evaluation inputs (R2) */
        for (int q = 0; q < n_act; ++q) {
            double *t = tr + (size_t)act[q] * (P + 1) * 3;
            for (int c = 0; c < 3; ++c) { t[c] = x1[q * 3 + c]; t[3 + c] = v1[q * 3 + c]; }
            for (int k = 0; k + 2 <= P; ++k)
                for (int c = 0; c < 3; ++c) t[(k + 2) * 3 + c] = d1[((size_t)q * (P + 1) + k) * 3 + c];
        }
    }
    for (int q = 0; q < n_act; ++q) {
        const int i = act[q];
        const double dt = (double)(Tn - T[i]) * tick;
        double d0[(ORC_MAXP + 1) * 3], hi[2 * ORC_MAXSYS * 3];
        const double *e1 = d1 + (size_t)q * (P + 1) * 3;
        for (int k = 0; k <= P; ++k)
            for (int c = 0; c < 3; ++c) d0[k * 3 + c] = derivs[((size_t)i * K + k) * 3 + c];
        orc_hermite_interp(p, dt, d0, e1, K, hi);
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c)
                derivs[((size_t)i * K + k) * 3 + c] = (k <= P) ? e1[k * 3 + c] : hi[k * 3 + c];
        for (int c = 0; c < 3; ++c) { x[3 * i + c] = x1[q * 3 + c]; v[3 * i + c] = v1[q * 3 + c]; }
        T[i] = Tn;
        level[i] = orc_block_level(orc_aarseth_dt(derivs + (size_t)i * K * 3, eta), dt_max, k_max,
                                   level[i], Tn);
    }
    free(act); free(tr); free(ap); free(d1); free(one); free(x1); free(v1);
    *T_out = Tn;
    return n_act;
}
