/*
 * Binary128 CPU oracle for the double-double form of the modified Hermite
 * integrators of Dittmann (2020), "Modified Hermite Integrators of Arbitrary
 * Order", MNRAS.
 *
 * TEST INFRASTRUCTURE ONLY.  It is the reference that the CUDA double-double
 * path is checked against; only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * constant or table with the CUDA library.
 *
 * The steps are those of the FP64 oracle (mh_oracle.c), in the paper's order
 * and notation, with every operation in IEEE binary128 (_Float128: 113-bit
 * significand, unit roundoff 2^-113 ~ 1e-34), so that a double-double
 * implementation (106 bits, unit roundoff ~2^-104 per operation) can be
 * checked down to its own rounding level:
 *   - scaled stack F+-_n and the even-column Pascal system A ...... Section 2, Eqs. 4, 5, 8
 *   - velocity / position quadrature with beta .................... Section 2, Eqs. 6, 7
 *   - optimal beta ................................................ Section 2.1, Eq. 20
 *   - softened pair acceleration and its time derivatives ......... Section 3 (intro)
 *   - explicit initial derivatives, Taylor predictor .............. Section 3 (intro)
 *   - P(EC)^n with constant shared steps .......................... Section 2.1 (end), Section 3
 *   - energy, Laplace-Runge-Lenz vectors .......................... Appendix A, Eq. A1
 * with the readings R1-R4 of mh_oracle.c (predictor depth, relative a of the
 * previous evaluation, end-of-step Hermite interpolation, softened potential).
 *
 * Boundary: every real value crosses as a double-double pair (hi, lo) stored
 * consecutively (value = hi + lo): vectors are N x 3 x 2, derivative stacks
 * N x K x 3 x 2.  On entry hi + lo is formed in binary128 (exact for the pairs
 * the tests pass: doubles, and pairs rounded from binary128); on exit a value q
 * is returned as hi = RN(q), lo = RN(q - hi).  Masses, eps, G and dt are doubles
 * and enter exactly.
 *
 * Compiled with -ffp-contract=off.
 */
#define __STDC_WANT_IEC_60559_TYPES_EXT__ 1
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef _Float128 Q;

#define ORQ_MAXP 9           /* highest acceleration derivative in a pair (12th-order initialisation) */
#define ORQ_MAXSYS 8         /* largest Pascal sub-system */

/* ------------------------------------------------------------------------- */
/* helpers                                                                    */
/* ------------------------------------------------------------------------- */

static Q q_in(const double *p) { return (Q)p[0] + (Q)p[1]; }

static void q_out(Q q, double *p)
{
    const double h = (double)q;
    p[0] = h;
    p[1] = (double)(q - (Q)h);
}

static Q qbinom(int n, int k)
{
    if (k < 0 || k > n) return 0;
    Q r = 1;
    for (int i = 1; i <= k; ++i) r = r * (Q)(n - k + i) / (Q)i;   /* exact: every partial product is an integer */
    return r;
}

static Q qfact(int n)
{
    Q r = 1;
    for (int i = 2; i <= n; ++i) r *= (Q)i;
    return r;
}

static Q qpow(Q x, int n)
{
    Q r = 1;
    for (int i = 0; i < n; ++i) r *= x;
    return r;
}

static Q qdot3(const Q *a, const Q *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static Q qabs(Q x) { return x < 0 ? -x : x; }

/* M y = b by Gaussian elimination with partial pivoting (M, b overwritten). */
static void qgauss(int n, Q M[ORQ_MAXSYS][ORQ_MAXSYS], Q *b)
{
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (qabs(M[r][c]) > qabs(M[piv][c])) piv = r;
        if (piv != c) {
            for (int k = 0; k < n; ++k) { Q t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
            Q t = b[c]; b[c] = b[piv]; b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            Q f = M[r][c] / M[c][c];
            for (int k = c; k < n; ++k) M[r][k] -= f * M[c][k];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        Q s = b[r];
        for (int k = r + 1; k < n; ++k) s -= M[r][k] * b[k];
        b[r] = s / M[r][r];
    }
}

/* ------------------------------------------------------------------------- */
/* Section 2: Hermite algebra                                                 */
/* ------------------------------------------------------------------------- */

/* Eq. 20: beta = 1 + (-1)^(p+1) (2p+2)!! / (2p+1)!! */
static Q qbeta(int p)
{
    Q even = 1, odd = 1;
    for (int k = 2 * p + 2; k > 1; k -= 2) even *= (Q)k;
    for (int k = 2 * p + 1; k > 1; k -= 2) odd *= (Q)k;
    return 1 + ((p + 1) % 2 ? (Q)-1 : (Q)1) * even / odd;
}

/* Weights c on [F+_0, F-_1, F+_2, ...] with Delta/Delta t = sum_n c_n Fpm_n:
 * Eq. 8 writes the F+- vector as A [F_0, F_2, ...] with A_nk = C(2k, n), and
 * Eqs. 6/7 weight F_2k by 1/(2k+1), the last weight times wlast (beta in Eq. 7),
 * so c solves A^T c = w. */
static void qquad_weights(int nsys, Q wlast, Q *c)
{
    Q M[ORQ_MAXSYS][ORQ_MAXSYS];
    for (int n = 0; n < nsys; ++n)
        for (int k = 0; k < nsys; ++k) M[k][n] = qbinom(2 * k, n);
    for (int k = 0; k < nsys; ++k) c[k] = (Q)1 / (Q)(2 * k + 1);
    c[nsys - 1] *= wlast;
    qgauss(nsys, M, c);
}

static void qcorrector_weights(int p, int beta_mode, Q *cv, Q *cx)
{
    qquad_weights(p + 1, 1, cv);
    qquad_weights(p + 2, beta_mode == 0 ? qbeta(p) : (Q)1, cx);
}

/* cv: p+1 pairs, cx: p+2 pairs (the velocity and position weights of Eqs. 6, 7). */
void orq_corrector_weights(int p, int beta_mode, double *cv2, double *cx2)
{
    Q cv[ORQ_MAXSYS], cx[ORQ_MAXSYS];
    qcorrector_weights(p, beta_mode, cv, cx);
    for (int k = 0; k <= p; ++k) q_out(cv[k], cv2 + 2 * k);
    for (int k = 0; k <= p + 1; ++k) q_out(cx[k], cx2 + 2 * k);
}

/* f^(n)(t+h), n < nout, of the degree-(2p+1) Hermite interpolant through
 * f^(0..p) at t-h and t+h (R3): F+-_n (Eq. 5), the even system A (Eq. 8) for
 * F_0, F_2, ..., its odd analogue A'_nk = C(2k+1, n) on [F-_0, F+_1, ...] for
 * F_1, F_3, ..., the Pascal shift to t+h (Eq. 3), unscaled by n!/h^n (Eq. 1).
 * f0, f1: (p+1) x 3; out: nout x 3. */
static void qhermite_interp(int p, Q dt, const Q *f0, const Q *f1, int nout, Q *out)
{
    const Q h = dt / 2;
    const int ns = p + 1;
    for (int c = 0; c < 3; ++c) {
        Q Fev[ORQ_MAXSYS], Fod[ORQ_MAXSYS];
        Q Me[ORQ_MAXSYS][ORQ_MAXSYS], Mo[ORQ_MAXSYS][ORQ_MAXSYS];
        for (int n = 0; n < ns; ++n) {
            const Q sc = qpow(h, n) / (2 * qfact(n));
            const Q plus = sc * (f1[n * 3 + c] + f0[n * 3 + c]);
            const Q minus = sc * (f1[n * 3 + c] - f0[n * 3 + c]);
            Fev[n] = (n % 2 == 0) ? plus : minus;
            Fod[n] = (n % 2 == 0) ? minus : plus;
            for (int k = 0; k < ns; ++k) {
                Me[n][k] = qbinom(2 * k, n);
                Mo[n][k] = qbinom(2 * k + 1, n);
            }
        }
        qgauss(ns, Me, Fev);
        qgauss(ns, Mo, Fod);
        Q F[2 * ORQ_MAXSYS];
        for (int k = 0; k < ns; ++k) { F[2 * k] = Fev[k]; F[2 * k + 1] = Fod[k]; }
        for (int n = 0; n < nout; ++n) {
            Q s = 0;
            for (int k = n; k < 2 * ns; ++k) s += qbinom(k, n) * F[k];
            out[n * 3 + c] = s * qfact(n) / qpow(h, n);
        }
    }
}

void orq_hermite_interp(int p, double dt, const double *f0_2, const double *f1_2, int nout, double *out2)
{
    Q f0[(ORQ_MAXSYS) * 3], f1[(ORQ_MAXSYS) * 3], out[2 * ORQ_MAXSYS * 3];
    for (int q = 0; q < (p + 1) * 3; ++q) { f0[q] = q_in(f0_2 + 2 * q); f1[q] = q_in(f1_2 + 2 * q); }
    qhermite_interp(p, (Q)dt, f0, f1, nout, out);
    for (int q = 0; q < nout * 3; ++q) q_out(out[q], out2 + 2 * q);
}

/* ------------------------------------------------------------------------- */
/* Section 3: pair derivatives, direct summation, initialisation, predictor   */
/* ------------------------------------------------------------------------- */

/* a^(n), n = 0..P, of a = G m r (r.r + eps^2)^(-3/2) along the relative
 * trajectory r[k] (Leibniz form: s^(n) = sum_k C(n,k) r^(k).r^(n-k);
 * S = s^(-3/2) from s S' = -(3/2) s' S differentiated n-1 times;
 * a^(n) = G m sum_k C(n,k) r^(k) S^(n-k)). */
static void qpair_derivs(int P, const Q *r, Q eps2, Q Gm, Q *out)
{
    Q s[ORQ_MAXP + 1], S[ORQ_MAXP + 1];
    for (int n = 0; n <= P; ++n) {
        Q acc = 0;
        for (int k = 0; k <= n; ++k) acc += qbinom(n, k) * qdot3(r + 3 * k, r + 3 * (n - k));
        s[n] = acc;
    }
    s[0] += eps2;
    S[0] = 1 / (s[0] * sqrtf128(s[0]));
    for (int n = 1; n <= P; ++n) {
        Q rhs = 0;
        for (int k = 0; k <= n - 1; ++k) rhs += qbinom(n - 1, k) * s[k + 1] * S[n - 1 - k];
        rhs *= (Q)-1.5;
        for (int k = 1; k <= n - 1; ++k) rhs -= qbinom(n - 1, k) * s[k] * S[n - k];
        S[n] = rhs / s[0];
    }
    for (int n = 0; n <= P; ++n)
        for (int c = 0; c < 3; ++c) {
            Q acc = 0;
            for (int k = 0; k <= n; ++k) acc += qbinom(n, k) * r[3 * k + c] * S[n - k];
            out[3 * n + c] = Gm * acc;
        }
}

/* out_i^(n) = sum_{j != i} pair derivatives, i = 0..N-1; tr: N x (P+1) x 3. */
static void qevaluate(int N, int P, const double *m, const Q *tr, Q eps2, Q G, Q *out)
{
    const int K = P + 1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < N; ++i) {
        Q acc[(ORQ_MAXP + 1) * 3], r[(ORQ_MAXP + 1) * 3], d[(ORQ_MAXP + 1) * 3];
        for (int q = 0; q < K * 3; ++q) acc[q] = 0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int q = 0; q < K * 3; ++q) r[q] = tr[(size_t)j * K * 3 + q] - tr[(size_t)i * K * 3 + q];
            qpair_derivs(P, r, eps2, G * (Q)m[j], d);
            for (int q = 0; q < K * 3; ++q) acc[q] += d[q];
        }
        for (int q = 0; q < K * 3; ++q) out[(size_t)i * K * 3 + q] = acc[q];
    }
}

/* out_i^(n) = sum_{j != i} pair derivatives for i in [i0, i1) only (sampled
 * checks at sizes where every i would be too slow).  tr2: N x (P+1) x 3 x 2
 * trajectory pairs; out2: (i1-i0) x (P+1) x 3 x 2. */
void orq_evaluate(int N, int P, const double *m, const double *tr2, double eps, double G, int i0, int i1,
                  double *out2)
{
    const int K = P + 1;
    Q *tr = (Q *)malloc((size_t)N * K * 3 * sizeof(Q));
    for (size_t q = 0; q < (size_t)N * K * 3; ++q) tr[q] = q_in(tr2 + 2 * q);
    const Q eps2 = (Q)eps * (Q)eps;
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = i0; i < i1; ++i) {
        Q acc[(ORQ_MAXP + 1) * 3], r[(ORQ_MAXP + 1) * 3], d[(ORQ_MAXP + 1) * 3];
        for (int q = 0; q < K * 3; ++q) acc[q] = 0;
        for (int j = 0; j < N; ++j) {
            if (j == i) continue;
            for (int q = 0; q < K * 3; ++q) r[q] = tr[(size_t)j * K * 3 + q] - tr[(size_t)i * K * 3 + q];
            qpair_derivs(P, r, eps2, (Q)G * (Q)m[j], d);
            for (int q = 0; q < K * 3; ++q) acc[q] += d[q];
        }
        for (int q = 0; q < K * 3; ++q) q_out(acc[q], out2 + 2 * ((size_t)(i - i0) * K * 3 + q));
    }
    free(tr);
}

/* a^(0..2p-1) at the start from x, v in passes of two orders (Section 3 intro). */
static void qinitialise(int N, int p, const double *m, const Q *x, const Q *v, Q eps2, Q G, Q *derivs)
{
    const int K = 2 * p, T = K + 2;
    Q *tr = (Q *)calloc((size_t)N * T * 3, sizeof(Q));
    Q *trP = (Q *)malloc((size_t)N * T * 3 * sizeof(Q));
    Q *out = (Q *)malloc((size_t)N * T * 3 * sizeof(Q));
    for (int i = 0; i < N; ++i)
        for (int c = 0; c < 3; ++c) {
            tr[((size_t)i * T + 0) * 3 + c] = x[i * 3 + c];
            tr[((size_t)i * T + 1) * 3 + c] = v[i * 3 + c];
        }
    for (int have = 0; have < K; have += 2) {
        const int P = have + 1;
        for (int i = 0; i < N; ++i)
            memcpy(trP + (size_t)i * (P + 1) * 3, tr + (size_t)i * T * 3, (size_t)(P + 1) * 3 * sizeof(Q));
        qevaluate(N, P, m, trP, eps2, G, out);
        for (int i = 0; i < N; ++i)
            for (int n = have; n <= P && n < K; ++n)
                for (int c = 0; c < 3; ++c)
                    tr[((size_t)i * T + 2 + n) * 3 + c] = out[((size_t)i * (P + 1) + n) * 3 + c];
    }
    for (int i = 0; i < N; ++i)
        for (int k = 0; k < K; ++k)
            for (int c = 0; c < 3; ++c)
                derivs[((size_t)i * K + k) * 3 + c] = tr[((size_t)i * T + 2 + k) * 3 + c];
    free(tr); free(trP); free(out);
}

/* Taylor predictor of one body to dt (R1): x, v and a^(0..p-2). */
static void qpredict_one(int p, Q dt, const Q *x, const Q *v, const Q *d, Q *xp, Q *vp, Q *ap)
{
    const int K = 2 * p;
    for (int c = 0; c < 3; ++c) {
        Q sx = x[c] + v[c] * dt, sv = v[c];
        for (int k = 0; k < K; ++k) {
            sx += d[k * 3 + c] * qpow(dt, k + 2) / qfact(k + 2);
            sv += d[k * 3 + c] * qpow(dt, k + 1) / qfact(k + 1);
        }
        xp[c] = sx;
        vp[c] = sv;
        for (int q = 0; q + 2 <= p; ++q) {
            Q sa = 0;
            for (int k = q; k < K; ++k) sa += d[k * 3 + c] * qpow(dt, k - q) / qfact(k - q);
            ap[q * 3 + c] = sa;
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Section 2 (Eqs. 5-7): the corrector; one P(EC)^n step                      */
/* ------------------------------------------------------------------------- */

/* Velocity (Eq. 6, f = a), then position (Eq. 7, f = v with the new v1). */
static void qcorrect_one(int p, Q dt, const Q *cv, const Q *cx, const Q *x0, const Q *v0,
                         const Q *d0, const Q *d1, Q *x1, Q *v1)
{
    const Q h = dt / 2;
    for (int c = 0; c < 3; ++c) {
        Q dv = 0;
        for (int n = 0; n <= p; ++n) {
            const Q sc = qpow(h, n) / (2 * qfact(n));
            const Q fpm = (n % 2 == 0) ? sc * (d1[n * 3 + c] + d0[n * 3 + c])
                                       : sc * (d1[n * 3 + c] - d0[n * 3 + c]);
            dv += cv[n] * fpm;
        }
        v1[c] = v0[c] + dv * dt;
    }
    for (int c = 0; c < 3; ++c) {
        Q dx = 0;
        for (int n = 0; n <= p + 1; ++n) {
            const Q f1 = (n == 0) ? v1[c] : d1[(n - 1) * 3 + c];
            const Q f0 = (n == 0) ? v0[c] : d0[(n - 1) * 3 + c];
            const Q sc = qpow(h, n) / (2 * qfact(n));
            const Q fpm = (n % 2 == 0) ? sc * (f1 + f0) : sc * (f1 - f0);
            dx += cx[n] * fpm;
        }
        x1[c] = x0[c] + dx * dt;
    }
}

/* One shared P(EC)^n step of constant dt in place (no evaluation after the
 * last correction; a^(p+1..2p-1) at the end by interpolation, R3). */
static void qstep(int N, int p, const Q *cv, const Q *cx, int n_iter, Q dt, const double *m,
                  Q eps2, Q G, Q *x, Q *v, Q *derivs, Q *work)
{
    const int K = 2 * p, P = p, na = p > 1 ? p - 1 : 1;
    Q *xp = work, *vp = xp + (size_t)N * 3, *ap = vp + (size_t)N * 3;
    Q *tr = ap + (size_t)N * na * 3, *d1 = tr + (size_t)N * (P + 1) * 3;
    Q *x1 = d1 + (size_t)N * (P + 1) * 3, *v1 = x1 + (size_t)N * 3;
    for (int i = 0; i < N; ++i)
        qpredict_one(p, dt, x + 3 * i, v + 3 * i, derivs + (size_t)i * K * 3,
                     xp + 3 * i, vp + 3 * i, ap + (size_t)i * na * 3);
    memcpy(x1, xp, (size_t)N * 3 * sizeof(Q));
    memcpy(v1, vp, (size_t)N * 3 * sizeof(Q));
    for (int it = 0; it < n_iter; ++it) {
        for (int i = 0; i < N; ++i) {
            Q *t = tr + (size_t)i * (P + 1) * 3;
            for (int c = 0; c < 3; ++c) { t[c] = x1[i * 3 + c]; t[3 + c] = v1[i * 3 + c]; }
            for (int q = 0; q + 2 <= P; ++q)      /* R2: predicted, then the previous evaluation's */
                for (int c = 0; c < 3; ++c)
                    t[(q + 2) * 3 + c] = (it == 0) ? ap[((size_t)i * na + q) * 3 + c]
                                                   : d1[((size_t)i * (P + 1) + q) * 3 + c];
        }
        qevaluate(N, P, m, tr, eps2, G, d1);
        for (int i = 0; i < N; ++i) {
            Q d0[(ORQ_MAXP + 1) * 3];
            for (int q = 0; q <= P; ++q)
                for (int c = 0; c < 3; ++c) d0[q * 3 + c] = derivs[((size_t)i * K + q) * 3 + c];
            qcorrect_one(p, dt, cv, cx, x + 3 * i, v + 3 * i, d0, d1 + (size_t)i * (P + 1) * 3,
                         x1 + 3 * i, v1 + 3 * i);
        }
    }
    for (int i = 0; i < N; ++i) {
        Q d0[(ORQ_MAXP + 1) * 3], hi[2 * ORQ_MAXSYS * 3];
        const Q *e1 = d1 + (size_t)i * (P + 1) * 3;
        for (int q = 0; q <= P; ++q)
            for (int c = 0; c < 3; ++c) d0[q * 3 + c] = derivs[((size_t)i * K + q) * 3 + c];
        if (K > P + 1) qhermite_interp(p, dt, d0, e1, K, hi);
        for (int q = 0; q < K; ++q)
            for (int c = 0; c < 3; ++c)
                derivs[((size_t)i * K + q) * 3 + c] = (q <= P) ? e1[q * 3 + c] : hi[q * 3 + c];
        for (int c = 0; c < 3; ++c) { x[i * 3 + c] = x1[i * 3 + c]; v[i * 3 + c] = v1[i * 3 + c]; }
    }
}

/* Initialise (init != 0: a^(0..2p-1) from x, v; else from d2) and take nsteps
 * constant steps, all in binary128.  x2, v2: N x 3 x 2 in/out; d2: N x 2p x 3 x 2
 * in (init == 0) / out. */
void orq_run(int N, int p, int beta_mode, int n_iter, double dt, int nsteps, const double *m,
             double eps, double G, int init, double *x2, double *v2, double *d2)
{
    const int K = 2 * p, na = p > 1 ? p - 1 : 1;
    Q *x = (Q *)malloc((size_t)N * 3 * sizeof(Q));
    Q *v = (Q *)malloc((size_t)N * 3 * sizeof(Q));
    Q *d = (Q *)malloc((size_t)N * K * 3 * sizeof(Q));
    Q *work = (Q *)malloc((size_t)N * (3 * 4 + na * 3 + 2 * (p + 1) * 3) * sizeof(Q));
    for (int q = 0; q < N * 3; ++q) { x[q] = q_in(x2 + 2 * q); v[q] = q_in(v2 + 2 * q); }
    const Q eps2 = (Q)eps * (Q)eps;
    if (init) qinitialise(N, p, m, x, v, eps2, (Q)G, d);
    else for (int q = 0; q < N * K * 3; ++q) d[q] = q_in(d2 + 2 * q);
    Q cv[ORQ_MAXSYS], cx[ORQ_MAXSYS];
    qcorrector_weights(p, beta_mode, cv, cx);
    for (int s = 0; s < nsteps; ++s) qstep(N, p, cv, cx, n_iter, (Q)dt, m, eps2, (Q)G, x, v, d, work);
    for (int q = 0; q < N * 3; ++q) { q_out(x[q], x2 + 2 * q); q_out(v[q], v2 + 2 * q); }
    for (int q = 0; q < N * K * 3; ++q) q_out(d[q], d2 + 2 * q);
    free(x); free(v); free(d); free(work);
}

/* ------------------------------------------------------------------------- */
/* Diagnostics                                                                */
/* ------------------------------------------------------------------------- */

/* E = sum_i m_i |v_i|^2 / 2 - sum_{i<j} G m_i m_j / sqrt(r_ij^2 + eps^2)  (R4) */
void orq_energy(int N, const double *m, const double *x2, const double *v2, double eps, double G,
                double *E2)
{
    Q kin = 0, pot = 0;
    const Q eps2 = (Q)eps * (Q)eps;
    for (int i = 0; i < N; ++i) {
        Q u[3] = {q_in(v2 + 6 * i), q_in(v2 + 6 * i + 2), q_in(v2 + 6 * i + 4)};
        kin += (Q)m[i] * qdot3(u, u) / 2;
    }
    for (int i = 0; i < N; ++i) {
        Q pi = 0;
        for (int j = i + 1; j < N; ++j) {
            Q dd[3];
            for (int c = 0; c < 3; ++c) dd[c] = q_in(x2 + 6 * j + 2 * c) - q_in(x2 + 6 * i + 2 * c);
            pi += (Q)m[j] / sqrtf128(qdot3(dd, dd) + eps2);
        }
        pot += (Q)G * (Q)m[i] * pi;
    }
    q_out(kin - pot, E2);
}

/* Eccentricity vectors about body `central` (Appendix A, Eq. A1):
 * mu e = (|v|^2 - mu/|r|) r - (r.v) v, mu = G (m_c + m_i); e2: N x 3 x 2. */
void orq_ecc(int N, const double *m, const double *x2, const double *v2, double G, int central, double *e2)
{
    for (int i = 0; i < N; ++i) {
        if (i == central) { for (int q = 0; q < 6; ++q) e2[6 * i + q] = 0.0; continue; }
        Q r[3], u[3];
        for (int c = 0; c < 3; ++c) {
            r[c] = q_in(x2 + 6 * i + 2 * c) - q_in(x2 + 6 * central + 2 * c);
            u[c] = q_in(v2 + 6 * i + 2 * c) - q_in(v2 + 6 * central + 2 * c);
        }
        const Q mu = (Q)G * ((Q)m[central] + (Q)m[i]);
        const Q rn = sqrtf128(qdot3(r, r)), w2 = qdot3(u, u), rv = qdot3(r, u);
        for (int c = 0; c < 3; ++c) q_out(((w2 - mu / rn) * r[c] - rv * u[c]) / mu, e2 + 6 * i + 2 * c);
    }
}
