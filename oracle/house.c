/*
 * CPU oracle for Householder QR and least squares, FP64.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * reference that the CUDA path is checked against.  It shares no code,
 * header, table or helper with the CUDA library, and nothing in the product
 * path may call it: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark load it.
 *
 * What it computes (all matrices column-major, element (i,j) at a[i + j*ld]):
 *
 *  - house_qr: unblocked right-looking Householder QR, the b = 1 instance of
 *    the recursive template (Algorithm 1; Appendix A calls it 1D-house).  On
 *    return the strict lower trapezoid of A holds the Householder vectors V
 *    (unit diagonal implied), the upper triangle holds R, and tau[j] is the
 *    scaling of reflector j, H_j = I - tau_j v_j v_j^T, with
 *    Q = H_0 H_1 ... H_{n-1} (Section 2.3, Householder representation).
 *
 *    Sign reading: beta = -sgn(alpha) * ||[alpha; x]||, sgn(0) = +1, with no
 *    exception when x = 0 (then tau = 2 and the reflector negates coordinate
 *    j).  This is the convention that the reconstruction of Householder
 *    vectors from TSQR (Appendix C.2) produces: its Q-factor has -S X on the
 *    top diagonal, which a tau = 0 (identity) reflector cannot reproduce.  A
 *    column that is exactly zero gets v = e_j, tau = 2, beta = 0.
 *
 *  - larft: the kernel T of the compact-WY representation Q = I - V T V^T
 *    (Section 2.3), by the forward recurrence T(j,j) = tau_j,
 *    T(0:j, j) = -tau_j * T(0:j, 0:j) * (V(:, 0:j)^T v_j).
 *
 *  - t_from_gram: the same T by the closed form stated in Section 2.3,
 *    T = (striu(V^T V) + diag(diag(V^T V))/2)^{-1}, read with a strictly
 *    upper triangle (the printed "-1" diagonal offset is taken as garbled):
 *    an independent construction used to cross-check larft.
 *
 *  - apply_qt / apply_q / form_q: Q^T B, Q B and the thin factor Q [I; 0],
 *    one reflector at a time (the update of eq. basis-kernel-update with
 *    the reflectors taken singly).
 *
 *  - trsv_upper, ls_solve: back substitution with R and the least-squares
 *    solution x = R^{-1} (Q^T b)(0:n) of min ||A x - b|| (m >= n, Section 2.1).
 *
 * Nothing here is blocked, fused or reordered beyond those definitions.
 *
 * Built twice: plain (one thread) and with -fopenmp (all cores).  The OpenMP
 * pragmas only share out loops whose iterations write disjoint columns
 * (the columns that one reflector updates, the columns one reflector is
 * applied to, the entries of one column of T); each iteration's own
 * arithmetic and its order are unchanged, so both builds give bit-identical
 * results.
 */

#include <math.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(a, i, j, ld) ((a)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

static double sgn(double x) { return x < 0.0 ? -1.0 : 1.0; }

/* 2-norm of x[0:n] scaled by its largest magnitude, so that squaring can
 * neither overflow nor underflow for representable inputs. */
static double nrm2(long n, const double *x)
{
    double amax = 0.0;
    for (long i = 0; i < n; ++i) {
        double t = fabs(x[i]);
        if (t > amax) amax = t;
    }
    if (amax == 0.0) return 0.0;
    double s = 0.0;
    for (long i = 0; i < n; ++i) {
        double t = x[i] / amax;
        s += t * t;
    }
    return amax * sqrt(s);
}

/* Householder QR of the m x n matrix A, first nsteps <= min(m, n)
 * reflectors.  nsteps < min(m, n) leaves a partial factorization: columns
 * 0..nsteps-1 hold V\R and columns nsteps..n-1 hold
 * H_{nsteps-1} ... H_0 A(:, nsteps:n).  With m < n the m reflectors of the
 * leading m x m block are applied to every column, which is the wide-matrix
 * construction of Section 2.1: A = [A1 A2], A1 = Q R1, R = [R1, Q^T A2]. */
int orc_house_qr(long m, long n, double *a, long lda, double *tau, long nsteps)
{
    if (m < 0 || n < 0 || lda < (m > 1 ? m : 1)) return 1;
    if (nsteps > n) nsteps = n;
    if (nsteps > m) nsteps = m;
    for (long j = 0; j < nsteps; ++j) {
        double alpha = AT(a, j, j, lda);
        double xnorm = nrm2(m - j - 1, &AT(a, j + 1, j, lda));
        double norm = hypot(alpha, xnorm);
        double beta = -sgn(alpha) * norm;
        if (beta == 0.0) {
            /* zero column: v = e_j (already zero below), tau = 2 */
            tau[j] = 2.0;
            AT(a, j, j, lda) = 0.0;
        } else {
            tau[j] = (beta - alpha) / beta;
            double d = alpha - beta;
            for (long r = j + 1; r < m; ++r) AT(a, r, j, lda) /= d;
            AT(a, j, j, lda) = beta;
        }
        /* apply H_j = I - tau_j v v^T to A(j:m, j+1:n), v = [1; A(j+1:m, j)] */
#pragma omp parallel for schedule(static) if (m * (n - j) > 65536)
        for (long c = j + 1; c < n; ++c) {
            double w = AT(a, j, c, lda);
            for (long r = j + 1; r < m; ++r) w += AT(a, r, j, lda) * AT(a, r, c, lda);
            w *= tau[j];
            AT(a, j, c, lda) -= w;
            for (long r = j + 1; r < m; ++r) AT(a, r, c, lda) -= w * AT(a, r, j, lda);
        }
    }
    return 0;
}

/* v_i^T v_j for i < j, with v_k = [0 (k entries); 1; V(k+1:m, k)]. */
static double vdot(long m, const double *v, long ldv, long i, long j)
{
    double s = AT(v, j, i, ldv); /* row j: v_i(j) * v_j(j) with v_j(j) = 1 */
    for (long r = j + 1; r < m; ++r) s += AT(v, r, i, ldv) * AT(v, r, j, ldv);
    return s;
}

/* T (n x n, upper triangular, zeros written below the diagonal) by the
 * forward recurrence. */
int orc_larft(long m, long n, const double *v, long ldv, const double *tau, double *t, long ldt)
{
    if (m < n || ldv < (m > 1 ? m : 1) || ldt < (n > 1 ? n : 1)) return 1;
    double *z = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!z) return 2;
    for (long j = 0; j < n; ++j) {
        for (long i = 0; i < n; ++i) AT(t, i, j, ldt) = 0.0;
#pragma omp parallel for schedule(static) if (m * j > 65536)
        for (long i = 0; i < j; ++i) z[i] = vdot(m, v, ldv, i, j);
#pragma omp parallel for schedule(static) if (j * j > 65536)
        for (long i = 0; i < j; ++i) {
            double s = 0.0;
            for (long k = i; k < j; ++k) s += AT(t, i, k, ldt) * z[k];
            AT(t, i, j, ldt) = -tau[j] * s;
        }
        AT(t, j, j, ldt) = tau[j];
    }
    free(z);
    return 0;
}

/* T = (striu(V^T V) + diag(V^T V)/2)^{-1}, the inverse of an upper
 * triangular matrix taken column by column by back substitution. */
int orc_t_from_gram(long m, long n, const double *v, long ldv, double *t, long ldt)
{
    if (m < n || ldv < (m > 1 ? m : 1) || ldt < (n > 1 ? n : 1)) return 1;
    double *g = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n * n : 1));
    if (!g) return 2;
    /* G = striu(V^T V) + diag(V^T V)/2, stored n x n column-major */
    for (long j = 0; j < n; ++j) {
        for (long i = 0; i < n; ++i) g[i + j * n] = 0.0;
        for (long i = 0; i < j; ++i) g[i + j * n] = vdot(m, v, ldv, i, j);
        double d = 1.0;
        for (long r = j + 1; r < m; ++r) d += AT(v, r, j, ldv) * AT(v, r, j, ldv);
        g[j + j * n] = d / 2.0;
    }
    /* solve G * T(:, j) = e_j for each j */
    for (long j = 0; j < n; ++j) {
        for (long i = 0; i < n; ++i) AT(t, i, j, ldt) = 0.0;
        for (long i = j; i >= 0; --i) {
            double s = (i == j) ? 1.0 : 0.0;
            for (long k = i + 1; k <= j; ++k) s -= g[i + k * n] * AT(t, k, j, ldt);
            AT(t, i, j, ldt) = s / g[i + i * n];
        }
    }
    free(g);
    return 0;
}

/* Apply H_j to columns of B: B(j:m, :) -= tau_j v_j (v_j^T B(j:m, :)). */
static void apply_reflector(long m, long j, const double *v, long ldv, double tauj,
                            long nrhs, double *b, long ldb)
{
#pragma omp parallel for schedule(static) if (m * nrhs > 65536)
    for (long c = 0; c < nrhs; ++c) {
        double w = AT(b, j, c, ldb);
        for (long r = j + 1; r < m; ++r) w += AT(v, r, j, ldv) * AT(b, r, c, ldb);
        w *= tauj;
        AT(b, j, c, ldb) -= w;
        for (long r = j + 1; r < m; ++r) AT(b, r, c, ldb) -= w * AT(v, r, j, ldv);
    }
}

/* B <- Q^T B = H_{n-1} ... H_0 B  (B is m x nrhs). */
int orc_apply_qt(long m, long n, const double *v, long ldv, const double *tau,
                 long nrhs, double *b, long ldb)
{
    if (m < n || ldv < (m > 1 ? m : 1) || ldb < (m > 1 ? m : 1)) return 1;
    for (long j = 0; j < n; ++j) apply_reflector(m, j, v, ldv, tau[j], nrhs, b, ldb);
    return 0;
}

/* B <- Q B = H_0 ... H_{n-1} B. */
int orc_apply_q(long m, long n, const double *v, long ldv, const double *tau,
                long nrhs, double *b, long ldb)
{
    if (m < n || ldv < (m > 1 ? m : 1) || ldb < (m > 1 ? m : 1)) return 1;
    for (long j = n - 1; j >= 0; --j) apply_reflector(m, j, v, ldv, tau[j], nrhs, b, ldb);
    return 0;
}

/* Thin Q factor: Q(:, 0:n) = Q [I_n; 0]. */
int orc_form_q(long m, long n, const double *v, long ldv, const double *tau, double *q, long ldq)
{
    if (m < n || ldq < (m > 1 ? m : 1)) return 1;
    for (long j = 0; j < n; ++j)
        for (long i = 0; i < m; ++i) AT(q, i, j, ldq) = (i == j) ? 1.0 : 0.0;
    return orc_apply_q(m, n, v, ldv, tau, n, q, ldq);
}

/* Solve R x = c in place (x holds c on entry), R upper triangular n x n. */
int orc_trsv_upper(long n, const double *r, long ldr, double *x)
{
    for (long i = n - 1; i >= 0; --i) {
        double s = x[i];
        for (long k = i + 1; k < n; ++k) s -= AT(r, i, k, ldr) * x[k];
        x[i] = s / AT(r, i, i, ldr);
    }
    return 0;
}

/* Least squares min ||A x - b||_2 for m x n A (m >= n) of full rank.
 * A and b are not modified.  x receives n entries; *resnorm receives
 * ||(Q^T b)(n:m)||_2, the norm of the residual b - A x. */
int orc_ls_solve(long m, long n, const double *a, long lda, const double *b,
                 double *x, double *resnorm)
{
    if (m < n || lda < (m > 1 ? m : 1)) return 1;
    double *w = (double *)malloc(sizeof(double) * (size_t)(m * (n > 0 ? n : 1)));
    double *tau = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *c = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!w || !tau || !c) { free(w); free(tau); free(c); return 2; }
    for (long j = 0; j < n; ++j)
        for (long i = 0; i < m; ++i) w[i + j * m] = AT(a, i, j, lda);
    for (long i = 0; i < m; ++i) c[i] = b[i];
    int rc = orc_house_qr(m, n, w, m, tau, n);
    if (rc == 0) rc = orc_apply_qt(m, n, w, m, tau, 1, c, m);
    if (rc == 0) {
        for (long i = 0; i < n; ++i) x[i] = c[i];
        orc_trsv_upper(n, w, m, x);
        if (resnorm) *resnorm = nrm2(m - n, c + n);
    }
    free(w); free(tau); free(c);
    return rc;
}

/* Threads the loops above share out: omp_get_max_threads() in the OpenMP
 * build, 1 in the plain one. */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
