/*
 * Plain FP64 CPU oracle for the reduction of a dense matrix to compact band form.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct statement of
 * what the reduction computes; it is used by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark, never by the library.  It shares no code, header
 * or constant with the CUDA path.
 *
 * Paper: Rodriguez-Sanchez, Catalan, Herrero, Quintana-Orti, Tomas, "Look-Ahead in the
 * Two-Sided Reduction to Compact Band Forms for Symmetric Eigenvalue Problems and the
 * SVD" (arXiv:1709.00302).
 *
 * Reading of the method used here (one reflector at a time, full dense storage):
 *
 *  - Symmetric band reduction, Section 2.1 (Eqs. updateA0 .. updateA2syr2k) read
 *    unblocked: for each column c the reflector that annihilates A(c+w+1:n, c) is
 *    applied from both sides, A := H A H.  Because the block size satisfies b <= w
 *    (Section 2.1), a blocked implementation produces the same reflectors in exact
 *    arithmetic: a panel column c+i (i < b <= w) never lies in the column range
 *    (>= c+w) touched by the right-hand application of the panel's earlier reflectors.
 *  - Triangular-band reduction for the SVD, Section 3.1 (Eqs. updateB .. updateD) read
 *    unblocked: alternating a left reflector on column c and a right reflector on row c
 *    beyond the superdiagonal w.
 *  - Householder convention (the paper defers to Golub & Van Loan): for x = [alpha; x2],
 *    beta = -sign(alpha) * ||x||_2 with sign(0) = +1, tau = (beta - alpha)/beta,
 *    v = [1; x2/(alpha - beta)].  When ||x2|| = 0 (or x has length 1) tau = 0 and
 *    beta = alpha, so H = I.
 *
 * Index conventions: 0-based, column-major, A(i,j) = A[i + j*lda].
 *
 * Outputs (packed, the same layout the library writes):
 *  sy2sb: the lower band 0 <= i-j <= w of A holds the band matrix B; for reflector c
 *         (c = 0 .. n-w-1), A(c+w, c) = beta_c and A(c+w+1 : n, c) holds v_c below its
 *         implicit unit entry; tau[c] = tau_c (tau[n-w-1] = 0: a length-1 reflector).
 *         The oracle keeps the full symmetric matrix while it works; on return the
 *         strictly upper triangle holds the mirror of the band and zeros elsewhere.
 *  ge2gb: upper triangular band 0 <= j-i <= w of A holds B (m >= n); the left reflector
 *         c has beta on A(c,c) and v below the diagonal (tauq[c], c = 0..n-1); the right
 *         reflector c (c = 0 .. n-w-1) has beta on A(c, c+w) and v in A(c, c+w+1 : n)
 *         (taup[c]).
 *
 * Each sweep over the columns of the trailing matrix is optionally split over OpenMP
 * threads; every element is computed by one thread in a fixed order, so the results do
 * not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define AT(A, lda, i, j) ((A)[(int64_t)(i) + (int64_t)(j) * (int64_t)(lda)])

static int oracle_threads = 1;

/* Number of threads the sweeps may use (1 = serial). Returns the value in effect. */
int oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t < 1) t = omp_get_max_threads();
    oracle_threads = t;
#else
    (void)t;
    oracle_threads = 1;
#endif
    return oracle_threads;
}

int oracle_get_threads(void) { return oracle_threads; }

/* ||x||_2 of a strided vector, scaled by max|x_i| so that squares neither overflow nor
 * underflow (two passes: the plain textbook statement of a safe norm). */
static double safe_norm(int64_t len, const double *x, int64_t inc) {
    double amax = 0.0;
    for (int64_t i = 0; i < len; ++i) {
        double a = fabs(x[i * inc]);
        if (a > amax || isnan(a)) amax = a;
    }
    if (amax == 0.0 || isnan(amax) || isinf(amax)) return amax;
    double s = 0.0;
    for (int64_t i = 0; i < len; ++i) {
        double t = x[i * inc] / amax;
        s += t * t;
    }
    return amax * sqrt(s);
}

/* Householder reflector for x = [x[0]; x[inc], x[2 inc], ...] of length len.
 * On return x[0] = beta, x[1..] = v(2..) (v(1) = 1 implicit), *tau set. */
static void house(int64_t len, double *x, int64_t inc, double *tau) {
    if (len <= 1) { *tau = 0.0; return; }
    double alpha = x[0];
    double xnorm = safe_norm(len - 1, x + inc, inc);
    if (xnorm == 0.0) { *tau = 0.0; return; }
    double h = hypot(alpha, xnorm);
    double beta = (alpha >= 0.0) ? -h : h;   /* sign(0) = +1 */
    *tau = (beta - alpha) / beta;
    double scal = 1.0 / (alpha - beta);
    for (int64_t i = 1; i < len; ++i) x[i * inc] *= scal;
    x[0] = beta;
}

/* p[i] = t * sum_j M(i,j) v[j] for an nrow x len column-major block M.  Each p[i] is
 * summed over j in increasing order; threads own disjoint ranges of rows. */
static void row_times_v(int64_t nrow, int64_t len, const double *M, int64_t lda, const double *v,
                        double t, double *p) {
    const int64_t chunk = 256;
#pragma omp parallel for num_threads(oracle_threads) schedule(static) if (oracle_threads > 1)
    for (int64_t ib = 0; ib < nrow; ib += chunk) {
        int64_t ie = ib + chunk < nrow ? ib + chunk : nrow;
        for (int64_t i = ib; i < ie; ++i) p[i] = 0.0;
        for (int64_t j = 0; j < len; ++j) {
            const double *col = &AT(M, lda, 0, j);
            double vj = v[j];
            for (int64_t i = ib; i < ie; ++i) p[i] += col[i] * vj;
        }
        for (int64_t i = ib; i < ie; ++i) p[i] *= t;
    }
}

/* ---------------------------------------------------------------------------------
 * Symmetric A (full storage, both triangles) -> symmetric band, bandwidth w.
 * Section 2.1, Eqs. updateA0, updateA1, updateA2, one reflector at a time.
 * Only the lower triangle of the input is read: it is mirrored first.
 * ncols >= 0 stops after that many reflectors (a bounded sample for timing);
 * ncols < 0 runs to completion.  Returns 0, or -i for an invalid i-th argument.
 * ---------------------------------------------------------------------------------*/
int oracle_sy2sb(int64_t n, int64_t w, double *A, int64_t lda, double *tau, int64_t ncols) {
    if (n < 0) return -1;
    if (w < 1) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j + 1; i < n; ++i) AT(A, lda, j, i) = AT(A, lda, i, j);
    int64_t nref = n - w; /* reflectors c = 0 .. n-w-1 (the last one has length 1) */
    if (nref <= 0) return 0;
    for (int64_t c = 0; c < nref; ++c) tau[c] = 0.0;
    double *v = (double *)malloc(sizeof(double) * (size_t)n);
    double *p = (double *)malloc(sizeof(double) * (size_t)n);
    if (!v || !p) { free(v); free(p); return -100; }
    int64_t last = (ncols >= 0 && ncols < nref) ? ncols : nref;
    for (int64_t c = 0; c < last; ++c) {
        int64_t r0 = c + w;      /* first row the reflector acts on */
        int64_t len = n - r0;    /* reflector length */
        double t;
        house(len, &AT(A, lda, r0, c), 1, &t);
        tau[c] = t;
        if (t == 0.0) continue;  /* H = I: nothing else changes */
        v[0] = 1.0;
        for (int64_t i = 1; i < len; ++i) v[i] = AT(A, lda, r0 + i, c);
        /* Left application H * A(r0:n, c+1:n): each column independently. */
        int64_t ncol = n - (c + 1);
#pragma omp parallel for num_threads(oracle_threads) schedule(static) if (oracle_threads > 1)
        for (int64_t jj = 0; jj < ncol; ++jj) {
            double *col = &AT(A, lda, r0, c + 1 + jj);
            double s = 0.0;
            for (int64_t i = 0; i < len; ++i) s += v[i] * col[i];
            s *= t;
            for (int64_t i = 0; i < len; ++i) col[i] -= s * v[i];
        }
        /* Right application A(c+1:n, r0:n) * H: p = A(c+1:n, r0:n) v, then rank-1. */
        int64_t nrow = n - (c + 1);
        row_times_v(nrow, len, &AT(A, lda, c + 1, r0), lda, v, t, p);
#pragma omp parallel for num_threads(oracle_threads) schedule(static) if (oracle_threads > 1)
        for (int64_t jj = 0; jj < len; ++jj) {
            double *col = &AT(A, lda, c + 1, r0 + jj);
            double vj = v[jj];
            for (int64_t ii = 0; ii < nrow; ++ii) col[ii] -= p[ii] * vj;
        }
        /* Row c: the mirror of column c is beta at (c, r0) and zeros beyond. */
        AT(A, lda, c, r0) = AT(A, lda, r0, c);
        for (int64_t jj = r0 + 1; jj < n; ++jj) AT(A, lda, c, jj) = 0.0;
    }
    free(v);
    free(p);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * General A (m x n, m >= n) -> upper triangular band with upper bandwidth w.
 * Section 3.1, Eqs. updateB, updateCD, updateC, updateD, one reflector at a time.
 * ncols >= 0 stops after that many (left, right) reflector pairs.
 * ---------------------------------------------------------------------------------*/
int oracle_ge2gb(int64_t m, int64_t n, int64_t w, double *A, int64_t lda, double *tauq,
                 double *taup, int64_t ncols) {
    if (m < 0) return -1;
    if (n < 0 || n > m) return -2;
    if (w < 1) return -3;
    if (lda < (m > 1 ? m : 1)) return -5;
    for (int64_t c = 0; c < n; ++c) tauq[c] = 0.0;
    int64_t nrp = n - w > 0 ? n - w : 0;
    for (int64_t c = 0; c < nrp; ++c) taup[c] = 0.0;
    int64_t maxlen = m > n ? m : n;
    double *v = (double *)malloc(sizeof(double) * (size_t)(maxlen + 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(maxlen + 1));
    if (!v || !p) { free(v); free(p); return -100; }
    int64_t last = (ncols >= 0 && ncols < n) ? ncols : n;
    for (int64_t c = 0; c < last; ++c) {
        /* Left reflector on column c, rows c..m-1, applied to columns c+1..n-1. */
        int64_t len = m - c;
        double t;
        house(len, &AT(A, lda, c, c), 1, &t);
        tauq[c] = t;
        if (t != 0.0) {
            v[0] = 1.0;
            for (int64_t i = 1; i < len; ++i) v[i] = AT(A, lda, c + i, c);
            int64_t ncol = n - (c + 1);
#pragma omp parallel for num_threads(oracle_threads) schedule(static) if (oracle_threads > 1)
            for (int64_t jj = 0; jj < ncol; ++jj) {
                double *col = &AT(A, lda, c, c + 1 + jj);
                double s = 0.0;
                for (int64_t i = 0; i < len; ++i) s += v[i] * col[i];
                s *= t;
                for (int64_t i = 0; i < len; ++i) col[i] -= s * v[i];
            }
        }
        /* Right reflector on row c, columns c+w..n-1, applied to rows c+1..m-1. */
        if (c < nrp) {
            int64_t r0 = c + w;
            int64_t rlen = n - r0;
            house(rlen, &AT(A, lda, c, r0), lda, &t);
            taup[c] = t;
            if (t != 0.0) {
                v[0] = 1.0;
                for (int64_t j = 1; j < rlen; ++j) v[j] = AT(A, lda, c, r0 + j);
                int64_t nrow = m - (c + 1);
                row_times_v(nrow, rlen, &AT(A, lda, c + 1, r0), lda, v, t, p);
#pragma omp parallel for num_threads(oracle_threads) schedule(static) if (oracle_threads > 1)
                for (int64_t jj = 0; jj < rlen; ++jj) {
                    double *col = &AT(A, lda, c + 1, r0 + jj);
                    double vj = v[jj];
                    for (int64_t ii = 0; ii < nrow; ++ii) col[ii] -= p[ii] * vj;
                }
            }
        }
    }
    free(v);
    free(p);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * General A (m x n) -> band with lower AND upper bandwidth w (the SVD band form of
 * Section 3.3, Eqs. updateB0 .. gebrd_2k, read unblocked): for c = 0, 1, ... a left
 * reflector annihilates A(c+w+1 : m, c) (acting on rows c+w .. m-1) and a right reflector
 * annihilates A(c, c+w+1 : n) (acting on columns c+w .. n-1).  With b <= w the blocked
 * algorithm gives the same reflectors in exact arithmetic: a block's left reflectors act
 * on rows >= k+w, below its right panel's rows, and its right reflectors on columns
 * >= k+w, right of its left panel's columns.
 * Outputs: B in the band |i-j| <= w; left reflector c (c = 0 .. min(n, m-w)-1): beta on
 * A(c+w, c), v in A(c+w+1 : m, c), tauq[c]; right reflector c (c = 0 .. min(m, n-w)-1):
 * beta on A(c, c+w), v in A(c, c+w+1 : n), taup[c].
 * ncols >= 0 stops after that many (left, right) pairs.
 * ---------------------------------------------------------------------------------*/
int oracle_ge2bb(int64_t m, int64_t n, int64_t w, double *A, int64_t lda, double *tauq,
                 double *taup, int64_t ncols) {
    if (m < 0) return -1;
    if (n < 0) return -2;
    if (w < 1) return -3;
    if (lda < (m > 1 ? m : 1)) return -5;
    int64_t nlq = (m - w < n ? m - w : n), nrq = (n - w < m ? n - w : m);
    if (nlq < 0) nlq = 0;
    if (nrq < 0) nrq = 0;
    for (int64_t c = 0; c < nlq; ++c) tauq[c] = 0.0;
    for (int64_t c = 0; c < nrq; ++c) taup[c] = 0.0;
    int64_t maxlen = m > n ? m : n;
    double *v = (double *)malloc(sizeof(double) * (size_t)(maxlen + 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(maxlen + 1));
    if (!v || !p) { free(v); free(p); return -100; }
    int64_t cmax = nlq > nrq ? nlq : nrq;
    int64_t last = (ncols >= 0 && ncols < cmax) ? ncols : cmax;
    for (int64_t c = 0; c < last; ++c) {
        double t;
        /* Left reflector on column c, rows c+w..m-1, applied to columns c+1..n-1. */
        if (c < nlq) {
            int64_t r0 = c + w, len = m - r0;
            house(len, &AT(A, lda, r0, c), 1, &t);
            tauq[c] = t;
            if (t != 0.0) {
                v[0] = 1.0;
                for (int64_t i = 1; i < len; ++i) v[i] = AT(A, lda, r0 + i, c);
                int64_t ncol = n - (c + 1);
#pragma omp parallel for num_threads(oracle_threads) schedule(static) if (oracle_threads > 1)
                for (int64_t jj = 0; jj < ncol; ++jj) {
                    double *col = &AT(A, lda, r0, c + 1 + jj);
                    double s = 0.0;
                    for (int64_t i = 0; i < len; ++i) s += v[i] * col[i];
                    s *= t;
                    for (int64_t i = 0; i < len; ++i) col[i] -= s * v[i];
                }
            }
        }
        /* Right reflector on row c, columns c+w..n-1, applied to rows c+1..m-1. */
        if (c < nrq) {
            int64_t r0 = c + w, rlen = n - r0;
            house(rlen, &AT(A, lda, c, r0), lda, &t);
            taup[c] = t;
            if (t != 0.0) {
                v[0] = 1.0;
                for (int64_t j = 1; j < rlen; ++j) v[j] = AT(A, lda, c, r0 + j);
                int64_t nrow = m - (c + 1);
                row_times_v(nrow, rlen, &AT(A, lda, c + 1, r0), lda, v, t, p);
#pragma omp parallel for num_threads(oracle_threads) schedule(static) if (oracle_threads > 1)
                for (int64_t jj = 0; jj < rlen; ++jj) {
                    double *col = &AT(A, lda, c + 1, r0 + jj);
                    double vj = v[jj];
                    for (int64_t ii = 0; ii < nrow; ++ii) col[ii] -= p[ii] * vj;
                }
            }
        }
    }
    free(v);
    free(p);
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Eigenvalues of a small symmetric matrix by the cyclic Jacobi method (Golub & Van
 * Loan, "Matrices Computations", the symmetric Schur decomposition of 2x2 blocks
 * applied row by row until the off-diagonal norm is negligible).  Only the lower
 * triangle of A is read; A is copied.  Eigenvalues are returned unsorted in lam[n].
 * Returns the number of sweeps used, or -1 when it did not converge.
 * ---------------------------------------------------------------------------------*/
int oracle_jacobi_eig(int64_t n, const double *A, int64_t lda, double *lam) {
    double *S = (double *)malloc(sizeof(double) * (size_t)(n * n + 1));
    if (!S) return -100;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i)
            S[i + j * n] = (i >= j) ? AT(A, lda, i, j) : AT(A, lda, j, i);
    int sweeps = -1;
    for (int sweep = 1; sweep <= 100; ++sweep) {
        int rotated = 0;
        for (int64_t p = 0; p < n - 1; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                double apq = S[p + q * n];
                double app = S[p + p * n], aqq = S[q + q * n];
                /* Negligible coupling (relative to the two diagonal entries): skip. */
                if (fabs(apq) <= 1e-17 * sqrt(fabs(app * aqq)) || fabs(apq) <= 1e-300) continue;
                rotated = 1;
                /* Rotation [c s; -s c] that zeroes the (p,q) entry of J^T S J. */
                double theta = (aqq - app) / (2.0 * apq);
                double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(1.0 + theta * theta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = t * cs;
                for (int64_t k = 0; k < n; ++k) { /* S := S J (columns p, q) */
                    double skp = S[k + p * n], skq = S[k + q * n];
                    S[k + p * n] = cs * skp - sn * skq;
                    S[k + q * n] = sn * skp + cs * skq;
                }
                for (int64_t k = 0; k < n; ++k) { /* S := J^T S (rows p, q) */
                    double spk = S[p + k * n], sqk = S[q + k * n];
                    S[p + k * n] = cs * spk - sn * sqk;
                    S[q + k * n] = sn * spk + cs * sqk;
                }
            }
        }
        if (!rotated) { sweeps = sweep; break; }
    }
    for (int64_t i = 0; i < n; ++i) lam[i] = S[i + i * n];
    free(S);
    return sweeps;
}

/* ---------------------------------------------------------------------------------
 * Singular values of a small m x n matrix (m >= n) by one-sided Jacobi (Hestenes):
 * orthogonalise pairs of columns by plane rotations until every pair is orthogonal to
 * working precision; the singular values are the final column norms (unsorted).
 * Returns the number of sweeps used, or -1 when it did not converge.
 * ---------------------------------------------------------------------------------*/
int oracle_jacobi_svd(int64_t m, int64_t n, const double *A, int64_t lda, double *sig) {
    double *U = (double *)malloc(sizeof(double) * (size_t)(m * n + 1));
    if (!U) return -100;
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < m; ++i) U[i + j * m] = AT(A, lda, i, j);
    int sweeps = -1;
    for (int sweep = 1; sweep <= 100; ++sweep) {
        int rotated = 0;
        for (int64_t p = 0; p < n - 1; ++p) {
            for (int64_t q = p + 1; q < n; ++q) {
                double alpha = 0.0, beta = 0.0, gamma = 0.0;
                for (int64_t k = 0; k < m; ++k) {
                    alpha += U[k + p * m] * U[k + p * m];
                    beta += U[k + q * m] * U[k + q * m];
                    gamma += U[k + p * m] * U[k + q * m];
                }
                if (gamma == 0.0 || fabs(gamma) <= 1e-16 * sqrt(alpha * beta)) continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
                for (int64_t k = 0; k < m; ++k) {
                    double up = U[k + p * m], uq = U[k + q * m];
                    U[k + p * m] = cs * up - sn * uq;
                    U[k + q * m] = sn * up + cs * uq;
                }
            }
        }
        if (!rotated) { sweeps = sweep; break; }
    }
    for (int64_t j = 0; j < n; ++j) {
        double s = 0.0;
        for (int64_t k = 0; k < m; ++k) s += U[k + j * m] * U[k + j * m];
        sig[j] = sqrt(s);
    }
    free(U);
    return sweeps;
}

/* ---------------------------------------------------------------------------------
 * Second stage (the step after the band form that the paper's eigenvalue experiments
 * take with SBRDT and DSTERF): symmetric band (bandwidth w) -> tridiagonal by bulge
 * chasing with Householder reflectors, then the eigenvalues of the tridiagonal.
 *
 * Band -> tridiagonal, one reflector at a time on a dense symmetric copy.  Sweep c
 * (c = 0 .. n-3) first annihilates A(c+2 : c+w+1, c) with a reflector on the index range
 * [c+1, c+1+w) (keeping A(c+1, c)), applied from both sides.  Its right application to
 * the rows below that range fills a triangle below the band (the bulge); the next
 * reflector of the sweep annihilates the bulge's first column below its in-band entry,
 * on the range shifted by w, and so on to the end of the matrix.  The other columns of a
 * bulge are annihilated by the sweeps that follow, whose ranges start one index later.
 * Every reflector follows the larfg convention above.  Each application touches only
 * the rows and columns within 2w of its range (everything else is zero there).
 * A: n x n, lower triangle holds the band (0 <= i-j <= w; the rest of it is ignored).
 * On return d[0..n) is the diagonal and e[0..n-1) the subdiagonal.
 * Returns 0, -i for an invalid i-th argument, -100 when out of memory.
 * ---------------------------------------------------------------------------------*/
int oracle_sb2st(int64_t n, int64_t w, const double *A, int64_t lda, double *d, double *e) {
    if (n < 0) return -1;
    if (w < 1) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n == 0) return 0;
    double *M = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
    double *v = (double *)malloc(sizeof(double) * (size_t)(w + 1));
    double *p = (double *)malloc(sizeof(double) * (size_t)(5 * w + 2));
    if (!M || !v || !p) { free(M); free(v); free(p); return -100; }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = j; i < n && i <= j + w; ++i) AT(M, n, i, j) = AT(M, n, j, i) = AT(A, lda, i, j);
    for (int64_t c = 0; c + 2 < n; ++c) {
        int64_t col = c, s = c + 1;
        while (1) {
            int64_t end = s + w < n ? s + w : n;
            int64_t len = end - s;
            if (len < 2) break;
            double t;
            house(len, &AT(M, n, s, col), 1, &t);
            /* the mirror of the annihilated column */
            for (int64_t i = 0; i < len; ++i) AT(M, n, col, s + i) = AT(M, n, s + i, col);
            if (t != 0.0) {
                v[0] = 1.0;
                for (int64_t i = 1; i < len; ++i) v[i] = AT(M, n, s + i, col);
                int64_t lo = s - 2 * w > 0 ? s - 2 * w : 0, hi = end + 2 * w < n ? end + 2 * w : n;
                /* left: rows [s, end) of columns [lo, hi) other than col, which is done */
                for (int64_t j = lo; j < hi; ++j) {
                    if (j == col) continue;
                    double z = 0.0;
                    for (int64_t i = 0; i < len; ++i) z += v[i] * AT(M, n, s + i, j);
                    z *= t;
                    for (int64_t i = 0; i < len; ++i) AT(M, n, s + i, j) -= z * v[i];
                }
                /* right: columns [s, end) of rows [lo, hi) other than col */
                for (int64_t i = lo; i < hi; ++i) {
                    if (i == col) continue;
                    double z = 0.0;
                    for (int64_t k = 0; k < len; ++k) z += AT(M, n, i, s + k) * v[k];
                    p[i - lo] = z * t;
                }
                for (int64_t k = 0; k < len; ++k)
                    for (int64_t i = lo; i < hi; ++i)
                        if (i != col) AT(M, n, i, s + k) -= p[i - lo] * v[k];
            }
            /* the annihilated entries are exactly zero */
            for (int64_t i = 1; i < len; ++i) AT(M, n, s + i, col) = AT(M, n, col, s + i) = 0.0;
            col = s;
            s += w;
        }
    }
    for (int64_t i = 0; i < n; ++i) d[i] = AT(M, n, i, i);
    for (int64_t i = 0; i + 1 < n; ++i) e[i] = AT(M, n, i + 1, i);
    free(M);
    free(v);
    free(p);
    return 0;
}

/* Number of eigenvalues of the symmetric tridiagonal (d, e) below x: the negative terms
 * of the Sturm sequence q_0 = d_0 - x, q_i = d_i - x - e_{i-1}^2 / q_{i-1} (Sylvester's law
 * of inertia for the LDL^T factorisation of T - x I).  A zero term is replaced by
 * -pivmin, a tiny negative number (x nudged past an eigenvalue at the pole). */
static int64_t sturm_count(int64_t n, const double *d, const double *e, double x, double pivmin) {
    int64_t neg = 0;
    double q = d[0] - x;
    if (fabs(q) < pivmin) q = -pivmin;
    if (q < 0.0) ++neg;
    for (int64_t i = 1; i < n; ++i) {
        q = d[i] - x - e[i - 1] * e[i - 1] / q;
        if (fabs(q) < pivmin) q = -pivmin;
        if (q < 0.0) ++neg;
    }
    return neg;
}

/* Eigenvalues of the symmetric tridiagonal T = (d, e), ascending, by bisection: lam[k]
 * is the point where the count of eigenvalues below x passes k, bracketed in the
 * Gershgorin interval and halved until the bracket is within a few units in the last
 * place of max |T|.  Returns 0, -i for an invalid i-th argument. */
int oracle_tridiag_eig(int64_t n, const double *d, const double *e, double *lam) {
    if (n < 0) return -1;
    if (n == 0) return 0;
    double gl = d[0], gu = d[0], tmax = 0.0, emax2 = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = (i > 0 ? fabs(e[i - 1]) : 0.0) + (i + 1 < n ? fabs(e[i]) : 0.0);
        if (d[i] - r < gl) gl = d[i] - r;
        if (d[i] + r > gu) gu = d[i] + r;
        if (fabs(d[i]) > tmax) tmax = fabs(d[i]);
        if (i + 1 < n) {
            if (fabs(e[i]) > tmax) tmax = fabs(e[i]);
            if (e[i] * e[i] > emax2) emax2 = e[i] * e[i];
        }
    }
    const double eps = 0x1p-53;
    const double pivmin = (emax2 > 1.0 ? emax2 : 1.0) * 0x1p-1020;
    const double tol = 4.0 * eps * (tmax > 0.0 ? tmax : 1.0);
    gl -= tol;
    gu += tol;
    for (int64_t k = 0; k < n; ++k) {
        double lo = gl, hi = gu;  /* count(lo) <= k < count(hi) */
        for (int it = 0; it < 200 && hi - lo > tol; ++it) {
            double mid = 0.5 * (lo + hi);
            if (mid <= lo || mid >= hi) break;
            if (sturm_count(n, d, e, mid, pivmin) > k)
                hi = mid;
            else
                lo = mid;
        }
        lam[k] = 0.5 * (lo + hi);
    }
    return 0;
}

/* ---------------------------------------------------------------------------------
 * Second stage for the SVD (the paper's introduction: the SVD's compact form is upper
 * triangular-band with upper bandwidth w, reduced to bidiagonal form in a second stage,
 * whose singular values follow): upper band -> upper bidiagonal by bulge chasing with
 * Householder reflectors, then the singular values of the bidiagonal.
 *
 * Band -> bidiagonal, one reflector at a time on a dense copy.  Sweep c (c = 0 .. n-2)
 * alternates right and left reflectors on index ranges that move down by w.  The right
 * reflector on columns [a, a+w) (a = c+1 first) annihilates row r's entries past its
 * first (r = c first) and is applied to every other row; on rows [a, a+w) it fills the
 * triangle below their diagonal (the lower bulge).  The left reflector on rows [a, a+w)
 * annihilates column a below its diagonal and is applied to every other column; on rows
 * [a, a+w) it fills the entries past the band (the upper bulge).  Then r = a and a moves
 * on by w: the next right reflector annihilates the upper bulge's first row past its
 * in-band entry, and so on to the end of the matrix.  The other rows and columns of each
 * bulge are annihilated by the sweeps that follow.  Every reflector follows the larfg
 * convention above.  Nonzeros never sit more than 2w - 1 above or w - 2 below the
 * diagonal, so a right reflector touches only the rows within 2w before and w after its
 * range, and a left one only the columns within w before and 2w after it.
 * A: n x n, its upper triangle holds the band (0 <= j-i <= w; the rest is ignored).
 * On return d[0..n) is the diagonal and e[0..n-1) the superdiagonal.
 * Returns 0, -i for an invalid i-th argument, -100 when out of memory.
 * ---------------------------------------------------------------------------------*/
int oracle_gb2bd(int64_t n, int64_t w, const double *A, int64_t lda, double *d, double *e) {
    if (n < 0) return -1;
    if (w < 1) return -2;
    if (lda < (n > 1 ? n : 1)) return -4;
    if (n == 0) return 0;
    double *M = (double *)calloc((size_t)n * (size_t)n, sizeof(double));
    double *v = (double *)malloc(sizeof(double) * (size_t)(w + 1));
    if (!M || !v) { free(M); free(v); return -100; }
    for (int64_t j = 0; j < n; ++j)
        for (int64_t i = (j - w > 0 ? j - w : 0); i <= j; ++i) AT(M, n, i, j) = AT(A, lda, i, j);
    for (int64_t c = 0; c + 1 < n; ++c) {
        int64_t r = c, a = c + 1;
        while (a < n) {
            int64_t end = a + w < n ? a + w : n;
            int64_t len = end - a;
            if (len < 2) break;
            double t;
            /* right: from row r, columns [a, end), applied to rows [a - 2w, end + w) */
            house(len, &AT(M, n, r, a), n, &t);
            if (t != 0.0) {
                v[0] = 1.0;
                for (int64_t k = 1; k < len; ++k) v[k] = AT(M, n, r, a + k);
                int64_t lo = a - 2 * w > 0 ? a - 2 * w : 0, hi = end + w < n ? end + w : n;
                for (int64_t i = lo; i < hi; ++i) {
                    if (i == r) continue;
                    double z = 0.0;
                    for (int64_t k = 0; k < len; ++k) z += AT(M, n, i, a + k) * v[k];
                    z *= t;
                    for (int64_t k = 0; k < len; ++k) AT(M, n, i, a + k) -= z * v[k];
                }
            }
            for (int64_t k = 1; k < len; ++k) AT(M, n, r, a + k) = 0.0;
            /* left: from column a, rows [a, end), applied to columns [a - w, end + 2w) */
            house(len, &AT(M, n, a, a), 1, &t);
            if (t != 0.0) {
                v[0] = 1.0;
                for (int64_t i = 1; i < len; ++i) v[i] = AT(M, n, a + i, a);
                int64_t lo = a - w > 0 ? a - w : 0, hi = end + 2 * w < n ? end + 2 * w : n;
                for (int64_t j = lo; j < hi; ++j) {
                    if (j == a) continue;
                    double z = 0.0;
                    for (int64_t i = 0; i < len; ++i) z += v[i] * AT(M, n, a + i, j);
                    z *= t;
                    for (int64_t i = 0; i < len; ++i) AT(M, n, a + i, j) -= z * v[i];
                }
            }
            for (int64_t i = 1; i < len; ++i) AT(M, n, a + i, a) = 0.0;
            r = a;
            a += w;
        }
    }
    for (int64_t i = 0; i < n; ++i) d[i] = AT(M, n, i, i);
    for (int64_t i = 0; i + 1 < n; ++i) e[i] = AT(M, n, i, i + 1);
    free(M);
    free(v);
    return 0;
}

/* Singular values of the upper bidiagonal B = (d, e), descending: the eigenvalues of the
 * Golub-Kahan tridiagonal of order 2n (zero diagonal, off-diagonal d_0, e_0, d_1, e_1,
 * ..., d_{n-1}) are +-sigma_k, so its n largest, by the bisection above, are the singular
 * values.  Returns 0, -i for an invalid i-th argument, -100 when out of memory. */
int oracle_bd_singular_values(int64_t n, const double *d, const double *e, double *sig) {
    if (n < 0) return -1;
    if (n == 0) return 0;
    double *z = (double *)calloc((size_t)(2 * n), sizeof(double));
    double *o = (double *)calloc((size_t)(2 * n), sizeof(double));
    double *lam = (double *)malloc(sizeof(double) * (size_t)(2 * n));
    if (!z || !o || !lam) { free(z); free(o); free(lam); return -100; }
    for (int64_t i = 0; i < n; ++i) {
        o[2 * i] = d[i];
        if (i + 1 < n) o[2 * i + 1] = e[i];
    }
    int info = oracle_tridiag_eig(2 * n, z, o, lam);
    for (int64_t k = 0; k < n && info == 0; ++k) sig[k] = lam[2 * n - 1 - k];
    free(z);
    free(o);
    free(lam);
    return info;
}
