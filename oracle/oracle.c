/*
 * oracle.c -- the CPU oracle for U = sign(T), T real upper triangular.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path links, loads or calls
 * this file; only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header, table or helper with the CUDA
 * library.
 *
 * Storage: column-major float64, element (i,j) at M[i + j*ld], 0-based.
 * Compile with -ffp-contract=off (the build script does) so that every a*b and
 * every + below is one separately rounded IEEE operation: the rounding of the
 * oracle is then fixed by the order written here.
 *
 * Functions
 *   oracle_sign_tri        Parlett-Higham substitution (the method of the
 *                          paper's Section 3; Higham's Algorithm 5.5), derived
 *                          below from entry (i,j) of TU = UT (Eq. 1) and of
 *                          U^2 = I (Eq. 2).  Entry (i,j) needs the entries
 *                          (i,k) and (k,j) with i < k < j, so columns are
 *                          visited left to right and each column bottom to
 *                          top: j = 2..n outer, i = j-1..1 inner.
 *   oracle_sign_tri_count  Same, and counts the floating-point operations that
 *                          the inner sums execute (the useful-flop count).
 *   oracle_sign_tri_antidiag
 *                          Same per-entry arithmetic as oracle_sign_tri, but
 *                          entries are visited by anti-diagonal d = j-i, whose
 *                          entries depend only on entries with smaller d; the
 *                          entries of one anti-diagonal may run in parallel
 *                          (OpenMP).  The result is bit-identical to
 *                          oracle_sign_tri (a test checks this).
 *   oracle_sign_schur      The Schur route of Section 1 (and Algorithm 3's
 *                          first step) for a real Schur pair: with
 *                          A = Q T Q^T, Q orthogonal, T upper triangular,
 *                          sign(A) = Q U Q^T where U = sign(T) from
 *                          oracle_sign_tri_antidiag; then W = U Q^T and
 *                          S = Q W, each entry one plain sum over k ascending.
 *   oracle_sign_tri_complex, oracle_sign_schur_complex
 *                          The same substitution and route for a complex
 *                          upper triangular T (the paper's Schur form is
 *                          complex in general, Algorithm 3's first step):
 *                          u_ii = sign(Re t_ii) (Section 1: sign is defined
 *                          off the imaginary axis), then Eq. 1 / Eq. 2 entry
 *                          by entry in the order of oracle_sign_tri, in C99
 *                          complex arithmetic; S = Q U Q^H for unitary Q.
 *                          Matrices interleaved (re, im) column-major.
 *   oracle_funm            Parlett's substitution for a general function
 *                          phi (Section 2, Algorithm 1): f_ii = phi(t_ii),
 *                          then entry (i,j) of TF = FT solved for f_ij,
 *                          (t_ii - t_jj) f_ij = t_ij (f_ii - f_jj)
 *                                + sum_{i<k<j} (f_ik t_kj - t_ik f_kj),
 *                          in the order of oracle_sign_tri.  phi: 1 exp,
 *                          2 log (t_ii > 0), 3 sqrt (t_ii > 0), 4 sign
 *                          (the sign function through Eq. 1 alone).  Needs
 *                          distinct diagonal entries.
 *   oracle_sign_spectral   Brute force from the definition in Section 1:
 *                          sign(T) = Z sign(D) Z^{-1}, with Z the (unit upper
 *                          triangular) eigenvector matrix of T, in long double.
 *                          For small n only.
 *
 * Status codes: 0 ok, 1 bad argument, 2 a diagonal entry is zero (sign(0) is
 * undefined, Section 1), 3 a diagonal entry is NaN or infinite.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_OK 0
#define ORACLE_BAD_ARG 1
#define ORACLE_ZERO_EIGENVALUE 2
#define ORACLE_NONFINITE 3

#define AT(M, ld, i, j) ((M)[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

/* Scalar sign of Section 1 for a real nonzero argument. */
static double scalar_sign(double x) { return x > 0.0 ? 1.0 : -1.0; }

static int check_args(int n, const double *T, int ldt, const double *U, int ldu)
{
    if (n < 0 || ldt < (n > 1 ? n : 1) || ldu < (n > 1 ? n : 1)) return ORACLE_BAD_ARG;
    if (n > 0 && (T == NULL || U == NULL)) return ORACLE_BAD_ARG;
    for (int i = 0; i < n; i++) {
        double t = AT(T, ldt, i, i);
        if (!isfinite(t)) return ORACLE_NONFINITE;
        if (t == 0.0) return ORACLE_ZERO_EIGENVALUE;
    }
    return ORACLE_OK;
}

/*
 * Parlett-Higham substitution.  For i < j, entry (i,j) of TU = UT (Eq. 1),
 * with U and T upper triangular, reads
 *       t_ii u_ij + t_ij u_jj + sum_{i<k<j} t_ik u_kj
 *     = u_ii t_ij + u_ij t_jj + sum_{i<k<j} u_ik t_kj,
 * and entry (i,j) of U^2 = I (Eq. 2) reads
 *       u_ii u_ij + u_ij u_jj + sum_{i<k<j} u_ik u_kj = 0.
 * The second fixes u_ij whenever u_ii + u_jj != 0 (equal signs, |u_ii +
 * u_jj| = 2); when the signs differ it is empty and the first is used, its
 * divisor t_ii - t_jj being nonzero then:
 *   if u_ii + u_jj = 0 (signs differ), from Eq. 1:
 *       u_ij = t_ij (u_ii - u_jj)/(t_ii - t_jj)
 *              + [sum_{k=i+1}^{j-1} (u_ik t_kj - t_ik u_kj)] / (t_ii - t_jj)
 *   else, from Eq. 2:
 *       u_ij = -[sum_{k=i+1}^{j-1} u_ik u_kj] / (u_ii + u_jj)
 * The strictly lower triangle of U is set to zero.
 * inner_flops, when not NULL, receives the number of floating-point
 * operations executed by the inner sums: 2 per term of the U^2 = I sum
 * (one multiply, one add) and 4 per term of the TU = UT sum (two multiplies,
 * one subtract, one add).
 */
int oracle_sign_tri_count(int n, const double *T, int ldt, double *U, int ldu,
                          long long *inner_flops)
{
    int st = check_args(n, T, ldt, U, ldu);
    if (st != ORACLE_OK) return st;
    long long flops = 0;
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) AT(U, ldu, i, j) = 0.0;
    for (int i = 0; i < n; i++) AT(U, ldu, i, i) = scalar_sign(AT(T, ldt, i, i));
    for (int j = 1; j < n; j++) {
        for (int i = j - 1; i >= 0; i--) {
            double uii = AT(U, ldu, i, i), ujj = AT(U, ldu, j, j);
            if (uii + ujj == 0.0) {
                double s = 0.0;
                for (int k = i + 1; k <= j - 1; k++) {
                    double a = AT(U, ldu, i, k) * AT(T, ldt, k, j);
                    double b = AT(T, ldt, i, k) * AT(U, ldu, k, j);
                    s = s + (a - b);
                }
                flops += 4LL * (j - i - 1);
                double den = AT(T, ldt, i, i) - AT(T, ldt, j, j);
                AT(U, ldu, i, j) = AT(T, ldt, i, j) * (uii - ujj) / den + s / den;
            } else {
                double s = 0.0;
                for (int k = i + 1; k <= j - 1; k++) s = s + AT(U, ldu, i, k) * AT(U, ldu, k, j);
                flops += 2LL * (j - i - 1);
                AT(U, ldu, i, j) = -s / (uii + ujj);
            }
        }
    }
    if (inner_flops) *inner_flops = flops;
    return ORACLE_OK;
}

int oracle_sign_tri(int n, const double *T, int ldt, double *U, int ldu)
{
    return oracle_sign_tri_count(n, T, ldt, U, ldu, NULL);
}

/*
 * The same entries, visited by anti-diagonal d = j - i = 1..n-1.  Entry (i,j)
 * reads u_ik (k < j, anti-diagonal k-i < d) and u_kj (k > i, anti-diagonal
 * j-k < d), so every entry of anti-diagonal d can be computed once all
 * smaller anti-diagonals are done.  Row-major copies UR, TR give contiguous
 * access to the rows u_i*, t_i*; they hold the same values as U and T, and
 * each entry performs exactly the operations of oracle_sign_tri in the same
 * order, so the results are bit-identical.
 * nthreads <= 0 uses the OpenMP default.
 */
int oracle_sign_tri_antidiag(int n, const double *T, int ldt, double *U, int ldu, int nthreads)
{
    int st = check_args(n, T, ldt, U, ldu);
    if (st != ORACLE_OK) return st;
    size_t nn = (size_t)n * (size_t)n;
    double *UR = (double *)calloc(nn > 0 ? nn : 1, sizeof(double));
    double *TR = (double *)calloc(nn > 0 ? nn : 1, sizeof(double));
    if (!UR || !TR) { free(UR); free(TR); return ORACLE_BAD_ARG; }
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            AT(U, ldu, i, j) = 0.0;
            TR[(size_t)i * n + j] = (i <= j) ? AT(T, ldt, i, j) : 0.0;
        }
    for (int i = 0; i < n; i++) {
        double u = scalar_sign(AT(T, ldt, i, i));
        AT(U, ldu, i, i) = u;
        UR[(size_t)i * n + i] = u;
    }
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    for (int d = 1; d < n; d++) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int i = 0; i < n - d; i++) {
            int j = i + d;
            const double *urow = UR + (size_t)i * n;
            const double *trow = TR + (size_t)i * n;
            const double *ucol = &AT(U, ldu, 0, j);
            const double *tcol = &AT(T, ldt, 0, j);
            double uii = urow[i], ujj = UR[(size_t)j * n + j];
            double uij;
            if (uii + ujj == 0.0) {
                double s = 0.0;
                for (int k = i + 1; k <= j - 1; k++) {
                    double a = urow[k] * tcol[k];
                    double b = trow[k] * ucol[k];
                    s = s + (a - b);
                }
                double den = trow[i] - TR[(size_t)j * n + j];
                uij = tcol[i] * (uii - ujj) / den + s / den;
            } else {
                double s = 0.0;
                for (int k = i + 1; k <= j - 1; k++) s = s + urow[k] * ucol[k];
                uij = -s / (uii + ujj);
            }
            AT(U, ldu, i, j) = uij;
            UR[(size_t)i * n + j] = uij;
        }
    }
    free(UR);
    free(TR);
    return ORACLE_OK;
}

/*
 * Brute force from the spectral definition (Section 1): for T with distinct
 * diagonal entries, T = Z D Z^{-1} with D = diag(t_ii) and Z unit upper
 * triangular, column j solving (T - t_jj I) z = 0 with z_jj = 1:
 *     z_ij = [sum_{k=i+1}^{j} t_ik z_kj] / (t_jj - t_ii),   i = j-1, ..., 1.
 * W = Z^{-1} is unit upper triangular, from Z W = I column by column:
 *     w_ij = -sum_{k=i+1}^{j} z_ik w_kj.
 * Then sign(T) = Z diag(sign(t_ii)) W.  All in long double.  Requires
 * distinct diagonal entries; n <= 64.
 */
int oracle_sign_spectral(int n, const double *T, int ldt, double *U, int ldu)
{
    int st = check_args(n, T, ldt, U, ldu);
    if (st != ORACLE_OK) return st;
    if (n > 64) return ORACLE_BAD_ARG;
    long double Z[64][64], W[64][64];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) { Z[i][j] = 0.0L; W[i][j] = 0.0L; }
    for (int j = 0; j < n; j++) {
        Z[j][j] = 1.0L;
        for (int i = j - 1; i >= 0; i--) {
            long double s = 0.0L;
            for (int k = i + 1; k <= j; k++) s += (long double)AT(T, ldt, i, k) * Z[k][j];
            long double den = (long double)AT(T, ldt, j, j) - (long double)AT(T, ldt, i, i);
            if (den == 0.0L) return ORACLE_BAD_ARG;
            Z[i][j] = s / den;
        }
    }
    for (int j = 0; j < n; j++) {
        W[j][j] = 1.0L;
        for (int i = j - 1; i >= 0; i--) {
            long double s = 0.0L;
            for (int k = i + 1; k <= j; k++) s += Z[i][k] * W[k][j];
            W[i][j] = -s;
        }
    }
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) {
            long double s = 0.0L;
            for (int k = i; k <= j; k++)
                s += Z[i][k] * (long double)scalar_sign(AT(T, ldt, k, k)) * W[k][j];
            AT(U, ldu, i, j) = (i <= j) ? (double)s : 0.0;
        }
    return ORACLE_OK;
}

int oracle_sign_schur(int n, const double *Q, int ldq, const double *T, int ldt, double *S, int lds, int nthreads)
{
    if (n < 0 || ldq < (n > 1 ? n : 1) || lds < (n > 1 ? n : 1)) return ORACLE_BAD_ARG;
    if (n > 0 && (Q == NULL || S == NULL)) return ORACLE_BAD_ARG;
    size_t nn = (size_t)n * (size_t)n;
    double *U = (double *)calloc(nn > 0 ? nn : 1, sizeof(double));
    double *W = (double *)calloc(nn > 0 ? nn : 1, sizeof(double));
    if (!U || !W) { free(U); free(W); return ORACLE_BAD_ARG; }
    int st = oracle_sign_tri_antidiag(n, T, ldt, U, n > 1 ? n : 1, nthreads);
    if (st == ORACLE_OK) {
        /* W(:, j) = sum_k U(:, k) Q(j, k)  (W = U Q^T) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int j = 0; j < n; j++) {
            double *w = W + (size_t)j * n;
            for (int k = 0; k < n; k++) {
                const double q = AT(Q, ldq, j, k);
                const double *u = U + (size_t)k * n;
                for (int i = 0; i < n; i++) w[i] = w[i] + u[i] * q;
            }
        }
        /* S(:, j) = sum_k Q(:, k) W(k, j)  (S = Q W) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int j = 0; j < n; j++) {
            double *sc = &AT(S, lds, 0, j);
            for (int i = 0; i < n; i++) sc[i] = 0.0;
            for (int k = 0; k < n; k++) {
                const double wkj = W[(size_t)j * n + k];
                const double *q = &AT(Q, ldq, 0, k);
                for (int i = 0; i < n; i++) sc[i] = sc[i] + q[i] * wkj;
            }
        }
    }
    free(U);
    free(W);
    return st;
}

/*
 * Complex T (interleaved re, im; element (i,j) at 2 (i + j ld)).  Status 2
 * when some Re t_ii == 0 (sign undefined on the imaginary axis, Section 1),
 * 3 when some t_ii is not finite.  Per entry the arithmetic of
 * oracle_sign_tri with complex operands: for differing signs the divisor
 * t_ii - t_jj has real parts of opposite sign, hence is nonzero.
 */
#define CAT(M, ld, i, j) (((double complex *)(M))[(size_t)(i) + (size_t)(j) * (size_t)(ld)])

int oracle_sign_tri_complex(int n, const double *T, int ldt, double *U, int ldu)
{
    if (n < 0 || ldt < (n > 1 ? n : 1) || ldu < (n > 1 ? n : 1)) return ORACLE_BAD_ARG;
    if (n > 0 && (T == NULL || U == NULL)) return ORACLE_BAD_ARG;
    for (int i = 0; i < n; i++) {
        double complex t = CAT(T, ldt, i, i);
        if (!isfinite(creal(t)) || !isfinite(cimag(t))) return ORACLE_NONFINITE;
        if (creal(t) == 0.0) return ORACLE_ZERO_EIGENVALUE;
    }
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) CAT(U, ldu, i, j) = 0.0;
    for (int i = 0; i < n; i++) CAT(U, ldu, i, i) = scalar_sign(creal(CAT(T, ldt, i, i)));
    for (int j = 1; j < n; j++) {
        for (int i = j - 1; i >= 0; i--) {
            double complex uii = CAT(U, ldu, i, i), ujj = CAT(U, ldu, j, j);
            if (uii + ujj == 0.0) {
                double complex s = 0.0;
                for (int k = i + 1; k <= j - 1; k++) {
                    double complex a = CAT(U, ldu, i, k) * CAT(T, ldt, k, j);
                    double complex b = CAT(T, ldt, i, k) * CAT(U, ldu, k, j);
                    s = s + (a - b);
                }
                double complex den = CAT(T, ldt, i, i) - CAT(T, ldt, j, j);
                CAT(U, ldu, i, j) = CAT(T, ldt, i, j) * (uii - ujj) / den + s / den;
            } else {
                double complex s = 0.0;
                for (int k = i + 1; k <= j - 1; k++) s = s + CAT(U, ldu, i, k) * CAT(U, ldu, k, j);
                CAT(U, ldu, i, j) = -s / (uii + ujj);
            }
        }
    }
    return ORACLE_OK;
}

/* S = Q U Q^H, U = sign(T), Q unitary: W = U Q^H, then S = Q W, each entry
   one plain sum over k ascending. */
int oracle_sign_schur_complex(int n, const double *Q, int ldq, const double *T, int ldt, double *S, int lds)
{
    if (n < 0 || ldq < (n > 1 ? n : 1) || lds < (n > 1 ? n : 1)) return ORACLE_BAD_ARG;
    if (n > 0 && (Q == NULL || S == NULL)) return ORACLE_BAD_ARG;
    size_t nn = (size_t)n * (size_t)n;
    double complex *U = (double complex *)calloc(nn > 0 ? nn : 1, sizeof(double complex));
    double complex *W = (double complex *)calloc(nn > 0 ? nn : 1, sizeof(double complex));
    if (!U || !W) { free(U); free(W); return ORACLE_BAD_ARG; }
    int st = oracle_sign_tri_complex(n, T, ldt, (double *)U, n > 1 ? n : 1);
    if (st == ORACLE_OK) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int j = 0; j < n; j++) {
            double complex *w = W + (size_t)j * n;
            for (int k = 0; k < n; k++) {
                const double complex q = conj(CAT(Q, ldq, j, k));
                const double complex *u = U + (size_t)k * n;
                for (int i = 0; i < n; i++) w[i] = w[i] + u[i] * q;
            }
        }
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
        for (int j = 0; j < n; j++) {
            double complex *sc = &CAT(S, lds, 0, j);
            for (int i = 0; i < n; i++) sc[i] = 0.0;
            for (int k = 0; k < n; k++) {
                const double complex wkj = W[(size_t)j * n + k];
                const double complex *q = &CAT(Q, ldq, 0, k);
                for (int i = 0; i < n; i++) sc[i] = sc[i] + q[i] * wkj;
            }
        }
    }
    free(U);
    free(W);
    return st;
}

/*
 * Status 1 also for a repeated diagonal entry (Algorithm 1 divides by
 * t_ii - t_jj) and for a phi outside its domain (log, sqrt of t_ii <= 0).
 */
static double scalar_phi(int phi, double x)
{
    switch (phi) {
    case 1: return exp(x);
    case 2: return log(x);
    case 3: return sqrt(x);
    default: return scalar_sign(x);
    }
}

int oracle_funm(int n, const double *T, int ldt, double *F, int ldf, int phi)
{
    int st = check_args(n, T, ldt, F, ldf);
    if (st != ORACLE_OK) return st;
    if (phi < 1 || phi > 4) return ORACLE_BAD_ARG;
    for (int i = 0; i < n; i++) {
        if ((phi == 2 || phi == 3) && !(AT(T, ldt, i, i) > 0.0)) return ORACLE_BAD_ARG;
        for (int j = i + 1; j < n; j++)
            if (AT(T, ldt, i, i) == AT(T, ldt, j, j)) return ORACLE_BAD_ARG;
    }
    for (int j = 0; j < n; j++)
        for (int i = 0; i < n; i++) AT(F, ldf, i, j) = 0.0;
    for (int i = 0; i < n; i++) AT(F, ldf, i, i) = scalar_phi(phi, AT(T, ldt, i, i));
    for (int j = 1; j < n; j++) {
        for (int i = j - 1; i >= 0; i--) {
            double s = 0.0;
            for (int k = i + 1; k <= j - 1; k++) {
                double a = AT(F, ldf, i, k) * AT(T, ldt, k, j);
                double b = AT(T, ldt, i, k) * AT(F, ldf, k, j);
                s = s + (a - b);
            }
            double den = AT(T, ldt, i, i) - AT(T, ldt, j, j);
            AT(F, ldf, i, j) = (AT(T, ldt, i, j) * (AT(F, ldf, i, i) - AT(F, ldf, j, j)) + s) / den;
        }
    }
    return ORACLE_OK;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
