/*
 * Plain FP64 CPU oracle for the inverse-overlap factorization Z Z^T = S^{-1}.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code with the CUDA library.
 *
 * Everything is row-major, N x N, double precision, written as the plain
 * definitions: triple loops in i-k-j order (OpenMP over rows), no blocking,
 * no fusion.  Citations are to arXiv:2404.19163 (Habib, Finkelstein,
 * Niklasson).
 *
 * Notation (Sec. 3, Eq. np1 and the delta-form that follows Algorithm 1):
 *   X_n   = Z_n^T S Z_n
 *   d_n   = I - X_n                      (sign convention: d = I - X)
 *   p(d)  = sum_{k=0..m} c_k d^k,  c_k = binom(2k,k)/4^k
 *           (the Taylor series of (1-t)^{-1/2}; for m = 2 this is
 *            I + d/2 + 3 d^2/8, identical to a0 I + a1 X + a2 X^2 with the
 *            Appendix A coefficients a = 15/8, -5/4, 3/8)
 *   Z_{n+1} = Z_n p(d_n) = Z_n + Z_n Q_n,   Q_n = p(d_n) - I
 *   Err_n = ||X_n - I||_F                (Algorithm 2)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int zo_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void zo_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* C = A B (N x N), plain i-k-j triple loop. */
void zo_matmul(const double* A, const double* B, double* C, int64_t n) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double* c = C + i * n;
        for (int64_t j = 0; j < n; ++j) c[j] = 0.0;
        for (int64_t k = 0; k < n; ++k) {
            const double a = A[i * n + k];
            const double* b = B + k * n;
            for (int64_t j = 0; j < n; ++j) c[j] += a * b[j];
        }
    }
}

/* C = A^T B (N x N): C_ij = sum_k A_ki B_kj, evaluated for i <= j only and
 * mirrored, because the result is symmetric in exact arithmetic when B = S A
 * with S symmetric (the paper's X = Z^T S Z, Sec. 3.2, Eq. Xn).  The
 * upper-triangle-and-mirror definition is the one the GPU path also uses. */
void zo_atb_sym(const double* A, const double* B, double* C, int64_t n) {
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i; j < n; ++j) {
            double s = 0.0;
            for (int64_t k = 0; k < n; ++k) s += A[k * n + i] * B[k * n + j];
            C[i * n + j] = s;
        }
    }
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < i; ++j) C[i * n + j] = C[j * n + i];
}

/* d = I - Z^T S Z (upper triangle mirrored); returns ||d||_F.
 * Eq. np1 second line, and Err = ||X - I||_F of Algorithm 2. */
double zo_residual(const double* S, const double* Z, double* d, int64_t n) {
    double* A = (double*)malloc(sizeof(double) * n * n);
    zo_matmul(S, Z, A, n);           /* A = S Z */
    zo_atb_sym(Z, A, d, n);          /* X = Z^T A */
    double ss = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = 0; j < n; ++j) {
            double v = (i == j ? 1.0 : 0.0) - d[i * n + j];
            d[i * n + j] = v;
            ss += v * v;
        }
    }
    free(A);
    return sqrt(ss);
}

/* H_perp = Z^T H Z (upper triangle mirrored): the congruence transform of Sec. 2
 * (Eq. standard_form, H_perp = Z^T H Z) that turns H C = S C e into a standard
 * eigenproblem once Z^T S Z = I. */
void zo_congruence(const double* H, const double* Z, double* Hp, int64_t n) {
    double* A = (double*)malloc(sizeof(double) * n * n);
    zo_matmul(H, Z, A, n);           /* A = H Z */
    zo_atb_sym(Z, A, Hp, n);         /* Z^T A */
    free(A);
}

/* c_k = binom(2k, k) / 4^k, k = 0..m (Taylor coefficients of (1-t)^{-1/2}). */
void zo_coeffs(int m, double* c) {
    c[0] = 1.0;
    for (int k = 1; k <= m; ++k) c[k] = c[k - 1] * (double)(2 * k - 1) / (double)(2 * k);
}

/* Q = p_m(d) - I = sum_{k=1..m} c_k d^k, by explicit powers P_k = P_{k-1} d. */
void zo_poly(const double* d, int m, double* Q, int64_t n) {
    double c[8];
    zo_coeffs(m, c);
    double* P = (double*)malloc(sizeof(double) * n * n);
    double* T = (double*)malloc(sizeof(double) * n * n);
    memcpy(P, d, sizeof(double) * n * n);
    for (int64_t e = 0; e < n * n; ++e) Q[e] = c[1] * d[e];
    for (int k = 2; k <= m; ++k) {
        zo_matmul(P, d, T, n);
        memcpy(P, T, sizeof(double) * n * n);
        for (int64_t e = 0; e < n * n; ++e) Q[e] += c[k] * P[e];
    }
    free(P);
    free(T);
}

/* Z <- Z + Z Q  (Z_{n+1} = Z_n p(d_n)). */
void zo_update(double* Z, const double* Q, int64_t n) {
    double* T = (double*)malloc(sizeof(double) * n * n);
    zo_matmul(Z, Q, T, n);
    for (int64_t e = 0; e < n * n; ++e) Z[e] += T[e];
    free(T);
}

/* Z0 = I / sqrt(max_i sum_j |S_ij|): Gershgorin bound on lambda_max, so that
 * X0 = Z0^T S Z0 has spectrum in (0, 1] and ||X0 - I||_2 < 1 (Sec. 3, the
 * convergence condition after Eq. np1). */
double zo_gershgorin_scale(const double* S, int64_t n) {
    double mx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double r = 0.0;
        for (int64_t j = 0; j < n; ++j) r += fabs(S[i * n + j]);
        if (r > mx) mx = r;
    }
    return 1.0 / sqrt(mx);
}

/* Stop decision after Err[i] has been formed, i >= 1.
 *   rule 0: Algorithm 2, break when Err[i] > Err[i-1]^3, plus two guards the
 *           paper leaves implicit: Err[i] >= Err[i-1] (no longer decreasing)
 *           and a non-finite Err.
 *   rule 1: Algorithm 1, break when Err[i] / sqrt(N) <= tol. */
static int zo_should_stop(int rule, double cur, double prev, double tol, int64_t n) {
    if (!isfinite(cur)) return 1;
    if (rule == 1) return cur / sqrt((double)n) <= tol;
    if (cur > prev * prev * prev) return 1;
    if (cur >= prev) return 1;
    return 0;
}

/* Algorithm 2 (and Algorithm 1 with rule 1) in FP64.
 *   Z0 == NULL: Gershgorin-scaled identity.
 *   fixed_iters > 0: perform exactly that many updates, no stop test.
 * Writes Z, hist[0..iters] (Err of every iterate, hist[0] = ||d_0||_F),
 * returns the number of updates performed, or -1 for a non-finite Err. */
int zo_refine(const double* S, const double* Z0, int64_t n, int m, int nmax,
              int fixed_iters, int rule, double tol,
              double* Z, double* hist, int hist_cap) {
    double* d = (double*)malloc(sizeof(double) * n * n);
    double* Q = (double*)malloc(sizeof(double) * n * n);
    if (Z0) {
        memcpy(Z, Z0, sizeof(double) * n * n);
    } else {
        const double s = zo_gershgorin_scale(S, n);
        for (int64_t e = 0; e < n * n; ++e) Z[e] = 0.0;
        for (int64_t i = 0; i < n; ++i) Z[i * n + i] = s;
    }
    double err = zo_residual(S, Z, d, n);
    if (hist_cap > 0) hist[0] = err;
    int it = 0;
    int status = 0;
    const int limit = fixed_iters > 0 ? fixed_iters : nmax;
    if (!isfinite(err)) status = -1;
    if (rule == 1 && fixed_iters <= 0 && err / sqrt((double)n) <= tol) goto done;
    while (status == 0 && it < limit) {
        zo_poly(d, m, Q, n);
        zo_update(Z, Q, n);
        const double prev = err;
        err = zo_residual(S, Z, d, n);
        ++it;
        if (it < hist_cap) hist[it] = err;
        if (!isfinite(err)) { status = -1; break; }
        if (fixed_iters <= 0 && zo_should_stop(rule, err, prev, tol, n)) break;
    }
done:
    free(d);
    free(Q);
    return status < 0 ? -1 : it;
}
