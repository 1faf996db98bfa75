/*
 * Plain FP64 CPU oracle for the projected density matrix D = f(Hp).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is compiled into a separate shared
 * library that only the test suite, the smoke check and the benchmark's CPU
 * baseline load.  It shares no code, header or constant with the GPU library,
 * and the GPU library never calls it.
 *
 * Paper: Khadatkar & Motamarri, "Subspace recursive Fermi-operator expansion
 * strategies for large-scale DFT eigenvalue problems on HPC architectures"
 * (arXiv 2301.04642).
 *
 * What is defined here, each function citing the passage it follows:
 *   - Sec. II-A: the zero-temperature density matrix D = theta(mu I - H)
 *     (projector onto the N_occ lowest eigenvectors) and the finite-
 *     temperature one D = [exp(beta (H - mu I)) + I]^{-1}.  Both are formed
 *     from an explicit eigendecomposition H = Q diag(lambda) Q^T, which is
 *     computed by this file's own Householder tridiagonalisation + implicit
 *     QL, or by cyclic Jacobi (the two cross-check each other).
 *   - Sec. II-B1, Eq. (1): SP2 recursion X_{n+1} = X_n +/- (X_n - X_n^2)
 *     with the sign picked so that the trace moves toward N_occ.
 *   - Sec. III-B: tr(X^2) evaluated as the squared Frobenius norm.
 *   - Sec. III-C: error metrics eps1 and eps2.
 *   - Sec. III-A: the plain products either side of the expansion in
 *     subspace iteration (Rayleigh-Ritz projection, rotation by D).
 *   - Sec. II-C: spectral bounds, taken as Gershgorin discs.
 *   - Finite temperature (Sec. II-B3, Eq. (2)): a recursive expansion that
 *     doubles the inverse temperature at every step, z <- 2 z (I + z^2)^{-1}
 *     with z = I - 2D = tanh(beta (H - mu)/2) (the paper's truncated form
 *     stops short of Fermi-Dirac; this one converges to it).  The inverse is
 *     a plain Cholesky solve.
 *   - Sec. II-B2: accelerated SP2 (A-Z-RFOE), read as the SP2 polynomials
 *     shifted and scaled with bounds on the HOMO and LUMO eigenvalues.
 *   - Sec. II-B3, Eq. (2), as printed: the truncated SP2 expansion G_m(H)
 *     (T-RFOE), with m read as the first step whose step function is as
 *     steep as Fermi-Dirac at the Fermi level.
 *
 * All matrices are dense, row-major, n x n, FP64.  No blocking or fusion
 * beyond what each definition states; the only parallelism is an OpenMP loop
 * over output rows in the plain matrix products.
 */
#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdint.h>

#define IDX(i, j, n) ((size_t)(i) * (size_t)(n) + (size_t)(j))

/* ------------------------------------------------------------------ */
/* small helpers                                                        */
/* ------------------------------------------------------------------ */

/* C = A * B, all n x n row-major.  Plain triple loop (i, k, j order). */
void oracle_matmul(int n, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        double *ci = C + IDX(i, 0, n);
        for (int j = 0; j < n; ++j) ci[j] = 0.0;
        for (int k = 0; k < n; ++k) {
            const double a = A[IDX(i, k, n)];
            const double *bk = B + IDX(k, 0, n);
            for (int j = 0; j < n; ++j) ci[j] += a * bk[j];
        }
    }
}

/* C (m x n) = op(A) op(B), op(X) = X or X^T (ta, tb), inner dimension k;
 * A is stored m x k (or k x m when ta), B k x n (or n x k when tb), all
 * row-major with the given leading dimensions.  Plain loops over k for each
 * entry of C (the products either side of the expansion in subspace
 * iteration, Sec. III-A: Psi^T (H Psi) and Psi D). */
void oracle_gemm(int m, int n, int k, const double *A, int lda, int ta, const double *B, int ldb, int tb,
                 double *C, int ldc)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int p = 0; p < k; ++p) {
                const double a = ta ? A[(size_t)p * lda + i] : A[(size_t)i * lda + p];
                const double b = tb ? B[(size_t)j * ldb + p] : B[(size_t)p * ldb + j];
                s += a * b;
            }
            C[(size_t)i * ldc + j] = s;
        }
}

double oracle_trace(int n, const double *A)
{
    double t = 0.0;
    for (int i = 0; i < n; ++i) t += A[IDX(i, i, n)];
    return t;
}

/* sum_ij A_ij B_ij = tr(A B) for symmetric A, B */
double oracle_frob_dot(int n, const double *A, const double *B)
{
    double t = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) t += A[k] * B[k];
    return t;
}

/* ------------------------------------------------------------------ */
/* Gershgorin bounds (Sec. II-C needs eps_1, eps_N)                      */
/* ------------------------------------------------------------------ */
/* emin = min_i (H_ii - sum_{j != i} |H_ij|), emax = max_i (H_ii + ...). */
void oracle_gershgorin(int n, const double *H, double *emin, double *emax)
{
    double lo = INFINITY, hi = -INFINITY;
    for (int i = 0; i < n; ++i) {
        double r = 0.0;
        for (int j = 0; j < n; ++j)
            if (j != i) r += fabs(H[IDX(i, j, n)]);
        const double d = H[IDX(i, i, n)];
        if (d - r < lo) lo = d - r;
        if (d + r > hi) hi = d + r;
    }
    *emin = lo;
    *emax = hi;
}

/* ------------------------------------------------------------------ */
/* Eigensolver 1: Householder reduction to tridiagonal form + implicit  */
/* QL with Wilkinson shifts (textbook symmetric eigenvalue algorithm).   */
/* ------------------------------------------------------------------ */

/* Reduce symmetric A (overwritten) to tridiagonal T = Q^T A Q.
 * diag[0..n-1], off[0..n-2] (off[i] couples i and i+1), Q row-major n x n. */
static void householder_tridiag(int n, double *A, double *diag, double *off,
                                double *Q)
{
    double *v = (double *)malloc(sizeof(double) * n);
    double *p = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Q[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;

    for (int k = 0; k + 2 < n; ++k) {
        /* x = A[k+1:n, k]; build v with v[0] = 1 so that (I - tau v v^T) x = alpha e_1 */
        const int m = n - k - 1;
        double xnorm2 = 0.0;
        for (int r = 0; r < m; ++r) {
            v[r] = A[IDX(k + 1 + r, k, n)];
            xnorm2 += v[r] * v[r];
        }
        const double tail2 = xnorm2 - v[0] * v[0];
        if (tail2 == 0.0) continue; /* column already reduced */
        const double xnorm = sqrt(xnorm2);
        const double alpha = (v[0] >= 0.0) ? -xnorm : xnorm;
        const double v0 = v[0] - alpha;
        for (int r = 1; r < m; ++r) v[r] /= v0;
        v[0] = 1.0;
        double vtv = 1.0;
        for (int r = 1; r < m; ++r) vtv += v[r] * v[r];
        const double tau = 2.0 / vtv;

        /* two-sided update of the trailing block B = A[k+1:, k+1:]:
         * p = tau B v ; w = p - (tau/2)(p.v) v ; B -= v w^T + w v^T */
        for (int r = 0; r < m; ++r) {
            double s = 0.0;
            for (int c = 0; c < m; ++c) s += A[IDX(k + 1 + r, k + 1 + c, n)] * v[c];
            p[r] = tau * s;
        }
        double pv = 0.0;
        for (int r = 0; r < m; ++r) pv += p[r] * v[r];
        const double half = 0.5 * tau * pv;
        for (int r = 0; r < m; ++r) p[r] -= half * v[r];
        for (int r = 0; r < m; ++r)
            for (int c = 0; c < m; ++c)
                A[IDX(k + 1 + r, k + 1 + c, n)] -= v[r] * p[c] + p[r] * v[c];
        /* column k below the subdiagonal becomes (alpha, 0, ..., 0) */
        A[IDX(k + 1, k, n)] = alpha;
        A[IDX(k, k + 1, n)] = alpha;
        for (int r = 1; r < m; ++r) {
            A[IDX(k + 1 + r, k, n)] = 0.0;
            A[IDX(k, k + 1 + r, n)] = 0.0;
        }
        /* accumulate Q <- Q (I - tau v v^T) on columns k+1.. */
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int c = 0; c < m; ++c) s += Q[IDX(i, k + 1 + c, n)] * v[c];
            s *= tau;
            for (int c = 0; c < m; ++c) Q[IDX(i, k + 1 + c, n)] -= s * v[c];
        }
    }
    for (int i = 0; i < n; ++i) diag[i] = A[IDX(i, i, n)];
    for (int i = 0; i + 1 < n; ++i) off[i] = A[IDX(i + 1, i, n)];
    free(v);
    free(p);
}

/* Implicit-shift QL on the symmetric tridiagonal (diag, off), rotating the
 * columns of Q so that on exit A = Q diag(lambda) Q^T.  Returns 0 on success,
 * -1 if an eigenvalue needed more than 60 sweeps. */
static int tridiag_ql(int n, double *diag, double *off, double *Q)
{
    /* e[i] couples i and i+1; e[n-1] = 0 as a sentinel */
    double *e = (double *)malloc(sizeof(double) * n);
    for (int i = 0; i + 1 < n; ++i) e[i] = off[i];
    e[n - 1] = 0.0;
    int status = 0;

    for (int l = 0; l < n; ++l) {
        int sweeps = 0;
        for (;;) {
            /* locate the first negligible coupling at or after l */
            int m = l;
            for (; m + 1 < n; ++m) {
                const double scale = fabs(diag[m]) + fabs(diag[m + 1]);
                if (fabs(e[m]) <= DBL_EPSILON * scale || fabs(e[m]) < 1e-300) break;
            }
            if (m == l) break; /* diag[l] has converged */
            if (++sweeps > 60) { status = -1; break; }

            /* Wilkinson-type shift from the leading 2x2 block at l */
            const double delta = (diag[l + 1] - diag[l]) / (2.0 * e[l]);
            const double rad = hypot(delta, 1.0);
            const double shift = diag[l] - e[l] / (delta + (delta >= 0.0 ? rad : -rad));

            /* chase the bulge from the bottom (row m) up to row l */
            double g = diag[m] - shift;
            double c = 1.0, s = 1.0, pprev = 0.0;
            int early = 0;
            for (int i = m - 1; i >= l; --i) {
                const double f = s * e[i];
                const double b = c * e[i];
                const double r = hypot(f, g);
                e[i + 1] = r;
                if (r == 0.0) { /* underflow: deflate and restart */
                    diag[i + 1] -= pprev;
                    e[m] = 0.0;
                    early = 1;
                    break;
                }
                s = f / r;
                c = g / r;
                const double t = diag[i + 1] - pprev;
                const double rr = (diag[i] - t) * s + 2.0 * c * b;
                pprev = s * rr;
                diag[i + 1] = t + pprev;
                g = c * rr - b;
                /* rotate columns i and i+1 of Q */
                for (int row = 0; row < n; ++row) {
                    const double qi1 = Q[IDX(row, i + 1, n)];
                    const double qi = Q[IDX(row, i, n)];
                    Q[IDX(row, i + 1, n)] = s * qi + c * qi1;
                    Q[IDX(row, i, n)] = c * qi - s * qi1;
                }
            }
            if (early) continue;
            diag[l] -= pprev;
            e[l] = g;
            e[m] = 0.0;
        }
        if (status) break;
    }
    free(e);
    return status;
}

/* Sort eigenpairs ascending (stable insertion sort on indices). */
static void sort_eigpairs(int n, double *w, double *Q)
{
    int *idx = (int *)malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) idx[i] = i;
    for (int i = 1; i < n; ++i) {
        const int key = idx[i];
        int j = i - 1;
        while (j >= 0 && w[idx[j]] > w[key]) { idx[j + 1] = idx[j]; --j; }
        idx[j + 1] = key;
    }
    double *w2 = (double *)malloc(sizeof(double) * n);
    double *Q2 = (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int c = 0; c < n; ++c) {
        w2[c] = w[idx[c]];
        for (int r = 0; r < n; ++r) Q2[IDX(r, c, n)] = Q[IDX(r, idx[c], n)];
    }
    memcpy(w, w2, sizeof(double) * n);
    memcpy(Q, Q2, sizeof(double) * (size_t)n * n);
    free(idx); free(w2); free(Q2);
}

/* H = Q diag(w) Q^T, w ascending, columns of Q are eigenvectors.  H is not
 * modified.  Returns 0 on success. */
int oracle_eigh_ql(int n, const double *H, double *w, double *Q)
{
    if (n == 1) { w[0] = H[0]; Q[0] = 1.0; return 0; }
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *off = (double *)malloc(sizeof(double) * n);
    memcpy(A, H, sizeof(double) * (size_t)n * n);
    householder_tridiag(n, A, w, off, Q);
    const int st = tridiag_ql(n, w, off, Q);
    free(A); free(off);
    if (st == 0) sort_eigpairs(n, w, Q);
    return st;
}

/* ------------------------------------------------------------------ */
/* Eigensolver 2: cyclic Jacobi rotations (cross-check for small n).    */
/* ------------------------------------------------------------------ */
int oracle_eigh_jacobi(int n, const double *H, double *w, double *V, int max_sweeps)
{
    double *A = (double *)malloc(sizeof(double) * (size_t)n * n);
    memcpy(A, H, sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) V[IDX(i, j, n)] = (i == j) ? 1.0 : 0.0;
    double total = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) total += A[k] * A[k];
    int status = -1;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        double offn = 0.0;
        for (int p = 0; p < n; ++p)
            for (int q = p + 1; q < n; ++q) offn += 2.0 * A[IDX(p, q, n)] * A[IDX(p, q, n)];
        if (offn <= 1e-30 * total) { status = 0; break; }
        for (int p = 0; p < n; ++p) {
            for (int q = p + 1; q < n; ++q) {
                const double apq = A[IDX(p, q, n)];
                if (fabs(apq) < 1e-300) continue;
                /* rotation angle that zeroes A_pq: cot(2 phi) = (A_qq - A_pp) / (2 A_pq) */
                const double theta = (A[IDX(q, q, n)] - A[IDX(p, p, n)]) / (2.0 * apq);
                const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                const double c = 1.0 / sqrt(t * t + 1.0);
                const double s = t * c;
                /* A <- J^T A J with J the rotation in the (p, q) plane */
                for (int k = 0; k < n; ++k) {
                    const double akp = A[IDX(k, p, n)], akq = A[IDX(k, q, n)];
                    A[IDX(k, p, n)] = c * akp - s * akq;
                    A[IDX(k, q, n)] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    const double apk = A[IDX(p, k, n)], aqk = A[IDX(q, k, n)];
                    A[IDX(p, k, n)] = c * apk - s * aqk;
                    A[IDX(q, k, n)] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    const double vkp = V[IDX(k, p, n)], vkq = V[IDX(k, q, n)];
                    V[IDX(k, p, n)] = c * vkp - s * vkq;
                    V[IDX(k, q, n)] = s * vkp + c * vkq;
                }
            }
        }
    }
    for (int i = 0; i < n; ++i) w[i] = A[IDX(i, i, n)];
    free(A);
    sort_eigpairs(n, w, V);
    return status;
}

/* ------------------------------------------------------------------ */
/* Occupations (Sec. II-A)                                              */
/* ------------------------------------------------------------------ */

/* Fermi-Dirac occupation 1/(1 + exp((lam - mu)/kT)) without overflow. */
double oracle_fermi(double lam, double mu, double kT)
{
    const double x = (lam - mu) / kT;
    if (x > 0.0) {
        const double e = exp(-x);
        return e / (1.0 + e);
    }
    return 1.0 / (1.0 + exp(x));
}

/* w ascending.  kT == 0: f_i = 1 for the ne lowest states (ne integral),
 * mu = midpoint of the HOMO-LUMO gap.  kT > 0: mu by bisection so that
 * sum f = ne.  Returns mu. */
double oracle_occupations(int n, const double *w, double ne, double kT, double *f)
{
    if (kT == 0.0) {
        const int k = (int)llround(ne);
        for (int i = 0; i < n; ++i) f[i] = (i < k) ? 1.0 : 0.0;
        if (k <= 0) return w[0] - 1.0;
        if (k >= n) return w[n - 1] + 1.0;
        return 0.5 * (w[k - 1] + w[k]);
    }
    double lo = w[0] - 40.0 * kT, hi = w[n - 1] + 40.0 * kT, mu = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        mu = 0.5 * (lo + hi);
        double s = 0.0;
        for (int i = 0; i < n; ++i) s += oracle_fermi(w[i], mu, kT);
        if (fabs(s - ne) < 1e-12 || hi - lo < 1e-15 * (fabs(mu) + 1.0)) break;
        if (s > ne) hi = mu; else lo = mu;
    }
    for (int i = 0; i < n; ++i) f[i] = oracle_fermi(w[i], mu, kT);
    return mu;
}

/* D = Q diag(f) Q^T (columns of Q are eigenvectors). */
void oracle_density_from_eig(int n, const double *Q, const double *f, double *D)
{
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) {
            double s = 0.0;
            for (int k = 0; k < n; ++k) s += Q[IDX(i, k, n)] * f[k] * Q[IDX(j, k, n)];
            D[IDX(i, j, n)] = s;
        }
    }
}

/* One entry D_ij = sum_k Q_ik f_k Q_jk, for sampled checks at large n. */
double oracle_density_entry(int n, const double *Q, const double *f, int i, int j)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += Q[IDX(i, k, n)] * f[k] * Q[IDX(j, k, n)];
    return s;
}

/* Full oracle: eigendecompose H, occupy, form D.  Returns status (0 ok).
 * out[0] = mu, out[1] = E_band = sum f_i lambda_i, out[2] = sum f_i. */
int oracle_density(int n, const double *H, double ne, double kT, int use_jacobi,
                   double *D, double *w, double *f, double *out)
{
    double *Q = (double *)malloc(sizeof(double) * (size_t)n * n);
    const int st = use_jacobi ? oracle_eigh_jacobi(n, H, w, Q, 100) : oracle_eigh_ql(n, H, w, Q);
    const double mu = oracle_occupations(n, w, ne, kT, f);
    oracle_density_from_eig(n, Q, f, D);
    double e = 0.0, t = 0.0;
    for (int i = 0; i < n; ++i) { e += f[i] * w[i]; t += f[i]; }
    out[0] = mu; out[1] = e; out[2] = t;
    free(Q);
    return st;
}

/* ------------------------------------------------------------------ */
/* CPU SP2 (Sec. II-B1, Eq. (1); trace rule of Sec. III-B)              */
/* ------------------------------------------------------------------ */
/* X0 = (emax I - H)/(emax - emin) from Gershgorin bounds (occupied states
 * map toward 1).  Each step: t1 = tr X, t2 = ||X||_F^2 = tr X^2; choose
 * X^2 if |t2 - ne| <= |2 t1 - t2 - ne| else 2X - X^2.  Stop when the
 * relative trace change |t1_new - t1_old| / ne <= tol, or at max_iter.
 * branches[k] records 1 for X^2, 0 for 2X - X^2 (may be NULL).
 * Returns the number of products, or -1 if max_iter was reached. */
int oracle_sp2(int n, const double *H, double ne, double tol, int max_iter,
               double *X, int *branches)
{
    double emin, emax;
    oracle_gershgorin(n, H, &emin, &emax);
    const double w = emax - emin;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            X[IDX(i, j, n)] = ((i == j ? emax : 0.0) - H[IDX(i, j, n)]) / w;
    double *X2 = (double *)malloc(sizeof(double) * (size_t)n * n);
    double t1 = oracle_trace(n, X);
    int it = 0, done = 0;
    while (it < max_iter && !done) {
        double t2 = 0.0;
        for (size_t k = 0; k < (size_t)n * n; ++k) t2 += X[k] * X[k];
        const int sq = fabs(t2 - ne) <= fabs(2.0 * t1 - t2 - ne);
        oracle_matmul(n, X, X, X2);
        if (sq) {
            memcpy(X, X2, sizeof(double) * (size_t)n * n);
        } else {
            for (size_t k = 0; k < (size_t)n * n; ++k) X[k] = 2.0 * X[k] - X2[k];
        }
        if (branches) branches[it] = sq;
        ++it;
        const double t1n = oracle_trace(n, X);
        if (fabs(t1n - t1) <= tol * ne) done = 1;
        t1 = t1n;
    }
    free(X2);
    return done ? it : -1;
}

/* ------------------------------------------------------------------ */
/* Accelerated SP2 (A-Z-RFOE, Sec. II-B2)                               */
/* ------------------------------------------------------------------ */
/* The paper moves the eigenvalues toward 0 or 1 faster by shifting and
 * scaling the SP2 polynomials with the HOMO and LUMO eigenvalues (homo <
 * lumo, estimates from the caller).  With X0 as in oracle_sp2, unoccupied
 * eigenvalues of X lie in [0, a] and occupied ones in [b, 1], where
 * a = (emax - lumo)/w and b = (emax - homo)/w.  The bounds, not the trace,
 * say where the gap is, so each step takes the branch that moves the gap
 * toward the middle of [0, 1] (X^2 while a + b > 1, else 2X - X^2) as long
 * as max(a, 1 - b) >= 1e-3, and the SP2 trace rule on t1 = tr X,
 * t2 = tr X^2 after that (the folds are then negligible); it applies its
 * polynomial folded over the interval that has to shrink:
 *   X^2 branch:     p(x) = ((x - s)/(1 - s))^2,        s = a/2,
 *                   so p(0) = p(a), p(1) = 1;
 *   2X - X^2 branch: q(x) = (2 (1 - s) x - x^2)/(1 - s)^2, s = (1 - b)/2,
 *                   so q(b) = q(1), q(0) = 0;
 * then a <- f(a), b <- f(b) for the polynomial f applied.  A product's
 * rounding error enters the next iterate multiplied by r = 1/(1 - s)^2 and
 * turns the occupied subspace by that error over the gap b - a, so while
 * that gap is narrow (b - a < 1e-2) the fold point is capped at s <= 1/4
 * (r <= 16/9).  With s = 0 (no gap information: a = 0, b = 1, or bounds
 * that do not bracket a gap) a step is the SP2 step.
 *
 * The folds are valid only while every eigenvalue stays in [0, a] u [b, 1],
 * i.e. when the estimates lie inside the true gap (homo >= HOMO, lumo <=
 * LUMO).  With N_e states in [b, 1] and n - N_e in [0, a] after a step,
 *     N_e b <= tr X <= N_e + (n - N_e) a   and
 *     tr X - tr X^2 = sum x (1 - x) <= (n - N_e) a + N_e (1 - b);
 * estimates that put a state on the wrong side, or leave one between a and
 * b, break one of these by a whole state once a and 1 - b have shrunk, so a
 * violation by more than 1/2 stops the recursion with -2 (the caller then
 * runs plain SP2).  Stop as oracle_sp2 otherwise.  Returns the number of
 * products, -1 if max_iter was reached, or -2 if the estimates were found
 * inconsistent with the spectrum. */
int oracle_sp2_accel(int n, const double *H, double ne, double homo, double lumo, double tol,
                     int max_iter, double *X, int *branches)
{
    double emin, emax;
    oracle_gershgorin(n, H, &emin, &emax);
    const double w = emax - emin;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            X[IDX(i, j, n)] = ((i == j ? emax : 0.0) - H[IDX(i, j, n)]) / w;
    double a = (emax - lumo) / w, b = (emax - homo) / w;
    if (!(a >= 0.0 && b <= 1.0 && a < b)) {
        a = 0.0;
        b = 1.0;
    }
    const int informed = !(a == 0.0 && b == 1.0);
    double *X2 = (double *)malloc(sizeof(double) * (size_t)n * n);
    double t1 = oracle_trace(n, X);
    int it = 0, done = 0;
    while (it < max_iter && !done) {
        double t2 = 0.0;
        for (size_t k = 0; k < (size_t)n * n; ++k) t2 += X[k] * X[k];
        const int by_bounds = informed && fmax(a, 1.0 - b) >= 1e-3;
        const int sq = by_bounds ? (a + b > 1.0) : (fabs(t2 - ne) <= fabs(2.0 * t1 - t2 - ne));
        oracle_matmul(n, X, X, X2);
        double s = sq ? 0.5 * a : 0.5 * (1.0 - b);
        if (b - a < 1e-2 && s > 0.25) s = 0.25;
        const double r = 1.0 / ((1.0 - s) * (1.0 - s));
        if (sq) {
            for (int i = 0; i < n; ++i)
                for (int j = 0; j < n; ++j) {
                    const size_t k = IDX(i, j, n);
                    X[k] = (X2[k] - 2.0 * s * X[k] + (i == j ? s * s : 0.0)) * r;
                }
            a = (a - s) * (a - s) * r;
            b = (b - s) * (b - s) * r;
        } else {
            for (size_t k = 0; k < (size_t)n * n; ++k) X[k] = (2.0 * (1.0 - s) * X[k] - X2[k]) * r;
            a = (2.0 * (1.0 - s) * a - a * a) * r;
            b = (2.0 * (1.0 - s) * b - b * b) * r;
        }
        if (branches) branches[it] = sq;
        ++it;
        const double t1n = oracle_trace(n, X);
        if (informed) {
            double t2n = 0.0;
            for (size_t k = 0; k < (size_t)n * n; ++k) t2n += X[k] * X[k];
            const double lo = ne * b, hi = ne + ((double)n - ne) * a;
            const double spread = ((double)n - ne) * a + ne * (1.0 - b);
            if (t1n < lo - 0.5 || t1n > hi + 0.5 || t1n - t2n > spread + 0.5) {
                free(X2);
                return -2;
            }
        }
        if (fabs(t1n - t1) <= tol * ne) done = 1;
        t1 = t1n;
    }
    free(X2);
    return done ? it : -1;
}

/* ------------------------------------------------------------------ */
/* Truncated SP2 at finite temperature (T-RFOE, Sec. II-B3, Eq. (2))    */
/* ------------------------------------------------------------------ */
/* The paper smears the zero-temperature step with an intermediate iterate
 * of the SP2 recursion: D = G_m(H) = F_m(F_{m-1}(... F_0(X_0))), the same
 * trace-driven branches as oracle_sp2, stopped after m steps, with m larger
 * for lower temperature.  Its references fixing m are not in the text; the
 * reading used: every F is increasing on [0, 1], so G_k(x) crosses 1/2 at
 * one point x*_k, and the expansion stops at the first k whose step function
 * is as steep there as the Fermi-Dirac function at mu,
 *     |d G_k / d eps| (eps*) = (1/w) prod_j F_j'(u_j) >= beta / 4,
 * with u_0 = x*_k, u_{j+1} = F_j(u_j), u_k = 1/2, F' = 2u (X^2) or
 * 2 - 2u (2X - X^2), x = (emax - eps)/w, w = emax - emin.  The u_j follow
 * backwards from u_k = 1/2 by the closed-form inverses sqrt(y) and
 * 1 - sqrt(1 - y); eps* = emax - w u_0 is reported as mu.
 *
 * Because every step is a polynomial in H, G_m(H) = Q diag(G_m(x(lambda)))
 * Q^T: the recursion is run on the scalars x_i = (emax - lambda_i)/w of the
 * given eigenvalues, with t1 = sum x_i and t2 = sum x_i^2 deciding the
 * branch exactly as the matrix recursion's traces would, and x_out receives
 * G_m(x_i).  emin/emax are the spectral bounds of the matrix recursion
 * (Gershgorin, Sec. II-C).  branches[k] records 1 for X^2, 0 for 2X - X^2.
 * Returns m, or -1 if max_iter steps did not reach the slope. */
static double trfoe_slope(const int *bits, int m, double w, double *mid)
{
    double u = 0.5, d = 1.0;
    for (int k = m - 1; k >= 0; --k) {
        u = bits[k] ? sqrt(u) : 1.0 - sqrt(1.0 - u);   /* u_k = F_k^{-1}(u_{k+1}) */
        d *= bits[k] ? 2.0 * u : 2.0 - 2.0 * u;        /* F_k'(u_k) */
    }
    *mid = u;
    return d / w;
}

int oracle_trfoe(int n, const double *lam, double ne, double beta, double emin, double emax,
                 int max_iter, double *x_out, int *branches, double *mu)
{
    const double w = emax - emin;
    int *bits = (int *)malloc(sizeof(int) * (size_t)(max_iter + 1));
    for (int i = 0; i < n; ++i) x_out[i] = (emax - lam[i]) / w;
    int m = 0, reached = 0;
    for (;;) {
        double mid;
        const double slope = trfoe_slope(bits, m, w, &mid);
        *mu = emax - w * mid;
        if (slope >= 0.25 * beta) {
            reached = 1;
            break;
        }
        if (m >= max_iter) break;
        double t1 = 0.0, t2 = 0.0;
        for (int i = 0; i < n; ++i) {
            t1 += x_out[i];
            t2 += x_out[i] * x_out[i];
        }
        const int sq = fabs(t2 - ne) <= fabs(2.0 * t1 - t2 - ne);
        for (int i = 0; i < n; ++i) {
            const double x = x_out[i];
            x_out[i] = sq ? x * x : 2.0 * x - x * x;
        }
        bits[m] = sq;
        if (branches) branches[m] = sq;
        ++m;
    }
    free(bits);
    return reached ? m : -1;
}

/* ------------------------------------------------------------------ */
/* Finite temperature: recursive doubling of the inverse temperature    */
/* ------------------------------------------------------------------ */

/* In-place Cholesky factorisation of SPD A (lower triangle used).
 * Returns 0 on success. */
static int cholesky(int n, double *A)
{
    for (int j = 0; j < n; ++j) {
        double d = A[IDX(j, j, n)];
        for (int k = 0; k < j; ++k) d -= A[IDX(j, k, n)] * A[IDX(j, k, n)];
        if (d <= 0.0) return -1;
        d = sqrt(d);
        A[IDX(j, j, n)] = d;
#pragma omp parallel for schedule(static)
        for (int i = j + 1; i < n; ++i) {
            double s = A[IDX(i, j, n)];
            for (int k = 0; k < j; ++k) s -= A[IDX(i, k, n)] * A[IDX(j, k, n)];
            A[IDX(i, j, n)] = s / d;
        }
    }
    return 0;
}

/* Solve L L^T Xc = B in place for all n columns of B. */
static void cholesky_solve(int n, const double *L, double *B)
{
#pragma omp parallel for schedule(static)
    for (int c = 0; c < n; ++c) {
        for (int i = 0; i < n; ++i) {
            double s = B[IDX(i, c, n)];
            for (int k = 0; k < i; ++k) s -= L[IDX(i, k, n)] * B[IDX(k, c, n)];
            B[IDX(i, c, n)] = s / L[IDX(i, i, n)];
        }
        for (int i = n - 1; i >= 0; --i) {
            double s = B[IDX(i, c, n)];
            for (int k = i + 1; k < n; ++k) s -= L[IDX(k, i, n)] * B[IDX(k, c, n)];
            B[IDX(i, c, n)] = s / L[IDX(i, i, n)];
        }
    }
}

/* D(mu) by m doublings: z0 = (beta / 2^{m+1}) (H - mu I), then m times
 * z <- 2 z (I + z^2)^{-1} (the double-angle identity of tanh), D = (I - z)/2.
 * z_m approximates tanh(beta (H - mu)/2), so D approximates the Fermi-Dirac
 * matrix of Sec. II-A.  Returns 0 on success. */
int oracle_fermi_recursion(int n, const double *H, double mu, double kT, int m, double *D)
{
    const double beta = 1.0 / kT;
    const double a = beta / ldexp(1.0, m + 1);
    double *z = (double *)malloc(sizeof(double) * (size_t)n * n);
    double *M = (double *)malloc(sizeof(double) * (size_t)n * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            z[IDX(i, j, n)] = a * (H[IDX(i, j, n)] - (i == j ? mu : 0.0));
    int st = 0;
    for (int s = 0; s < m && st == 0; ++s) {
        oracle_matmul(n, z, z, M);                 /* M = z^2 */
        for (int i = 0; i < n; ++i) M[IDX(i, i, n)] += 1.0; /* I + z^2 */
        st = cholesky(n, M);
        for (size_t k = 0; k < (size_t)n * n; ++k) z[k] *= 2.0;
        if (st == 0) cholesky_solve(n, M, z);      /* z <- (I + z^2)^{-1} 2 z */
        /* symmetrise the rounding of the solve */
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                const double v = 0.5 * (z[IDX(i, j, n)] + z[IDX(j, i, n)]);
                z[IDX(i, j, n)] = v;
                z[IDX(j, i, n)] = v;
            }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            D[IDX(i, j, n)] = 0.5 * ((i == j ? 1.0 : 0.0) - z[IDX(i, j, n)]);
    free(z); free(M);
    return st;
}

/* ------------------------------------------------------------------ */
/* Error metrics (Sec. III-C)                                           */
/* ------------------------------------------------------------------ */
/* out[0] = ||D - Dref||_F, out[1] = ||Dref||_F, out[2] = tr(D H),
 * out[3] = tr(Dref H), out[4] = tr D, out[5] = ||D^2 - D||_F */
void oracle_metrics(int n, const double *D, const double *Dref, const double *H, double *out)
{
    double e = 0.0, r = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) {
        const double d = D[k] - Dref[k];
        e += d * d;
        r += Dref[k] * Dref[k];
    }
    out[0] = sqrt(e);
    out[1] = sqrt(r);
    out[2] = oracle_frob_dot(n, D, H);
    out[3] = oracle_frob_dot(n, Dref, H);
    out[4] = oracle_trace(n, D);
    double *D2 = (double *)malloc(sizeof(double) * (size_t)n * n);
    oracle_matmul(n, D, D, D2);
    double s = 0.0;
    for (size_t k = 0; k < (size_t)n * n; ++k) {
        const double d = D2[k] - D[k];
        s += d * d;
    }
    out[5] = sqrt(s);
    free(D2);
}
