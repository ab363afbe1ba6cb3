/*
 * mrc_oracle.c -- plain, slow FP64 reference for matrix renewal convolution.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or helper with the CUDA path, and the CUDA path never
 * calls it.
 *
 * Every routine below is the definition from Kordalis & Trevezas, "Algebraic
 * and FFT-Based Methods for Discrete-Time Matrix Convolutions with
 * Applications to Semi-Markov Models", written out with no blocking, fusion or
 * reordering.  Sequences are stored row-major, one r x c matrix per time
 * index, time slowest: X[k*r*c + i*c + j] = X(k)_{ij}.
 *
 * Parallelism: OpenMP over independent output columns/rows/time indices only;
 * every output element is computed by the same sequence of operations as in
 * the serial loop.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define IDX(k, i, j, r, c) ((size_t)(k) * (size_t)(r) * (size_t)(c) + (size_t)(i) * (size_t)(c) + (size_t)(j))

/*
 * Dense inverse of a d x d matrix by Gauss-Jordan elimination with partial
 * pivoting (the constant-term inverse A(0)^{-1} of Theorem 2.2 / Eq. (newton)).
 * Returns 0 on success, 1 if a pivot magnitude is <= d * 2^-52 * max|M|
 * (the singularity reading stated in the design notes).
 */
int orc_gauss_jordan(int d, const double *M, double *Minv)
{
    double *W = (double *)malloc(sizeof(double) * (size_t)d * 2 * d);
    if (!W) return 2;
    double amax = 0.0;
    for (int i = 0; i < d; ++i) {
        for (int j = 0; j < d; ++j) {
            W[i * 2 * d + j] = M[i * d + j];
            W[i * 2 * d + d + j] = (i == j) ? 1.0 : 0.0;
            if (fabs(M[i * d + j]) > amax) amax = fabs(M[i * d + j]);
        }
    }
    const double tol = (double)d * ldexp(1.0, -52) * amax;
    for (int col = 0; col < d; ++col) {
        int piv = col;
        for (int i = col + 1; i < d; ++i)
            if (fabs(W[i * 2 * d + col]) > fabs(W[piv * 2 * d + col])) piv = i;
        if (!(fabs(W[piv * 2 * d + col]) > tol)) { free(W); return 1; }
        if (piv != col)
            for (int j = 0; j < 2 * d; ++j) {
                double t = W[col * 2 * d + j];
                W[col * 2 * d + j] = W[piv * 2 * d + j];
                W[piv * 2 * d + j] = t;
            }
        const double p = W[col * 2 * d + col];
        for (int j = 0; j < 2 * d; ++j) W[col * 2 * d + j] /= p;
        for (int i = 0; i < d; ++i) {
            if (i == col) continue;
            const double f = W[i * 2 * d + col];
            if (f == 0.0) continue;
            for (int j = 0; j < 2 * d; ++j) W[i * 2 * d + j] -= f * W[col * 2 * d + j];
        }
    }
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) Minv[i * d + j] = W[i * 2 * d + d + j];
    free(W);
    return 0;
}

/*
 * Truncated matrix convolution, Eq. (convolution):
 *   C(k) = sum_{l=0..k} A(l) B(k-l),  k = 0..N-1,
 * A is [N][r][m], B is [N][m][c], C is [N][r][c] (rectangular allowed).
 */
void orc_convolve(int r, int m, int c, int64_t N, const double *A, const double *B, double *C)
{
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < N; ++k) {
        for (int i = 0; i < r; ++i)
            for (int j = 0; j < c; ++j) {
                double s = 0.0;
                for (int64_t l = 0; l <= k; ++l)
                    for (int t = 0; t < m; ++t)
                        s += A[IDX(l, i, t, r, m)] * B[IDX(k - l, t, j, m, c)];
                C[IDX(k, i, j, r, c)] = s;
            }
    }
}

/*
 * Left inverse by direct recursion on A * psi = e0 (Theorem 2.2; for
 * A = e0 - q with q(0) = 0 this is psi(k) = delta(k) I + sum_{l=1..k} q(l) psi(k-l),
 * Eq. (renewal-sequence)):
 *   psi(k) = A(0)^{-1} [ delta(k) I - sum_{l=1..k} A(l) psi(k-l) ].
 * Column j of psi depends only on column j of earlier coefficients, so the
 * columns are independent.  Returns 0, or 1 if A(0) is singular.
 */
int orc_inverse_left(int d, int64_t N, const double *A, double *psi)
{
    double *A0inv = (double *)malloc(sizeof(double) * (size_t)d * d);
    if (!A0inv) return 2;
    if (orc_gauss_jordan(d, A, A0inv)) { free(A0inv); return 1; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < d; ++j) {
        double *t = (double *)malloc(sizeof(double) * (size_t)d);
        for (int64_t k = 0; k < N; ++k) {
            for (int i = 0; i < d; ++i) {
                double s = (k == 0 && i == j) ? 1.0 : 0.0;
                for (int64_t l = 1; l <= k; ++l)
                    for (int u = 0; u < d; ++u)
                        s -= A[IDX(l, i, u, d, d)] * psi[IDX(k - l, u, j, d, d)];
                t[i] = s;
            }
            for (int i = 0; i < d; ++i) {
                double s = 0.0;
                for (int u = 0; u < d; ++u) s += A0inv[i * d + u] * t[u];
                psi[IDX(k, i, j, d, d)] = s;
            }
        }
        free(t);
    }
    free(A0inv);
    return 0;
}

/*
 * Right inverse by the coefficient recursion, Eq. (inverse-recursion):
 *   A^{(-1)}(0) = A(0)^{-1},
 *   A^{(-1)}(k) = - sum_{l=0..k-1} A^{(-1)}(l) A(k-l) A(0)^{-1},  k >= 1.
 * Row i of the result depends only on row i of earlier coefficients.
 * An independent formula from orc_inverse_left (two-sidedness, Theorem 2.2).
 */
int orc_inverse_right(int d, int64_t N, const double *A, double *psi)
{
    double *A0inv = (double *)malloc(sizeof(double) * (size_t)d * d);
    if (!A0inv) return 2;
    if (orc_gauss_jordan(d, A, A0inv)) { free(A0inv); return 1; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int i = 0; i < d; ++i) {
        double *t = (double *)malloc(sizeof(double) * (size_t)d);
        for (int j = 0; j < d; ++j) psi[IDX(0, i, j, d, d)] = A0inv[i * d + j];
        for (int64_t k = 1; k < N; ++k) {
            /* t = - sum_l psi(l) A(k-l), row i */
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int64_t l = 0; l < k; ++l)
                    for (int u = 0; u < d; ++u)
                        s -= psi[IDX(l, i, u, d, d)] * A[IDX(k - l, u, j, d, d)];
                t[j] = s;
            }
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int u = 0; u < d; ++u) s += t[u] * A0inv[u * d + j];
                psi[IDX(k, i, j, d, d)] = s;
            }
        }
        free(t);
    }
    free(A0inv);
    return 0;
}

/*
 * Left and right residuals of a computed inverse (Proposition 2.6):
 *   rho_L = e0 - A * psi,   rho_R = e0 - psi * A,   k = 0..N-1.
 * Either output may be NULL.
 */
void orc_residuals(int d, int64_t N, const double *A, const double *psi, double *rhoL, double *rhoR)
{
    const size_t n = (size_t)N * d * d;
    if (rhoL) {
        orc_convolve(d, d, d, N, A, psi, rhoL);
        for (size_t t = 0; t < n; ++t) rhoL[t] = -rhoL[t];
        for (int i = 0; i < d; ++i) rhoL[IDX(0, i, i, d, d)] += 1.0;
    }
    if (rhoR) {
        orc_convolve(d, d, d, N, psi, A, rhoR);
        for (size_t t = 0; t < n; ++t) rhoR[t] = -rhoR[t];
        for (int i = 0; i < d; ++i) rhoR[IDX(0, i, i, d, d)] += 1.0;
    }
}

/*
 * One coefficient of the left residual, rho_L(k) = delta(k) I - sum_{l<=k} A(l) psi(k-l),
 * for a single time index k (used to check sampled outputs of very long runs).
 * out is d x d.
 */
void orc_residual_left_at(int d, int64_t k, const double *A, const double *psi, double *out)
{
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            double s = (k == 0 && i == j) ? 1.0 : 0.0;
            for (int64_t l = 0; l <= k; ++l)
                for (int u = 0; u < d; ++u)
                    s -= A[IDX(l, i, u, d, d)] * psi[IDX(k - l, u, j, d, d)];
            out[i * d + j] = s;
        }
}

/*
 * One entry of each residual at one time index k (Proposition 2.6):
 *   rho_L(k)_{ij} = delta(k) delta_{ij} - sum_{l=0..k} sum_u A(l)_{iu} psi(k-l)_{uj},
 *   rho_R(k)_{ij} = delta(k) delta_{ij} - sum_{l=0..k} sum_u psi(l)_{iu} A(k-l)_{uj}.
 * Cost O(k d) each: checks sampled outputs of runs far too long for the full
 * residual.
 */
double orc_residual_left_entry(int d, int64_t k, int i, int j, const double *A, const double *psi)
{
    double s = (k == 0 && i == j) ? 1.0 : 0.0;
    for (int64_t l = 0; l <= k; ++l)
        for (int u = 0; u < d; ++u) s -= A[IDX(l, i, u, d, d)] * psi[IDX(k - l, u, j, d, d)];
    return s;
}

double orc_residual_right_entry(int d, int64_t k, int i, int j, const double *A, const double *psi)
{
    double s = (k == 0 && i == j) ? 1.0 : 0.0;
    for (int64_t l = 0; l <= k; ++l)
        for (int u = 0; u < d; ++u) s -= psi[IDX(l, i, u, d, d)] * A[IDX(k - l, u, j, d, d)];
    return s;
}

/*
 * Survival diagonal of the discrete kernel (Section 4.1):
 *   Hbar(k) = diag( 1 - sum_j sum_{l=1..k} q_ij(l) ),  stored as hbar[k*d + i].
 */
void orc_hbar(int d, int64_t N, const double *q, double *hbar)
{
    for (int i = 0; i < d; ++i) {
        double cum = 0.0;
        for (int64_t k = 0; k < N; ++k) {
            if (k >= 1)
                for (int j = 0; j < d; ++j) cum += q[IDX(k, i, j, d, d)];
            hbar[(size_t)k * d + i] = 1.0 - cum;
        }
    }
}

/*
 * Transition probabilities, Eq. (transition-discrete): P = psi * Hbar with
 * Hbar diagonal, i.e. P_ij(k) = sum_{l<=k} psi_ij(l) hbar_j(k-l).
 */
void orc_transition(int d, int64_t N, const double *psi, const double *q, double *P)
{
    double *hbar = (double *)malloc(sizeof(double) * (size_t)N * d);
    orc_hbar(d, N, q, hbar);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < N; ++k)
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                double s = 0.0;
                for (int64_t l = 0; l <= k; ++l) s += psi[IDX(l, i, j, d, d)] * hbar[(size_t)(k - l) * d + j];
                P[IDX(k, i, j, d, d)] = s;
            }
    free(hbar);
}

/*
 * First entrance into D (Eqs. (first-entrance-mass), (first-entrance-cdf)):
 *   g_D = (e0^C - q_CC)^{(-1)} * q_CD,   G_D(k) = sum_{l<=k} g_D(l),
 *   F_D(k) = alpha_C G_D(k) 1_D,          S_D(k) = 1 - F_D(k).
 * inD[i] != 0 marks i in D; C is the complement, both in increasing state order.
 * g is [N][|C|][|D|]; F, S are [N]; any of g, F, S may be NULL.
 * Returns 0, 1 if e0^C - q_CC is not invertible, 3 if C or D is empty.
 */
int orc_first_entrance(int d, int64_t N, const double *q, const int *inD, const double *alphaC,
                       double *g, double *F, double *S)
{
    int nC = 0, nD = 0;
    int *Ci = (int *)malloc(sizeof(int) * d), *Di = (int *)malloc(sizeof(int) * d);
    for (int i = 0; i < d; ++i) {
        if (inD[i]) Di[nD++] = i; else Ci[nC++] = i;
    }
    if (nC == 0 || nD == 0) { free(Ci); free(Di); return 3; }
    double *ACC = (double *)malloc(sizeof(double) * (size_t)N * nC * nC);
    double *qCD = (double *)malloc(sizeof(double) * (size_t)N * nC * nD);
    double *psiC = (double *)malloc(sizeof(double) * (size_t)N * nC * nC);
    double *gl = (double *)malloc(sizeof(double) * (size_t)N * nC * nD);
    for (int64_t k = 0; k < N; ++k) {
        for (int a = 0; a < nC; ++a) {
            for (int b = 0; b < nC; ++b)
                ACC[IDX(k, a, b, nC, nC)] = ((k == 0 && a == b) ? 1.0 : 0.0) - q[IDX(k, Ci[a], Ci[b], d, d)];
            for (int b = 0; b < nD; ++b) qCD[IDX(k, a, b, nC, nD)] = q[IDX(k, Ci[a], Di[b], d, d)];
        }
    }
    int rc = orc_inverse_left(nC, N, ACC, psiC);
    if (rc == 0) {
        orc_convolve(nC, nC, nD, N, psiC, qCD, gl);
        if (g) memcpy(g, gl, sizeof(double) * (size_t)N * nC * nD);
        if (F || S) {
            double *G = (double *)calloc((size_t)nC * nD, sizeof(double));
            for (int64_t k = 0; k < N; ++k) {
                for (int t = 0; t < nC * nD; ++t) G[t] += gl[(size_t)k * nC * nD + t];
                double f = 0.0;
                for (int a = 0; a < nC; ++a)
                    for (int b = 0; b < nD; ++b) f += alphaC[a] * G[a * nD + b];
                if (F) F[k] = f;
                if (S) S[k] = 1.0 - f;
            }
            free(G);
        }
    }
    free(Ci); free(Di); free(ACC); free(qCD); free(psiC); free(gl);
    return rc;
}

/*
 * Occupation probability of B (Table 2): A_B(k) = alpha P(k) 1_{E,B}.
 * Availability is the case B = up states.  inB[j] != 0 marks j in B.
 */
void orc_occupation(int d, int64_t N, const double *P, const double *alpha, const int *inB, double *out)
{
    for (int64_t k = 0; k < N; ++k) {
        double s = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j)
                if (inB[j]) s += alpha[i] * P[IDX(k, i, j, d, d)];
        out[k] = s;
    }
}

/*
 * Expected renewal visits to B, Eq. (renewal-visits):
 *   N_B(k) = alpha sum_{l<=k} psi(l) I_B 1_s.
 */
void orc_renewal_visits(int d, int64_t N, const double *psi, const double *alpha, const int *inB, double *out)
{
    double cum = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j)
                if (inB[j]) cum += alpha[i] * psi[IDX(k, i, j, d, d)];
        out[k] = cum;
    }
}

/* Horizon norm ||X||_{1,N} with the Frobenius norm per coefficient (an upper
 * bound of the spectral-norm version defined in Section 2). */
double orc_norm1_frob(int r, int c, int64_t N, const double *X)
{
    double tot = 0.0;
    for (int64_t k = 0; k < N; ++k) {
        double s = 0.0;
        for (int t = 0; t < r * c; ++t) s += X[(size_t)k * r * c + t] * X[(size_t)k * r * c + t];
        tot += sqrt(s);
    }
    return tot;
}

/* Spectral norm ||X||_2 of one r x c matrix: square root of the largest
 * eigenvalue of X^T X, by power iteration run to a fixed point (at most
 * 10000 steps).  Used for the Section 2 horizon norm ||.||_{1,N} on small d. */
double orc_spectral_norm(int r, int c, const double *X)
{
    double *v = (double *)malloc(sizeof(double) * c), *w = (double *)malloc(sizeof(double) * r);
    double *z = (double *)malloc(sizeof(double) * c);
    for (int j = 0; j < c; ++j) v[j] = 1.0 / sqrt((double)c) * (1.0 + 0.01 * j);
    double lam = 0.0;
    for (int it = 0; it < 10000; ++it) {
        for (int i = 0; i < r; ++i) {
            double s = 0.0;
            for (int j = 0; j < c; ++j) s += X[i * c + j] * v[j];
            w[i] = s;
        }
        double nz = 0.0;
        for (int j = 0; j < c; ++j) {
            double s = 0.0;
            for (int i = 0; i < r; ++i) s += X[i * c + j] * w[i];
            z[j] = s;
            nz += s * s;
        }
        nz = sqrt(nz);
        if (nz == 0.0) { lam = 0.0; break; }
        for (int j = 0; j < c; ++j) v[j] = z[j] / nz;
        if (fabs(nz - lam) <= 1e-15 * nz) { lam = nz; break; }
        lam = nz;
    }
    free(v); free(w); free(z);
    return sqrt(lam);
}

double orc_norm1_spec(int r, int c, int64_t N, const double *X)
{
    double tot = 0.0;
    for (int64_t k = 0; k < N; ++k) tot += orc_spectral_norm(r, c, X + (size_t)k * r * c);
    return tot;
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
