/*
 * bv_oracle.c -- plain, slow FP64 CPU oracle for the block-Vecchia Gaussian-process
 * log-likelihood of Pan, Abdulah, Genton and Sun, "Block Vecchia Approximation for
 * Scalable and Efficient Gaussian Process Computations" (arXiv 2410.04477).
 *
 * TEST INFRASTRUCTURE.  Only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg load this file.  The product path (the CUDA library) shares no code,
 * header, table or helper with it.
 *
 * Every routine follows the paper's definitions step by step, in FP64, with no blocking,
 * fusion or reordering beyond what the definition states:
 *   - Matern covariance, Eq. 5 (closed forms at nu = 1/2, 3/2, 5/2; general nu by the
 *     integral representation of K_nu), plus an absolute nugget on the diagonal.
 *   - K-means blocks (Sec. 2.1, Algorithm 1 "Clustering"): k-means++ seeding and Lloyd
 *     iterations, with the exact-integer conventions described at or_kmeans().
 *   - Random block permutation zeta (Sec. 2.1, Algorithm 1 "Block permutation").
 *   - Block nearest neighbours (Sec. 2.2; Algorithm 1 "Nearest neighbors").
 *   - Per-block conditional log-likelihood, literally the batched steps of Algorithm 1
 *     (POTRF, TRSM, TRSV, GEMM, GEMV, elementwise update, POTRF, TRSV, dot, log-det)
 *     and the final sum.
 *   - Exact GP log-likelihood, Eq. 1, by a dense Cholesky.
 *   - Prediction (Sec. 2.4, Algorithm 2): blocks of the new locations, their nearest
 *     observations, conditional means and covariances; univariate conditional
 *     simulation and the prediction interval coverage (Sec. 3.2).
 *   - Input generators built from the same definitions: an exact GP draw and the
 *     block-Vecchia draw (Eq. 4 read generatively).
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -shared -fPIC (no FMA contraction, so the
 * squared distances used by K-means and the neighbour search round exactly as written).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_EINVAL 1
#define OR_ENOMEM 2
#define OR_ENOTPD 4

typedef struct {
    double sigma2;   /* sigma^2, Eq. 5 */
    double range[3]; /* beta (range[0]) or per-axis ranges when aniso != 0 */
    double nu;       /* smoothness nu, Eq. 5 */
    double nugget;   /* tau^2, added on the diagonal (by point identity) */
    int32_t aniso;
    int32_t pad;
} or_theta;

/* ------------------------------------------------------------------------------------
 * Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014), used in counter form: draw number c of stream s is
 * the SplitMix64 finaliser applied to s + (c + 1) * golden-gamma.
 * ---------------------------------------------------------------------------------- */
static uint64_t or_sm64(uint64_t stream, uint64_t counter) {
    uint64_t z = stream + (counter + 1u) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* floor(r * n / 2^64): an exact uniform integer in [0, n) from a 64-bit draw. */
static uint64_t or_mulhi(uint64_t r, uint64_t n) {
    return (uint64_t)(((unsigned __int128)r * (unsigned __int128)n) >> 64);
}

uint64_t or_splitmix64(uint64_t stream, uint64_t counter) { return or_sm64(stream, counter); }

/* Stream constants (fixed; the CUDA library uses the same published generator with the
 * same stream derivation so that seeds mean the same thing on both sides). */
#define OR_STREAM_KPP(seed) ((seed) ^ 0x6b6d65616e732b2bULL)  /* "kmeans++" */
#define OR_STREAM_ZETA(seed) ((seed) ^ 0x7a6574615f6f7264ULL) /* "zeta_ord" */

/* ------------------------------------------------------------------------------------
 * Matern covariance, Eq. 5:  C(r) = sigma^2 2^{1-nu}/Gamma(nu) (r/beta)^nu K_nu(r/beta).
 * ---------------------------------------------------------------------------------- */

/* K_nu(x) = int_0^inf exp(-x cosh t) cosh(nu t) dt (DLMF 10.32.9), by the composite
 * trapezoidal rule, which converges geometrically for this doubly-exponentially decaying
 * analytic integrand.  Used only for general nu and as a pin for the closed forms. */
double or_bessel_k(double nu, double x) {
    if (!(x > 0.0)) return INFINITY;
    const double h = 1.0 / 256.0;
    double sum = 0.5 * exp(-x); /* t = 0 term, weight 1/2 */
    for (int64_t k = 1;; k++) {
        double t = (double)k * h;
        double e = -x * cosh(t) + nu * t;
        /* cosh(nu t) exp(-x cosh t) = (exp(nu t) + exp(-nu t))/2 * exp(-x cosh t) */
        double term = 0.5 * (exp(e) + exp(-x * cosh(t) - nu * t));
        sum += term;
        if (e < -745.0 && t > 1.0) break;
        if (k > 400000) break;
    }
    return sum * h;
}

/* Correlation rho(x) = 2^{1-nu}/Gamma(nu) x^nu K_nu(x) with rho(0) = 1.  For the
 * half-integer smoothness values used in the paper's studies (Sec. 3.1: nu = 0.5, 1.5,
 * 2.5) K_nu has the elementary closed forms (DLMF 10.49.12), which give
 *   nu = 1/2: exp(-x);  nu = 3/2: (1 + x) exp(-x);  nu = 5/2: (1 + x + x^2/3) exp(-x). */
double or_matern_corr(double nu, double x) {
    if (x == 0.0) return 1.0;
    if (nu == 0.5) return exp(-x);
    if (nu == 1.5) return (1.0 + x) * exp(-x);
    if (nu == 2.5) return (1.0 + x + x * x / 3.0) * exp(-x);
    return pow(2.0, 1.0 - nu) / tgamma(nu) * pow(x, nu) * or_bessel_k(nu, x);
}

/* Scaled distance x = ||s_i - s_j|| / beta (Eq. 5), or with per-axis ranges
 * x = sqrt(sum_k ((s_ik - s_jk)/beta_k)^2) when theta->aniso is set. */
static double or_scaled_dist(const or_theta* th, int d, const double* si, const double* sj) {
    double acc = 0.0;
    if (th->aniso) {
        for (int k = 0; k < d; k++) {
            double t = (si[k] - sj[k]) / th->range[k];
            acc += t * t;
        }
        return sqrt(acc);
    }
    for (int k = 0; k < d; k++) {
        double t = si[k] - sj[k];
        acc += t * t;
    }
    return sqrt(acc) / th->range[0];
}

/* Covariance between two locations; `same` is 1 when they are the same observation,
 * in which case the nugget tau^2 is added (absolute, not scaled by sigma^2). */
double or_cov(const or_theta* th, int d, const double* si, const double* sj, int same) {
    double c = th->sigma2 * or_matern_corr(th->nu, or_scaled_dist(th, d, si, sj));
    if (same) c += th->nugget;
    return c;
}

int or_theta_valid(const or_theta* th, int d) {
    if (!(th->sigma2 > 0.0) || !(th->nugget >= 0.0) || !(th->nu > 0.0)) return 0;
    int nr = th->aniso ? d : 1;
    for (int k = 0; k < nr; k++)
        if (!(th->range[k] > 0.0)) return 0;
    return 1;
}

/* ------------------------------------------------------------------------------------
 * Dense helpers (plain textbook loops).
 * ---------------------------------------------------------------------------------- */

/* In-place Cholesky A = L L^T of a symmetric n x n row-major matrix (lower triangle
 * used and overwritten; upper triangle zeroed).  Returns OR_ENOTPD on a non-positive
 * pivot. */
static int or_potrf(double* A, int64_t n) {
    for (int64_t j = 0; j < n; j++) {
        double s = A[j * n + j];
        for (int64_t k = 0; k < j; k++) s -= A[j * n + k] * A[j * n + k];
        if (!(s > 0.0)) return OR_ENOTPD;
        double ljj = sqrt(s);
        A[j * n + j] = ljj;
        for (int64_t i = j + 1; i < n; i++) {
            double t = A[i * n + j];
            for (int64_t k = 0; k < j; k++) t -= A[i * n + k] * A[j * n + k];
            A[i * n + j] = t / ljj;
        }
        for (int64_t i = 0; i < j; i++) A[i * n + j] = 0.0;
    }
    return OR_OK;
}

/* Forward substitution x = L^{-1} b for one vector (L lower, row-major n x n). */
static void or_trsv(const double* L, int64_t n, const double* b, double* x) {
    for (int64_t i = 0; i < n; i++) {
        double t = b[i];
        for (int64_t k = 0; k < i; k++) t -= L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
}

/* ------------------------------------------------------------------------------------
 * Per-block conditional log-likelihood, literally Algorithm 1:
 *   Sigma^lk = K(s_B, s_B), Sigma^con = K(s_NN, s_NN), Sigma^cross = K(s_NN, s_B) (m x b)
 *   L = POTRF(Sigma^con); Sigma'^cross = L^{-1} Sigma^cross (TRSM); y' = L^{-1} y_NN (TRSV)
 *   Sigma^cor = Sigma'^cross^T Sigma'^cross (GEMM); mu^cor = Sigma'^cross^T y' (GEMV)
 *   Sigma^new = Sigma^lk - Sigma^cor;  mu^new = mu^cor
 *   L' = POTRF(Sigma^new); v = L'^{-1}(y_B - mu^new) (TRSV); u = v^T v; d = 2 log det L'
 *   ell_i = -(u + d + l_i log 2 pi) / 2.
 * For a block with an empty conditioning set (m_i = 0, the first block in the order)
 * Sigma^new = Sigma^lk and mu^new = 0.
 * ---------------------------------------------------------------------------------- */
double or_block_loglik(const or_theta* th, const double* locs, const double* y, int d,
                       const int32_t* nn, int64_t m, const int32_t* blk, int64_t b,
                       int* status) {
    *status = OR_OK;
    double* Slk = (double*)calloc((size_t)(b * b), sizeof(double));
    double* Scon = (double*)calloc((size_t)(m * m + 1), sizeof(double));
    double* Scross = (double*)calloc((size_t)(m * b + 1), sizeof(double));
    double* yp = (double*)calloc((size_t)(m + 1), sizeof(double));
    double* col = (double*)calloc((size_t)(m + 1), sizeof(double));
    double* colx = (double*)calloc((size_t)(m + 1), sizeof(double));
    double* mu = (double*)calloc((size_t)(b + 1), sizeof(double));
    double* r = (double*)calloc((size_t)(b + 1), sizeof(double));
    double* v = (double*)calloc((size_t)(b + 1), sizeof(double));
    if (!Slk || !Scon || !Scross || !yp || !col || !colx || !mu || !r || !v) {
        *status = OR_ENOMEM;
        free(Slk); free(Scon); free(Scross); free(yp); free(col); free(colx);
        free(mu); free(r); free(v);
        return NAN;
    }
    double ell = NAN;
    /* Kernel matrices and vectors (Algorithm 1, "Kernel vector and matrix"). */
    for (int64_t j = 0; j < b; j++)
        for (int64_t k = 0; k < b; k++)
            Slk[j * b + k] = or_cov(th, d, locs + (int64_t)blk[j] * d,
                                    locs + (int64_t)blk[k] * d, blk[j] == blk[k]);
    for (int64_t j = 0; j < m; j++)
        for (int64_t k = 0; k < m; k++)
            Scon[j * m + k] = or_cov(th, d, locs + (int64_t)nn[j] * d,
                                     locs + (int64_t)nn[k] * d, nn[j] == nn[k]);
    for (int64_t j = 0; j < m; j++)
        for (int64_t k = 0; k < b; k++)
            Scross[j * b + k] = or_cov(th, d, locs + (int64_t)nn[j] * d,
                                       locs + (int64_t)blk[k] * d, nn[j] == blk[k]);
    /* Sigma^old <- Sigma^lk; mu^new stays 0 when m = 0. */
    if (m > 0) {
        /* L = POTRF(Sigma^con) */
        if (or_potrf(Scon, m) != OR_OK) { *status = OR_ENOTPD; goto done; }
        /* Sigma'^cross = TRSM(L, Sigma^cross), column by column */
        for (int64_t k = 0; k < b; k++) {
            for (int64_t j = 0; j < m; j++) col[j] = Scross[j * b + k];
            or_trsv(Scon, m, col, colx);
            for (int64_t j = 0; j < m; j++) Scross[j * b + k] = colx[j];
        }
        /* y' = TRSV(L, y_NN) */
        for (int64_t j = 0; j < m; j++) col[j] = y[nn[j]];
        or_trsv(Scon, m, col, yp);
        /* Sigma^cor = GEMM(Sigma'^cross^T, Sigma'^cross); Sigma^new = Sigma^old - Sigma^cor */
        for (int64_t j = 0; j < b; j++)
            for (int64_t k = 0; k < b; k++) {
                double s = 0.0;
                for (int64_t p = 0; p < m; p++) s += Scross[p * b + j] * Scross[p * b + k];
                Slk[j * b + k] -= s;
            }
        /* mu^cor = GEMV(Sigma'^cross^T, y'); mu^new = mu^cor */
        for (int64_t j = 0; j < b; j++) {
            double s = 0.0;
            for (int64_t p = 0; p < m; p++) s += Scross[p * b + j] * yp[p];
            mu[j] = s;
        }
    }
    /* L' = POTRF(Sigma^new) */
    if (or_potrf(Slk, b) != OR_OK) { *status = OR_ENOTPD; goto done; }
    /* v = TRSV(L', y_B - mu^new) */
    for (int64_t j = 0; j < b; j++) r[j] = y[blk[j]] - mu[j];
    or_trsv(Slk, b, r, v);
    {
        double u = 0.0, dl = 0.0;
        for (int64_t j = 0; j < b; j++) u += v[j] * v[j];           /* u = v^T v */
        for (int64_t j = 0; j < b; j++) dl += log(Slk[j * b + j]);  /* log det L' */
        dl *= 2.0;                                                  /* d = 2 log det L' */
        ell = -0.5 * (u + dl + (double)b * log(2.0 * M_PI));
    }
done:
    free(Slk); free(Scon); free(Scross); free(yp); free(col); free(colx);
    free(mu); free(r); free(v);
    return ell;
}

/* Neumaier's compensated summation (Neumaier 1974). */
static double or_neumaier(const double* x, int64_t n) {
    double s = 0.0, c = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double t = s + x[i];
        if (fabs(s) >= fabs(x[i])) c += (s - t) + x[i];
        else c += (x[i] - t) + s;
        s = t;
    }
    return s + c;
}

/* Block-Vecchia log-likelihood, Eq. 4 with Algorithm 1: the sum over blocks (in the
 * permuted order given by the CSR arrays) of the per-block conditional log-likelihoods.
 * block_ptr[bc+1] / point_idx[n]: block i holds points point_idx[block_ptr[i] ..
 * block_ptr[i+1]); nn_ptr[bc+1] / nn_idx: its conditioning set.  Blocks are independent
 * (Sec. 2.2), so they are evaluated in parallel; the sum is sequential in block order.
 * Returns OR_ENOTPD (and ell = -inf) if any block is not positive definite. */
int or_loglik(const or_theta* th, const double* locs, const double* y, int64_t n, int d,
              int64_t bc, const int64_t* block_ptr, const int32_t* point_idx,
              const int64_t* nn_ptr, const int32_t* nn_idx, double* out_ll,
              double* out_per_block) {
    (void)n;
    if (!or_theta_valid(th, d)) return OR_EINVAL;
    double* per = out_per_block ? out_per_block : (double*)malloc(sizeof(double) * (size_t)(bc + 1));
    if (!per) return OR_ENOMEM;
    int fail = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < bc; i++) {
        int st = OR_OK;
        per[i] = or_block_loglik(th, locs, y, d, nn_idx + nn_ptr[i], nn_ptr[i + 1] - nn_ptr[i],
                                 point_idx + block_ptr[i], block_ptr[i + 1] - block_ptr[i], &st);
        if (st != OR_OK) {
#pragma omp critical
            if (fail == OR_OK) fail = st;
        }
    }
    *out_ll = fail == OR_OK ? or_neumaier(per, bc) : -INFINITY;
    if (!out_per_block) free(per);
    return fail;
}

/* Exact GP log-likelihood, Eq. 1: -n/2 log 2pi - 1/2 log|Sigma| - 1/2 y^T Sigma^{-1} y,
 * through a dense Cholesky of the full covariance matrix. */
int or_exact_loglik(const or_theta* th, const double* locs, const double* y, int64_t n,
                    int d, double* out_ll) {
    if (!or_theta_valid(th, d)) return OR_EINVAL;
    double* S = (double*)malloc(sizeof(double) * (size_t)(n * n));
    double* z = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    if (!S || !z) { free(S); free(z); return OR_ENOMEM; }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            S[i * n + j] = or_cov(th, d, locs + i * d, locs + j * d, i == j);
    if (or_potrf(S, n) != OR_OK) { free(S); free(z); *out_ll = -INFINITY; return OR_ENOTPD; }
    or_trsv(S, n, y, z);
    double q = 0.0, ld = 0.0;
    for (int64_t i = 0; i < n; i++) q += z[i] * z[i];
    for (int64_t i = 0; i < n; i++) ld += log(S[i * n + i]);
    *out_ll = -0.5 * (double)n * log(2.0 * M_PI) - ld - 0.5 * q;
    free(S); free(z);
    return OR_OK;
}

/* Exact GP draw y = chol(Sigma) z (input generator for the small configuration). */
int or_exact_draw(const or_theta* th, const double* locs, int64_t n, int d, const double* z,
                  double* y) {
    if (!or_theta_valid(th, d)) return OR_EINVAL;
    double* S = (double*)malloc(sizeof(double) * (size_t)(n * n));
    if (!S) return OR_ENOMEM;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++)
        for (int64_t j = 0; j < n; j++)
            S[i * n + j] = or_cov(th, d, locs + i * d, locs + j * d, i == j);
    if (or_potrf(S, n) != OR_OK) { free(S); return OR_ENOTPD; }
    for (int64_t i = 0; i < n; i++) {
        double t = 0.0;
        for (int64_t k = 0; k <= i; k++) t += S[i * n + k] * z[k];
        y[i] = t;
    }
    free(S);
    return OR_OK;
}

/* Block-Vecchia draw: Eq. 4 read generatively.  Blocks are visited in the permuted order;
 * block i draws y_{B_i} = mu_i + L'_i z_{B_i}, where mu_i and L'_i = chol(Sigma^new_i)
 * come from the same steps as Algorithm 1 with the already drawn y_{NN_i}.  z is indexed
 * by point (z[j] belongs to point j). */
int or_bv_draw(const or_theta* th, const double* locs, int64_t n, int d, int64_t bc,
               const int64_t* block_ptr, const int32_t* point_idx, const int64_t* nn_ptr,
               const int32_t* nn_idx, const double* z, double* y) {
    (void)n;
    if (!or_theta_valid(th, d)) return OR_EINVAL;
    for (int64_t i = 0; i < bc; i++) {
        const int32_t* blk = point_idx + block_ptr[i];
        const int32_t* nn = nn_idx + nn_ptr[i];
        int64_t b = block_ptr[i + 1] - block_ptr[i], m = nn_ptr[i + 1] - nn_ptr[i];
        double* Slk = (double*)calloc((size_t)(b * b + 1), sizeof(double));
        double* Scon = (double*)calloc((size_t)(m * m + 1), sizeof(double));
        double* Scross = (double*)calloc((size_t)(m * b + 1), sizeof(double));
        double* yp = (double*)calloc((size_t)(m + 1), sizeof(double));
        double* col = (double*)calloc((size_t)(m + 1), sizeof(double));
        double* colx = (double*)calloc((size_t)(m + 1), sizeof(double));
        double* mu = (double*)calloc((size_t)(b + 1), sizeof(double));
        int st = OR_OK;
        if (!Slk || !Scon || !Scross || !yp || !col || !colx || !mu) st = OR_ENOMEM;
        if (st == OR_OK) {
            for (int64_t j = 0; j < b; j++)
                for (int64_t k = 0; k < b; k++)
                    Slk[j * b + k] = or_cov(th, d, locs + (int64_t)blk[j] * d,
                                            locs + (int64_t)blk[k] * d, blk[j] == blk[k]);
            if (m > 0) {
                for (int64_t j = 0; j < m; j++)
                    for (int64_t k = 0; k < m; k++)
                        Scon[j * m + k] = or_cov(th, d, locs + (int64_t)nn[j] * d,
                                                 locs + (int64_t)nn[k] * d, nn[j] == nn[k]);
                for (int64_t j = 0; j < m; j++)
                    for (int64_t k = 0; k < b; k++)
                        Scross[j * b + k] = or_cov(th, d, locs + (int64_t)nn[j] * d,
                                                   locs + (int64_t)blk[k] * d, nn[j] == blk[k]);
                if (or_potrf(Scon, m) != OR_OK) st = OR_ENOTPD;
                if (st == OR_OK) {
                    for (int64_t k = 0; k < b; k++) {
                        for (int64_t j = 0; j < m; j++) col[j] = Scross[j * b + k];
                        or_trsv(Scon, m, col, colx);
                        for (int64_t j = 0; j < m; j++) Scross[j * b + k] = colx[j];
                    }
                    for (int64_t j = 0; j < m; j++) col[j] = y[nn[j]];
                    or_trsv(Scon, m, col, yp);
                    for (int64_t j = 0; j < b; j++)
                        for (int64_t k = 0; k < b; k++) {
                            double s = 0.0;
                            for (int64_t p = 0; p < m; p++) s += Scross[p * b + j] * Scross[p * b + k];
                            Slk[j * b + k] -= s;
                        }
                    for (int64_t j = 0; j < b; j++) {
                        double s = 0.0;
                        for (int64_t p = 0; p < m; p++) s += Scross[p * b + j] * yp[p];
                        mu[j] = s;
                    }
                }
            }
            if (st == OR_OK && or_potrf(Slk, b) != OR_OK) st = OR_ENOTPD;
            if (st == OR_OK)
                for (int64_t j = 0; j < b; j++) {
                    double t = mu[j];
                    for (int64_t k = 0; k <= j; k++) t += Slk[j * b + k] * z[blk[k]];
                    y[blk[j]] = t;
                }
        }
        free(Slk); free(Scon); free(Scross); free(yp); free(col); free(colx); free(mu);
        if (st != OR_OK) return st;
    }
    return OR_OK;
}

/* ------------------------------------------------------------------------------------
 * K-means blocks (Sec. 2.1; Algorithm 1 "Clustering").  The paper names K-means but fixes
 * no initialisation, iteration count, tie rule or empty-cluster rule.  This oracle fixes
 * them so that the result is a deterministic function of (locations, k, seed, iters):
 *
 *  squared distance  D2(x, c) = sum_k (x_k - c_k)^2, left to right, each -, * and + rounded
 *                    separately (no fused multiply-add).
 *  k-means++ seeding (Arthur and Vassilvitskii 2007): the first centre is point
 *                    floor(r_0 n / 2^64); centre t >= 1 is drawn with probability
 *                    proportional to D2 to the nearest chosen centre, computed on integer
 *                    weights w_j = floor(D2_j 2^s) (s fixed from n and the bounding box so
 *                    that sum w < 2^62): target = floor(r_t W / 2^64), W = sum w, and the
 *                    chosen point is the first j whose inclusive prefix sum exceeds target.
 *                    If W = 0 the centre is point floor(r_t n / 2^64).
 *  Lloyd iteration   assign every point to argmin_c D2 (ties: lowest centre index); then
 *                    each centre becomes the mean of its members, computed as
 *                    ((double)S / (double)count) 2^-q from the exact int64 sum S of
 *                    llrint(x 2^q) (q fixed from n and the bounding box); an empty
 *                    cluster keeps its centre.
 *  After `iters` iterations a final assignment gives the labels.
 * r_t is draw t of the SplitMix64 stream OR_STREAM_KPP(seed).
 * ---------------------------------------------------------------------------------- */
static double or_d2(const double* x, const double* c, int d) {
    double acc = 0.0;
    for (int k = 0; k < d; k++) {
        double t = x[k] - c[k];
        double t2 = t * t;
        acc = acc + t2;
    }
    return acc;
}

static int or_ceil_log2_u64(uint64_t v) {
    int e = 0;
    while (e < 64 && ((uint64_t)1 << e) < v) e++;
    return e;
}

/* Exponents that keep the integer sums of the seeding weights and of the centroid
 * coordinates inside int64 (shared definition with the CUDA side, written in both). */
static void or_kmeans_scales(const double* locs, int64_t n, int d, int* s_out, int* q_out) {
    double lo[8], hi[8];
    for (int k = 0; k < d; k++) { lo[k] = locs[k]; hi[k] = locs[k]; }
    for (int64_t i = 0; i < n; i++)
        for (int k = 0; k < d; k++) {
            double v = locs[i * d + k];
            if (v < lo[k]) lo[k] = v;
            if (v > hi[k]) hi[k] = v;
        }
    double d2max = 0.0, amax = 0.0;
    for (int k = 0; k < d; k++) {
        double e = hi[k] - lo[k];
        d2max += e * e;
        if (fabs(lo[k]) > amax) amax = fabs(lo[k]);
        if (fabs(hi[k]) > amax) amax = fabs(hi[k]);
    }
    int ed = 0, ea = 0;
    frexp(d2max, &ed);  /* d2max < 2^ed */
    frexp(amax, &ea);   /* amax  < 2^ea */
    int ln = or_ceil_log2_u64((uint64_t)n);
    *s_out = 61 - ln - (ed + 1);
    *q_out = 61 - ln - (ea + 1);
}

static void or_assign(const double* locs, int64_t n, int d, const double* cent, int64_t k,
                      int32_t* label) {
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) {
        double best = INFINITY;
        int32_t bi = 0;
        for (int64_t c = 0; c < k; c++) {
            double t = or_d2(locs + i * d, cent + c * d, d);
            if (t < best) { best = t; bi = (int32_t)c; }
        }
        label[i] = bi;
    }
}

/* Centroid of the members of every cluster by the exact-integer rule; clusters with no
 * member keep `cent` unchanged.  counts[c] receives the member count. */
static void or_update(const double* locs, int64_t n, int d, const int32_t* label, int64_t k,
                      int q, double* cent, int64_t* counts) {
    int64_t* S = (int64_t*)calloc((size_t)(k * d), sizeof(int64_t));
    for (int64_t c = 0; c < k; c++) counts[c] = 0;
    for (int64_t i = 0; i < n; i++) {
        counts[label[i]]++;
        for (int j = 0; j < d; j++) S[(int64_t)label[i] * d + j] += llrint(ldexp(locs[i * d + j], q));
    }
    for (int64_t c = 0; c < k; c++)
        if (counts[c] > 0)
            for (int j = 0; j < d; j++)
                cent[c * d + j] = ldexp((double)S[c * d + j] / (double)counts[c], -q);
    free(S);
}

int or_kmeans(const double* locs, int64_t n, int d, int64_t k, uint64_t seed, int iters,
              int32_t* label, double* cent) {
    if (n <= 0 || d <= 0 || d > 8 || k <= 0 || k > n || iters < 0) return OR_EINVAL;
    int s = 0, q = 0;
    or_kmeans_scales(locs, n, d, &s, &q);
    uint64_t stream = OR_STREAM_KPP(seed);
    double* D2 = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t* counts = (int64_t*)malloc(sizeof(int64_t) * (size_t)k);
    if (!D2 || !counts) { free(D2); free(counts); return OR_ENOMEM; }
    /* k-means++ seeding */
    int64_t first = (int64_t)or_mulhi(or_sm64(stream, 0), (uint64_t)n);
    for (int j = 0; j < d; j++) cent[j] = locs[first * d + j];
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; i++) D2[i] = or_d2(locs + i * d, cent, d);
    for (int64_t t = 1; t < k; t++) {
        uint64_t W = 0;
        /* exact integer sum: the order of the additions does not matter */
#pragma omp parallel for schedule(static) reduction(+ : W)
        for (int64_t i = 0; i < n; i++) W += (uint64_t)ldexp(D2[i], s);
        uint64_t r = or_sm64(stream, (uint64_t)t);
        int64_t pick;
        if (W == 0) {
            pick = (int64_t)or_mulhi(r, (uint64_t)n);
        } else {
            uint64_t target = or_mulhi(r, W), pre = 0;
            pick = n - 1;
            for (int64_t i = 0; i < n; i++) {
                pre += (uint64_t)ldexp(D2[i], s);
                if (pre > target) { pick = i; break; }
            }
        }
        for (int j = 0; j < d; j++) cent[t * d + j] = locs[pick * d + j];
#pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < n; i++) {
            double v = or_d2(locs + i * d, cent + t * d, d);
            if (v < D2[i]) D2[i] = v;
        }
    }
    /* Lloyd iterations, then the final assignment */
    for (int it = 0; it < iters; it++) {
        or_assign(locs, n, d, cent, k, label);
        or_update(locs, n, d, label, k, q, cent, counts);
    }
    or_assign(locs, n, d, cent, k, label);
    free(D2); free(counts);
    return OR_OK;
}

/* ------------------------------------------------------------------------------------
 * Blocks in permuted order (Algorithm 1 "Clustering" + "Block permutation").
 * Non-empty clusters become blocks (in cluster-index order); zeta is a Fisher-Yates
 * shuffle of the blocks driven by stream OR_STREAM_ZETA(seed): for i = bc-1 .. 1,
 * j = floor(r_i (i+1) / 2^64), swap(perm[i], perm[j]); block position p holds cluster
 * perm[p].  Points inside a block are in ascending original index.  The block centroid
 * (the query point of the neighbour search) is the exact-integer mean of its members.
 * Returns the number of blocks, or a negative error code.
 * ---------------------------------------------------------------------------------- */
int64_t or_build_blocks(const double* locs, int64_t n, int d, int64_t bc, uint64_t seed,
                        int iters, int64_t* block_ptr, int32_t* point_idx, double* centroids) {
    int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* cent = (double*)malloc(sizeof(double) * (size_t)(bc * d));
    int64_t* counts = (int64_t*)calloc((size_t)bc, sizeof(int64_t));
    int64_t* cl2blk = (int64_t*)malloc(sizeof(int64_t) * (size_t)bc);
    if (!label || !cent || !counts || !cl2blk) {
        free(label); free(cent); free(counts); free(cl2blk);
        return -OR_ENOMEM;
    }
    int st = or_kmeans(locs, n, d, bc, seed, iters, label, cent);
    if (st != OR_OK) { free(label); free(cent); free(counts); free(cl2blk); return -st; }
    int s = 0, q = 0;
    or_kmeans_scales(locs, n, d, &s, &q);
    /* block centroids recomputed from the final members */
    or_update(locs, n, d, label, bc, q, cent, counts);
    int64_t nb = 0;
    for (int64_t c = 0; c < bc; c++) cl2blk[c] = counts[c] > 0 ? nb++ : -1;
    int64_t* perm = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb + 1));
    int64_t* clus_of_blk = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nb + 1));
    int64_t* pos_of_clus = (int64_t*)malloc(sizeof(int64_t) * (size_t)bc);
    for (int64_t c = 0; c < bc; c++)
        if (cl2blk[c] >= 0) clus_of_blk[cl2blk[c]] = c;
    for (int64_t p = 0; p < nb; p++) perm[p] = p;
    uint64_t zs = OR_STREAM_ZETA(seed);
    for (int64_t i = nb - 1; i >= 1; i--) {
        int64_t j = (int64_t)or_mulhi(or_sm64(zs, (uint64_t)i), (uint64_t)(i + 1));
        int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (int64_t c = 0; c < bc; c++) pos_of_clus[c] = -1;
    block_ptr[0] = 0;
    for (int64_t p = 0; p < nb; p++) {
        int64_t c = clus_of_blk[perm[p]];
        pos_of_clus[c] = p;
        block_ptr[p + 1] = block_ptr[p] + counts[c];
        for (int j = 0; j < d; j++) centroids[p * d + j] = cent[c * d + j];
    }
    int64_t* fill = (int64_t*)calloc((size_t)(nb + 1), sizeof(int64_t));
    for (int64_t i = 0; i < n; i++) {
        int64_t p = pos_of_clus[label[i]];
        point_idx[block_ptr[p] + fill[p]++] = (int32_t)i;
    }
    free(fill); free(perm); free(clus_of_blk); free(pos_of_clus);
    free(label); free(cent); free(counts); free(cl2blk);
    return nb;
}

/* ------------------------------------------------------------------------------------
 * Classic Vecchia (Sec. 1: the special case of blocks of size 1).  Every point is its own
 * block; the blocks follow a random order drawn by the Fisher-Yates shuffle of the
 * points with the block-permutation stream (for i = n-1 .. 1, j = floor(r_i (i+1) / 2^64),
 * swap(perm[i], perm[j])); a singleton's query point for the neighbour search is the
 * point itself.
 * ---------------------------------------------------------------------------------- */
int or_build_singletons(const double* locs, int64_t n, int d, uint64_t seed, int64_t* block_ptr,
                        int32_t* point_idx, double* centroids) {
    if (n <= 0 || n > INT32_MAX) return OR_EINVAL;
    for (int64_t i = 0; i < n; i++) point_idx[i] = (int32_t)i;
    uint64_t zs = OR_STREAM_ZETA(seed);
    for (int64_t i = n - 1; i >= 1; i--) {
        int64_t j = (int64_t)or_mulhi(or_sm64(zs, (uint64_t)i), (uint64_t)(i + 1));
        int32_t t = point_idx[i]; point_idx[i] = point_idx[j]; point_idx[j] = t;
    }
    for (int64_t p = 0; p <= n; p++) block_ptr[p] = p;
    for (int64_t p = 0; p < n; p++)
        for (int k = 0; k < d; k++) centroids[p * d + k] = locs[(int64_t)point_idx[p] * d + k];
    return OR_OK;
}

/* ------------------------------------------------------------------------------------
 * Block orderings (Sec. 2.1, the five permutations the paper compares; Sec. 3.1 KL study).
 * Each maps the current block sequence (positions 0 .. bc-1, centroids c_p) to a new one:
 * perm[q] = the old position placed at new position q.  Ties always go to the lower old
 * position.
 *   0 random   Fisher-Yates over positions with the block-permutation stream of `seed`
 *   1 maxmin   first the centroid nearest (squared distance) to the mean centroid; then
 *              repeatedly the centroid whose smallest squared distance to those already
 *              placed is largest (Guinness 2018)
 *   2 Morton   Z-order: coordinates scaled to 21-bit integers over the centroids'
 *              bounding box, q_k = min(2^21-1, floor((c_k - lo_k) / (hi_k - lo_k) 2^21)),
 *              bit b of axis k at key bit b d + k; ascending key
 *   3 KD-tree  recursive median split: at depth t sort the set by (coordinate t mod d,
 *              position), the first floor(|S|/2) form the left part, the rest the right;
 *              left before right, down to single blocks (Bentley 1975)
 *   4 Hilbert  the same 21-bit integers mapped to their Hilbert index by Skilling's
 *              axes-to-transpose transform (Skilling 2004), transposed bits read from the
 *              most significant level down, axis 0 first; ascending index
 * ---------------------------------------------------------------------------------- */
typedef struct { uint64_t key; int64_t pos; } or_okey;

static int or_okey_cmp(const void* a, const void* b) {
    const or_okey* x = (const or_okey*)a;
    const or_okey* y = (const or_okey*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

static void or_quantise21(const double* cent, int64_t bc, int d, uint64_t* q) {
    for (int k = 0; k < d; k++) {
        double lo = cent[k], hi = cent[k];
        for (int64_t p = 1; p < bc; p++) {
            if (cent[p * d + k] < lo) lo = cent[p * d + k];
            if (cent[p * d + k] > hi) hi = cent[p * d + k];
        }
        for (int64_t p = 0; p < bc; p++) {
            uint64_t v = 0;
            if (hi > lo) {
                double f = floor((cent[p * d + k] - lo) / (hi - lo) * 2097152.0);
                v = f >= 2097151.0 ? 2097151u : (uint64_t)f;
            }
            q[p * d + k] = v;
        }
    }
}

static uint64_t or_hilbert_key(const uint64_t* coords, int d) {
    uint64_t X[3] = {0, 0, 0};
    for (int i = 0; i < d; i++) X[i] = coords[i];
    const uint64_t M = 1u << 20;
    /* inverse undo of the excess work */
    for (uint64_t Q = M; Q > 1; Q >>= 1) {
        const uint64_t P = Q - 1;
        for (int i = 0; i < d; i++) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                uint64_t t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    /* Gray encode */
    for (int i = 1; i < d; i++) X[i] ^= X[i - 1];
    uint64_t t = 0;
    for (uint64_t Q = M; Q > 1; Q >>= 1)
        if (X[d - 1] & Q) t ^= Q - 1;
    for (int i = 0; i < d; i++) X[i] ^= t;
    uint64_t key = 0;
    for (int b = 20; b >= 0; b--)
        for (int i = 0; i < d; i++) key = (key << 1) | ((X[i] >> b) & 1u);
    return key;
}

static void or_kd_order(const double* cent, int d, int64_t* idx, int64_t n, int depth, or_okey* tmp) {
    if (n <= 1) return;
    const int ax = depth % d;
    /* sort idx[0..n) by (coordinate ax, position): insertion into tmp by qsort on a key
     * built from the coordinate's order-preserving bits */
    for (int64_t i = 0; i < n; i++) {
        double v = cent[idx[i] * d + ax];
        uint64_t u;
        memcpy(&u, &v, sizeof u);
        u = (u >> 63) ? ~u : (u | 0x8000000000000000ULL);
        tmp[i].key = u;
        tmp[i].pos = idx[i];
    }
    qsort(tmp, (size_t)n, sizeof(or_okey), or_okey_cmp);
    for (int64_t i = 0; i < n; i++) idx[i] = tmp[i].pos;
    const int64_t h = n / 2;
    or_kd_order(cent, d, idx, h, depth + 1, tmp);
    or_kd_order(cent, d, idx + h, n - h, depth + 1, tmp);
}

int or_order_blocks(const double* cent, int64_t bc, int d, int order, uint64_t seed, int64_t* perm) {
    if (bc <= 0 || d <= 0 || d > 3) return OR_EINVAL;
    if (order == 0) {
        for (int64_t p = 0; p < bc; p++) perm[p] = p;
        uint64_t zs = OR_STREAM_ZETA(seed);
        for (int64_t i = bc - 1; i >= 1; i--) {
            int64_t j = (int64_t)or_mulhi(or_sm64(zs, (uint64_t)i), (uint64_t)(i + 1));
            int64_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        return OR_OK;
    }
    if (order == 1) {
        double mean[3] = {0, 0, 0};
        for (int k = 0; k < d; k++) {
            double sacc = 0.0;
            for (int64_t p = 0; p < bc; p++) sacc += cent[p * d + k];
            mean[k] = sacc / (double)bc;
        }
        double* dmin = (double*)malloc(sizeof(double) * (size_t)bc);
        char* used = (char*)calloc((size_t)bc, 1);
        if (!dmin || !used) { free(dmin); free(used); return OR_ENOMEM; }
        int64_t first = 0;
        double best = INFINITY;
        for (int64_t p = 0; p < bc; p++) {
            double v = or_d2(cent + p * d, mean, d);
            if (v < best) { best = v; first = p; }
        }
        perm[0] = first;
        used[first] = 1;
        for (int64_t p = 0; p < bc; p++) dmin[p] = or_d2(cent + p * d, cent + first * d, d);
        for (int64_t q = 1; q < bc; q++) {
            int64_t pick = -1;
            double far = -1.0;
            for (int64_t p = 0; p < bc; p++)
                if (!used[p] && dmin[p] > far) { far = dmin[p]; pick = p; }
            perm[q] = pick;
            used[pick] = 1;
            for (int64_t p = 0; p < bc; p++) {
                double v = or_d2(cent + p * d, cent + pick * d, d);
                if (v < dmin[p]) dmin[p] = v;
            }
        }
        free(dmin); free(used);
        return OR_OK;
    }
    if (order == 2 || order == 4) {
        uint64_t* q = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(bc * d));
        or_okey* k = (or_okey*)malloc(sizeof(or_okey) * (size_t)bc);
        if (!q || !k) { free(q); free(k); return OR_ENOMEM; }
        or_quantise21(cent, bc, d, q);
        for (int64_t p = 0; p < bc; p++) {
            uint64_t key = 0;
            if (order == 2) {
                for (int b = 0; b < 21; b++)
                    for (int a = 0; a < d; a++) key |= ((q[p * d + a] >> b) & 1u) << (b * d + a);
            } else {
                key = or_hilbert_key(q + p * d, d);
            }
            k[p].key = key;
            k[p].pos = p;
        }
        qsort(k, (size_t)bc, sizeof(or_okey), or_okey_cmp);
        for (int64_t p = 0; p < bc; p++) perm[p] = k[p].pos;
        free(q); free(k);
        return OR_OK;
    }
    if (order == 3) {
        or_okey* tmp = (or_okey*)malloc(sizeof(or_okey) * (size_t)bc);
        if (!tmp) return OR_ENOMEM;
        for (int64_t p = 0; p < bc; p++) perm[p] = p;
        or_kd_order(cent, d, perm, bc, 0, tmp);
        free(tmp);
        return OR_OK;
    }
    return OR_EINVAL;
}

uint64_t or_hilbert_index(const uint64_t* coords, int d) { return or_hilbert_key(coords, d); }

/* ------------------------------------------------------------------------------------
 * Block nearest neighbours (Sec. 2.2; Algorithm 1 "Nearest neighbors").  For the block
 * at position i, the candidates are all points of the blocks at positions 0 .. i-1; the
 * query is the block centroid; the key of a candidate j is (D2(centroid, s_j), j) with D2
 * as in K-means; the conditioning set is the m_i smallest keys in ascending key order,
 * m_i = min(m or m_per_block[i], number of candidates).  The first block has none.
 * nn_ptr[bc+1] is filled; nn_idx must hold sum_i m_i entries (pass NULL to size only).
 * ---------------------------------------------------------------------------------- */
typedef struct { double d2; int32_t idx; } or_key;

static int or_key_less(or_key a, or_key b) {
    return a.d2 < b.d2 || (a.d2 == b.d2 && a.idx < b.idx);
}

/* max-heap of the m best keys seen so far */
static void or_heap_sift_down(or_key* h, int64_t sz, int64_t i) {
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, g = i;
        if (l < sz && or_key_less(h[g], h[l])) g = l;
        if (r < sz && or_key_less(h[g], h[r])) g = r;
        if (g == i) return;
        or_key t = h[i]; h[i] = h[g]; h[g] = t;
        i = g;
    }
}
static void or_heap_sift_up(or_key* h, int64_t i) {
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!or_key_less(h[p], h[i])) return;
        or_key t = h[i]; h[i] = h[p]; h[p] = t;
        i = p;
    }
}
static int or_key_cmp(const void* a, const void* b) {
    or_key x = *(const or_key*)a, y = *(const or_key*)b;
    if (or_key_less(x, y)) return -1;
    if (or_key_less(y, x)) return 1;
    return 0;
}

int or_select_neighbors(const double* locs, int64_t n, int d, int64_t bc,
                        const int64_t* block_ptr, const int32_t* point_idx,
                        const double* centroids, int32_t m, const int32_t* m_per_block,
                        int64_t* nn_ptr, int32_t* nn_idx) {
    (void)n;
    nn_ptr[0] = 0;
    for (int64_t i = 0; i < bc; i++) {
        int64_t want = m_per_block ? m_per_block[i] : m;
        if (want < 0) return OR_EINVAL;
        int64_t cand = block_ptr[i];
        nn_ptr[i + 1] = nn_ptr[i] + (want < cand ? want : cand);
    }
    if (!nn_idx) return OR_OK;
    int fail = OR_OK;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < bc; i++) {
        int64_t mi = nn_ptr[i + 1] - nn_ptr[i];
        if (mi == 0) continue;
        or_key* h = (or_key*)malloc(sizeof(or_key) * (size_t)mi);
        if (!h) { fail = OR_ENOMEM; continue; }
        int64_t sz = 0;
        const double* q = centroids + i * d;
        for (int64_t p = 0; p < block_ptr[i]; p++) {
            or_key key;
            key.idx = point_idx[p];
            key.d2 = or_d2(q, locs + (int64_t)key.idx * d, d);
            if (sz < mi) {
                h[sz] = key;
                or_heap_sift_up(h, sz);
                sz++;
            } else if (or_key_less(key, h[0])) {
                h[0] = key;
                or_heap_sift_down(h, sz, 0);
            }
        }
        qsort(h, (size_t)sz, sizeof(or_key), or_key_cmp);
        for (int64_t t = 0; t < sz; t++) nn_idx[nn_ptr[i] + t] = h[t].idx;
        free(h);
    }
    return fail;
}

/* ------------------------------------------------------------------------------------
 * Prediction (Sec. 2.4 "Block Vecchia Prediction", Algorithm 2).
 *
 * Clustering g: the new locations S* are split into blocks by the same K-means as
 * Algorithm 1 (same seeding, iterations and exact-integer conventions).  Algorithm 2 has
 * no block permutation (prediction blocks do not condition on one another), so blocks
 * keep cluster-index order, empty clusters dropped, members ascending, and the centroid
 * is the exact-integer mean of the members.
 * ---------------------------------------------------------------------------------- */
int64_t or_build_pred_blocks(const double* locs_star, int64_t n_star, int d, int64_t bc,
                             uint64_t seed, int iters, int64_t* block_ptr, int32_t* point_idx,
                             double* centroids) {
    int32_t* label = (int32_t*)malloc(sizeof(int32_t) * (size_t)n_star);
    double* cent = (double*)malloc(sizeof(double) * (size_t)(bc * d));
    int64_t* counts = (int64_t*)calloc((size_t)bc, sizeof(int64_t));
    int64_t* fill = (int64_t*)calloc((size_t)bc + 1, sizeof(int64_t));
    int64_t* blk_of = (int64_t*)malloc(sizeof(int64_t) * (size_t)bc);
    if (!label || !cent || !counts || !fill || !blk_of) {
        free(label); free(cent); free(counts); free(fill); free(blk_of);
        return -OR_ENOMEM;
    }
    int st = or_kmeans(locs_star, n_star, d, bc, seed, iters, label, cent);
    if (st != OR_OK) { free(label); free(cent); free(counts); free(fill); free(blk_of); return -st; }
    int s = 0, q = 0;
    or_kmeans_scales(locs_star, n_star, d, &s, &q);
    or_update(locs_star, n_star, d, label, bc, q, cent, counts);
    int64_t nb = 0;
    block_ptr[0] = 0;
    for (int64_t c = 0; c < bc; c++) {
        blk_of[c] = -1;
        if (counts[c] == 0) continue;
        blk_of[c] = nb;
        block_ptr[nb + 1] = block_ptr[nb] + counts[c];
        for (int j = 0; j < d; j++) centroids[nb * d + j] = cent[c * d + j];
        nb++;
    }
    for (int64_t i = 0; i < n_star; i++) {
        int64_t p = blk_of[label[i]];
        point_idx[block_ptr[p] + fill[p]++] = (int32_t)i;
    }
    free(label); free(cent); free(counts); free(fill); free(blk_of);
    return nb;
}

/* Algorithm 2 "Nearest neighbors": for prediction block i the candidates are all n
 * observations; the query is the block centroid; key (D2, index) as in Algorithm 1; the
 * conditioning set is the min(m, n) smallest keys in ascending key order. */
int or_select_pred_neighbors(const double* locs, int64_t n, int d, int64_t bc,
                             const double* centroids, int32_t m, int64_t* nn_ptr,
                             int32_t* nn_idx) {
    if (m < 0) return OR_EINVAL;
    const int64_t mi = m < n ? m : n;
    nn_ptr[0] = 0;
    for (int64_t i = 0; i < bc; i++) nn_ptr[i + 1] = nn_ptr[i] + mi;
    if (!nn_idx || mi == 0) return OR_OK;
    int fail = OR_OK;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < bc; i++) {
        or_key* h = (or_key*)malloc(sizeof(or_key) * (size_t)mi);
        if (!h) { fail = OR_ENOMEM; continue; }
        int64_t sz = 0;
        const double* qc = centroids + i * d;
        for (int64_t j = 0; j < n; j++) {
            or_key key;
            key.idx = (int32_t)j;
            key.d2 = or_d2(qc, locs + j * d, d);
            if (sz < mi) {
                h[sz] = key;
                or_heap_sift_up(h, sz);
                sz++;
            } else if (or_key_less(key, h[0])) {
                h[0] = key;
                or_heap_sift_down(h, sz, 0);
            }
        }
        qsort(h, (size_t)sz, sizeof(or_key), or_key_cmp);
        for (int64_t t = 0; t < sz; t++) nn_idx[nn_ptr[i] + t] = h[t].idx;
        free(h);
    }
    return fail;
}

/* Solve Sigma x = b with the Cholesky factor L of Sigma (forward, then backward
 * substitution with L^T). */
static void or_chol_solve(const double* L, int64_t n, const double* b, double* x) {
    for (int64_t i = 0; i < n; i++) {
        double t = b[i];
        for (int64_t k = 0; k < i; k++) t -= L[i * n + k] * x[k];
        x[i] = t / L[i * n + i];
    }
    for (int64_t i = n - 1; i >= 0; i--) {
        double t = x[i];
        for (int64_t k = i + 1; k < n; k++) t -= L[k * n + i] * x[k];
        x[i] = t / L[i * n + i];
    }
}

/* One prediction block, literally Algorithm 2:
 *   Sigma^con = cov(S_NN, S_NN), Sigma^cross = cov(S_NN, S_B*) (m x b), Sigma^lk =
 *   cov(S_B*, S_B*) with the nugget on the diagonal (a new location is its own point and
 *   is never the same point as an observation);
 *   mu = Sigma^cross^T (Sigma^con)^{-1} y_NN;
 *   Sigma_B = Sigma^lk - Sigma^cross^T (Sigma^con)^{-1} Sigma^cross.
 * mean[b] and cov[b x b] (row-major) are outputs. */
int or_predict_block(const or_theta* th, const double* locs, const double* y, int d,
                     const int32_t* nn, int64_t m, const double* locs_star, const int32_t* blk,
                     int64_t b, double* mean, double* cov) {
    double* Scon = (double*)calloc((size_t)(m * m + 1), sizeof(double));
    double* Scross = (double*)calloc((size_t)(m * b + 1), sizeof(double));
    double* W = (double*)calloc((size_t)(m * b + 1), sizeof(double));
    double* rhs = (double*)calloc((size_t)(m + 1), sizeof(double));
    double* x = (double*)calloc((size_t)(m + 1), sizeof(double));
    int st = OR_OK;
    if (!Scon || !Scross || !W || !rhs || !x) { st = OR_ENOMEM; goto done; }
    for (int64_t j = 0; j < b; j++)
        for (int64_t k = 0; k < b; k++)
            cov[j * b + k] = or_cov(th, d, locs_star + (int64_t)blk[j] * d,
                                    locs_star + (int64_t)blk[k] * d, blk[j] == blk[k]);
    for (int64_t j = 0; j < b; j++) mean[j] = 0.0;
    if (m == 0) goto done;
    for (int64_t j = 0; j < m; j++)
        for (int64_t k = 0; k < m; k++)
            Scon[j * m + k] = or_cov(th, d, locs + (int64_t)nn[j] * d, locs + (int64_t)nn[k] * d,
                                     nn[j] == nn[k]);
    for (int64_t j = 0; j < m; j++)
        for (int64_t k = 0; k < b; k++)
            Scross[j * b + k] = or_cov(th, d, locs + (int64_t)nn[j] * d,
                                       locs_star + (int64_t)blk[k] * d, 0);
    if (or_potrf(Scon, m) != OR_OK) { st = OR_ENOTPD; goto done; }
    /* (Sigma^con)^{-1} y_NN, then mu = Sigma^cross^T times it */
    for (int64_t j = 0; j < m; j++) rhs[j] = y[nn[j]];
    or_chol_solve(Scon, m, rhs, x);
    for (int64_t k = 0; k < b; k++) {
        double t = 0.0;
        for (int64_t j = 0; j < m; j++) t += Scross[j * b + k] * x[j];
        mean[k] = t;
    }
    /* W = (Sigma^con)^{-1} Sigma^cross, column by column; Sigma_B = Sigma^lk - Sigma^cross^T W */
    for (int64_t k = 0; k < b; k++) {
        for (int64_t j = 0; j < m; j++) rhs[j] = Scross[j * b + k];
        or_chol_solve(Scon, m, rhs, x);
        for (int64_t j = 0; j < m; j++) W[j * b + k] = x[j];
    }
    for (int64_t r = 0; r < b; r++)
        for (int64_t c = 0; c < b; c++) {
            double t = 0.0;
            for (int64_t j = 0; j < m; j++) t += Scross[j * b + r] * W[j * b + c];
            cov[r * b + c] -= t;
        }
done:
    free(Scon); free(Scross); free(W); free(rhs); free(x);
    return st;
}

/* Algorithm 2 over all blocks: mean[n_star] and var[n_star] (the diagonal of the block's
 * Sigma_B) by new-location index; cov_packed (optional) receives each block's Sigma_B
 * lower triangle, row by row, blocks in order (sum_i b_i (b_i + 1) / 2 entries). */
int or_predict(const or_theta* th, const double* locs, const double* y, int64_t n, int d,
               const double* locs_star, int64_t bc, const int64_t* block_ptr,
               const int32_t* point_idx, const int64_t* nn_ptr, const int32_t* nn_idx,
               double* mean, double* var, double* cov_packed) {
    (void)n;
    if (!or_theta_valid(th, d)) return OR_EINVAL;
    int fail = OR_OK;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = 0; i < bc; i++) {
        const int64_t b = block_ptr[i + 1] - block_ptr[i];
        const int32_t* blk = point_idx + block_ptr[i];
        double* mu = (double*)malloc(sizeof(double) * (size_t)(b + 1));
        double* C = (double*)malloc(sizeof(double) * (size_t)(b * b + 1));
        int st = (mu && C) ? or_predict_block(th, locs, y, d, nn_idx + nn_ptr[i], nn_ptr[i + 1] - nn_ptr[i],
                                              locs_star, blk, b, mu, C)
                           : OR_ENOMEM;
        if (st == OR_OK) {
            for (int64_t j = 0; j < b; j++) {
                mean[blk[j]] = mu[j];
                var[blk[j]] = C[j * b + j];
            }
            if (cov_packed) {
                int64_t off = 0;
                /* packed offset: sum over earlier blocks of b_k (b_k + 1) / 2 */
                for (int64_t k = 0; k < i; k++) {
                    const int64_t bk = block_ptr[k + 1] - block_ptr[k];
                    off += bk * (bk + 1) / 2;
                }
                for (int64_t r = 0; r < b; r++)
                    for (int64_t c = 0; c <= r; c++) cov_packed[off + r * (r + 1) / 2 + c] = C[r * b + c];
            }
        } else {
#pragma omp critical
            if (fail == OR_OK) fail = st;
        }
        free(mu); free(C);
    }
    return fail;
}

/* ------------------------------------------------------------------------------------
 * Univariate conditional simulation and the prediction interval (Sec. 2.4, last
 * paragraph; PICP of Sec. 3.2).  For new location j, draw r = 0 .. R-1 is
 * y_jr = mean_j + sqrt(var_j) z_jr with z_jr standard normal by the Box-Muller transform
 * (Box and Muller 1958), which turns two uniforms into two independent normals: pair
 * k = 0 .. ceil(R/2)-1 of location j uses c = j ceil(R/2) + k,
 *   u1 = 1 - (x_{2c} >> 11) 2^-53, u2 = (x_{2c+1} >> 11) 2^-53, rho = sqrt(-2 ln u1),
 *   z_{j,2k} = rho cos(2 pi u2),  z_{j,2k+1} = rho sin(2 pi u2)  (dropped when 2k+1 = R),
 * x_i = draw i of the SplitMix64 stream seed ^ "condsim_".  The sample mean and the sample
 * variance (divisor R - 1) of the y_jr give the interval [mean~ - z_crit sd~,
 * mean~ + z_crit sd~]; covered counts the held-out values inside it.
 * ---------------------------------------------------------------------------------- */
#define OR_STREAM_CSIM(seed) ((seed) ^ 0x636f6e6473696d5fULL) /* "condsim_" */

/* Normal number r of location j (pairs as above). */
double or_csim_normal(uint64_t seed, int64_t j, int32_t rounds, int32_t r) {
    const uint64_t st = OR_STREAM_CSIM(seed);
    const uint64_t half = ((uint64_t)rounds + 1) / 2;
    const uint64_t c = (uint64_t)j * half + (uint64_t)(r / 2);
    const double u1 = 1.0 - (double)(or_sm64(st, 2 * c) >> 11) * 0x1p-53;
    const double u2 = (double)(or_sm64(st, 2 * c + 1) >> 11) * 0x1p-53;
    const double rho = sqrt(-2.0 * log(u1));
    return (r % 2 == 0) ? rho * cos(2.0 * M_PI * u2) : rho * sin(2.0 * M_PI * u2);
}

int or_cond_sim(const double* mean, const double* var, int64_t n_star, int32_t rounds,
                uint64_t seed, double z_crit, const double* y_true, double* lower, double* upper,
                int64_t* covered) {
    if (rounds < 2 || n_star < 0) return OR_EINVAL;
    int64_t cov_count = 0;
#pragma omp parallel for schedule(static) reduction(+ : cov_count)
    for (int64_t i = 0; i < n_star; i++) {
        const double sd = sqrt(var[i] > 0.0 ? var[i] : 0.0);
        double sum = 0.0;
        for (int32_t r = 0; r < rounds; r++)
            sum += mean[i] + sd * or_csim_normal(seed, i, rounds, r);
        const double mt = sum / (double)rounds;
        double ss = 0.0;
        for (int32_t r = 0; r < rounds; r++) {
            const double e = mean[i] + sd * or_csim_normal(seed, i, rounds, r) - mt;
            ss += e * e;
        }
        const double st = sqrt(ss / (double)(rounds - 1));
        lower[i] = mt - z_crit * st;
        upper[i] = mt + z_crit * st;
        if (y_true && y_true[i] >= lower[i] && y_true[i] <= upper[i]) cov_count++;
    }
    if (covered) *covered = cov_count;
    return OR_OK;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads used by the parallel loops that the calling thread starts from now on (the
 * CPU baseline is timed both on every host core and on one). */
void or_set_num_threads(int k) {
#ifdef _OPENMP
    if (k >= 1) omp_set_num_threads(k);
#else
    (void)k;
#endif
}
