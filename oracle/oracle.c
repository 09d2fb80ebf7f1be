/*
 * Reference oracle for the all-families regression scores of arXiv 1901.07643.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark load it.  It shares no code with the CUDA library.
 *
 * What it computes (the plain definition the paper's method reaches exactly,
 * up to rounding order; abstract and Sec. 1, "exact calculation of regressions
 * for all child and parent-set combinations"):
 *
 *   for every child c in {0..m-1} and every parent set S of the other m-1
 *   variables (m * 2^(m-1) families, the count given in Sec. 1):
 *     1. Xc = X minus its column means (two-pass means, FP64).
 *     2. RSS(c|S) = squared norm of the least-squares residual of column c of
 *        Xc on the columns S of Xc (S empty: the centred sum of squares).
 *        The residual is formed with plain Householder QR of the n x (|S|+1)
 *        matrix [Xc_S (ascending variable index) | Xc_c], which is the "QRD of
 *        a family" of Sec. 1.1: after |S| reflections the trailing entries of
 *        the last column hold the residual.
 *     3. score(c|S) = n*ln(RSS/n) + |S|*ln(n)  (BIC-style local score; the
 *        paper leaves the score open, Sec. 1, so this one is fixed here).
 *   stored at idx(c,S) = c*2^(m-1) + compress(S,c), where compress deletes
 *   bit c from the m-bit mask of S.
 *
 * The "R0-reduced" variant runs step 2 on the m x m triangular factor R0 of
 * Xc (itself computed by the same Householder routine) instead of on Xc.
 * Because Xc_S = Q*R0_S with Q orthonormal, the residual norms agree
 * exactly; it exists so that m=20 can be checked in full in seconds.
 *
 * The gradient oracle differentiates sum_f w_f*score_f with respect to X in
 * closed form: per family beta = argmin |Xc_c - Xc_S beta|, e the residual,
 * d RSS/d Xc_c = 2e, d RSS/d Xc_S = -2 e beta^T, d score/d RSS = n/RSS, then
 * the centring adjoint (subtract each column's mean).
 *
 * Compiled with -O2 -ffp-contract=off (no fused multiply-add) so that every
 * operation is a separately rounded IEEE double operation.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* planted-mistake switch used only by the oracle's own mutation tests */
static int g_mutation = 0;
void oracle_set_mutation(int code) { g_mutation = code; }

int oracle_num_threads(int requested) {
#ifdef _OPENMP
    if (requested > 0) return requested;
    return omp_get_max_threads();
#else
    (void)requested;
    return 1;
#endif
}

/* Step 1: centre the columns of the row-major n x m matrix X (two-pass mean). */
void oracle_center(const double* X, int64_t n, int32_t m, double* Xc) {
    for (int32_t j = 0; j < m; ++j) {
        double s = 0.0;
        for (int64_t t = 0; t < n; ++t) s += X[t * m + j];
        double mu = s / (double)n;
        if (g_mutation == 1) mu = 0.0; /* planted: skip centring */
        for (int64_t t = 0; t < n; ++t) Xc[t * m + j] = X[t * m + j] - mu;
    }
}

/* compress(S,c): delete bit c of the parent mask S (S never contains c). */
uint64_t oracle_compress(uint64_t S, int32_t c) {
    uint64_t low = S & ((1ull << c) - 1ull);
    uint64_t high = (S >> (c + 1)) << c;
    if (g_mutation == 2) high = (S >> c) << c; /* planted: bit not removed */
    return low | high;
}

/*
 * Householder QR of the column-major rows x ncol matrix A (leading dimension
 * rows), applied in place to the first `nref` columns and to all later ones.
 * After the call, column j (j < nref) holds R's column above the diagonal and
 * the trailing columns hold Q^T times their original content.
 */
static void householder_inplace(double* A, int64_t rows, int32_t ncol, int32_t nref) {
    for (int32_t j = 0; j < nref && j < rows; ++j) {
        double* a = A + (int64_t)j * rows;
        double nrm2 = 0.0;
        for (int64_t t = j; t < rows; ++t) nrm2 += a[t] * a[t];
        double nrm = sqrt(nrm2);
        if (nrm == 0.0) continue;            /* zero column: reflection is I */
        double alpha = (a[j] >= 0.0) ? -nrm : nrm;
        /* v = a(j:) - alpha e_j, stored in a(j:) ; v^T v = 2 nrm (nrm + |a_j|) */
        double v0 = a[j] - alpha;
        double vtv = 2.0 * nrm * (nrm + fabs(a[j]));
        a[j] = v0;
        for (int32_t l = j + 1; l < ncol; ++l) {
            double* b = A + (int64_t)l * rows;
            double dot = 0.0;
            for (int64_t t = j; t < rows; ++t) dot += a[t] * b[t];
            double f = 2.0 * dot / vtv;
            if (g_mutation == 3) f = -f; /* planted: wrong sign in the update */
            for (int64_t t = j; t < rows; ++t) b[t] -= f * a[t];
        }
        a[j] = alpha;
        for (int64_t t = j + 1; t < rows; ++t) a[t] = 0.0;
    }
}

/*
 * RSS of column c on the columns in mask S of the row-major rows x m matrix A.
 * work must hold rows*(m+1) doubles.
 */
double oracle_family_rss(const double* A, int64_t rows, int32_t m, int32_t c, uint64_t S,
                         double* work) {
    int32_t k = 0;
    for (int32_t v = 0; v < m; ++v) {
        if (!((S >> v) & 1ull)) continue;
        for (int64_t t = 0; t < rows; ++t) work[(int64_t)k * rows + t] = A[t * m + v];
        ++k;
    }
    double* y = work + (int64_t)k * rows;
    for (int64_t t = 0; t < rows; ++t) y[t] = A[t * m + c];
    householder_inplace(work, rows, k + 1, k);
    double rss = 0.0;
    int64_t first = k;
    if (g_mutation == 4) first = k + 1; /* planted: drop one residual term */
    for (int64_t t = first; t < rows; ++t) rss += y[t] * y[t];
    return rss;
}

/* Penalised local score n*ln(RSS/n) + k*lam: lam = ln(n) is the BIC-style
 * score of the benchmark configurations, lam = 2 the AIC form (the paper
 * leaves the score open, Sec. 1; only the RSS is the method's result). */
double oracle_score(double rss, int64_t n, int32_t k, double lam) {
    double pen = (double)k;
    if (g_mutation == 5) pen = (double)(k + 1); /* planted: penalty off by one */
    return (double)n * log(rss / (double)n) + pen * lam;
}

double oracle_bic(double rss, int64_t n, int32_t k) { return oracle_score(rss, n, k, log((double)n)); }

/* Householder R factor (m x m, row-major, upper triangular) of row-major A. */
void oracle_r_factor(const double* A, int64_t rows, int32_t m, double* R) {
    double* w = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)m);
    for (int32_t j = 0; j < m; ++j)
        for (int64_t t = 0; t < rows; ++t) w[(int64_t)j * rows + t] = A[t * m + j];
    householder_inplace(w, rows, m, m);
    for (int32_t i = 0; i < m; ++i)
        for (int32_t j = 0; j < m; ++j)
            R[i * m + j] = (i <= j && i < rows) ? w[(int64_t)j * rows + i] : 0.0;
    free(w);
}

static int popcount64(uint64_t x) {
    int c = 0;
    while (x) { x &= x - 1; ++c; }
    return c;
}

/*
 * Fill rss_out and/or score_out (either may be NULL) for every family, using
 * the rows x m matrix A as the data (A = Xc for the direct oracle, A = R0 for
 * the reduced one).  n is the sample count used by the score.
 */
static void all_families(const double* A, int64_t rows, int32_t m, int64_t n, double* rss_out,
                         double* score_out, int nthreads) {
    const int64_t half = 1ll << (m - 1);
    const int64_t total = (int64_t)m * half;
#ifdef _OPENMP
#pragma omp parallel num_threads(oracle_num_threads(nthreads))
#endif
    {
        double* work = (double*)malloc(sizeof(double) * (size_t)rows * (size_t)(m + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 256)
#endif
        for (int64_t f = 0; f < total; ++f) {
            int32_t c = (int32_t)(f / half);
            uint64_t comp = (uint64_t)(f % half);
            /* expand: re-insert a zero bit at position c */
            uint64_t S = (comp & ((1ull << c) - 1ull)) | ((comp >> c) << (c + 1));
            double rss = oracle_family_rss(A, rows, m, c, S, work);
            int64_t slot = (int64_t)c * half + (int64_t)oracle_compress(S, c);
            if (rss_out) rss_out[slot] = rss;
            if (score_out) score_out[slot] = oracle_bic(rss, n, popcount64(S));
        }
        free(work);
    }
}

/* Scores with penalty lam per parent from a table of RSS in table layout. */
void oracle_table_scores(const double* rss, int64_t n, int32_t m, double lam, double* score) {
    const int64_t half = 1ll << (m - 1);
    for (int64_t f = 0; f < (int64_t)m * half; ++f)
        score[f] = oracle_score(rss[f], n, popcount64((uint64_t)(f % half)), lam);
}

/*
 * Least-squares coefficients of listed families, directly on the centred data
 * (Sec. 1.1: the regression of child[i] on the parents in mask[i]): Householder
 * QR of [Xc_S | Xc_c], then back substitution R b = (Q^T y)(0:k).  beta holds
 * m + 1 doubles per family: b_v at index v for v in S, 0 elsewhere, and the
 * intercept mean_c - sum_v b_v mean_v of the uncentred regression at index m.
 * Numerically dependent parents -- a pivot |r_jj| (parent j's residual on the
 * parents before it) at most 1e-12 times the norm of parent j's column --
 * give NaN coefficients; the RSS is still returned.
 */
int oracle_coefficients(const double* X, int64_t n, int32_t m, const int32_t* child,
                        const uint64_t* mask, int64_t count, double* beta, double* rss_out,
                        int nthreads) {
    if (m < 1 || m > 30 || n < 1) return -1;
    double* Xc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double mu[32];
    oracle_center(X, n, m, Xc);
    for (int32_t j = 0; j < m; ++j) { /* the column means, summed as in oracle_center */
        double s = 0.0;
        for (int64_t t = 0; t < n; ++t) s += X[t * m + j];
        mu[j] = s / (double)n;
    }
#ifdef _OPENMP
#pragma omp parallel num_threads(oracle_num_threads(nthreads))
#endif
    {
        double* work = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < count; ++i) {
            const int32_t c = child[i];
            const uint64_t S = mask[i];
            double* b = beta + i * (int64_t)(m + 1);
            int32_t cols[32];
            double bk[32], norm[32];
            int32_t k = 0;
            for (int32_t v = 0; v < m; ++v) {
                b[v] = 0.0;
                if (!((S >> v) & 1ull)) continue;
                cols[k] = v;
                double s2 = 0.0;
                for (int64_t t = 0; t < n; ++t) {
                    work[(int64_t)k * n + t] = Xc[t * m + v];
                    s2 += Xc[t * m + v] * Xc[t * m + v];
                }
                norm[k] = sqrt(s2);
                ++k;
            }
            double* y = work + (int64_t)k * n;
            for (int64_t t = 0; t < n; ++t) y[t] = Xc[t * m + c];
            householder_inplace(work, n, k + 1, k);
            int singular = 0;
            for (int32_t r = k - 1; r >= 0; --r) {
                double s = y[r];
                for (int32_t j = r + 1; j < k; ++j) s -= work[(int64_t)j * n + r] * bk[j];
                const double rii = work[(int64_t)r * n + r];
                if (!(fabs(rii) > 1e-12 * norm[r])) singular = 1;
                bk[r] = s / rii;
            }
            double rss = 0.0;
            for (int64_t t = k; t < n; ++t) rss += y[t] * y[t];
            double icpt = mu[c];
            for (int32_t j = 0; j < k; ++j) {
                const double bj = singular ? NAN : bk[j];
                b[cols[j]] = bj;
                icpt -= bj * mu[cols[j]];
            }
            b[m] = icpt;
            if (rss_out) rss_out[i] = rss;
        }
        free(work);
    }
    free(Xc);
    return 0;
}

/* Direct oracle: every family solved on the centred data. */
int oracle_scores(const double* X, int64_t n, int32_t m, double* rss_out, double* score_out,
                  int nthreads) {
    if (m < 1 || m > 30 || n < 1) return -1;
    double* Xc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
    oracle_center(X, n, m, Xc);
    all_families(Xc, n, m, n, rss_out, score_out, nthreads);
    free(Xc);
    return 0;
}

/* R0-reduced oracle: every family solved on the m x m factor R0 of Xc. */
int oracle_scores_reduced(const double* X, int64_t n, int32_t m, double* rss_out,
                          double* score_out, int nthreads) {
    if (m < 1 || m > 30 || n < 1) return -1;
    double* Xc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double* R0 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)m);
    oracle_center(X, n, m, Xc);
    oracle_r_factor(Xc, n, m, R0);
    all_families(R0, m, m, n, rss_out, score_out, nthreads);
    free(R0);
    free(Xc);
    return 0;
}

/* A list of families (child[i], parent mask[i]) solved directly on Xc. */
int oracle_scores_sampled(const double* X, int64_t n, int32_t m, const int32_t* child,
                          const uint64_t* mask, int64_t count, double* rss_out, double* score_out,
                          int nthreads) {
    if (m < 1 || m > 30 || n < 1) return -1;
    double* Xc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
    oracle_center(X, n, m, Xc);
#ifdef _OPENMP
#pragma omp parallel num_threads(oracle_num_threads(nthreads))
#endif
    {
        double* work = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (int64_t i = 0; i < count; ++i) {
            double rss = oracle_family_rss(Xc, n, m, child[i], mask[i], work);
            if (rss_out) rss_out[i] = rss;
            if (score_out) score_out[i] = oracle_bic(rss, n, popcount64(mask[i]));
        }
        free(work);
    }
    free(Xc);
    return 0;
}

/* A list of families solved on the oracle's own m x m Householder factor R0
 * of Xc (the R0-reduced variant: identical in exact arithmetic, m rows per
 * family instead of n). */
int oracle_scores_sampled_reduced(const double* X, int64_t n, int32_t m, const int32_t* child,
                                  const uint64_t* mask, int64_t count, double* rss_out,
                                  double* score_out, int nthreads) {
    if (m < 1 || m > 30 || n < 1) return -1;
    double* Xc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
    double* R0 = (double*)malloc(sizeof(double) * (size_t)m * (size_t)m);
    oracle_center(X, n, m, Xc);
    oracle_r_factor(Xc, n, m, R0);
#ifdef _OPENMP
#pragma omp parallel num_threads(oracle_num_threads(nthreads))
#endif
    {
        double* work = (double*)malloc(sizeof(double) * (size_t)m * (size_t)(m + 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1024)
#endif
        for (int64_t i = 0; i < count; ++i) {
            double rss = oracle_family_rss(R0, m, m, child[i], mask[i], work);
            if (rss_out) rss_out[i] = rss;
            if (score_out) score_out[i] = oracle_bic(rss, n, popcount64(mask[i]));
        }
        free(work);
    }
    free(R0);
    free(Xc);
    return 0;
}

/*
 * Gradient of sum_f w_f * score_f with respect to X (row-major n x m), where w
 * uses the table layout of the scores.  gX must hold n*m doubles.
 */
int oracle_grad(const double* X, int64_t n, int32_t m, const double* w, double* gX,
                int nthreads) {
    if (m < 1 || m > 30 || n < 1) return -1;
    const int64_t half = 1ll << (m - 1);
    const int64_t total = (int64_t)m * half;
    double* Xc = (double*)malloc(sizeof(double) * (size_t)n * (size_t)m);
    oracle_center(X, n, m, Xc);
    int nt = oracle_num_threads(nthreads);
    double* G = (double*)calloc((size_t)nt * (size_t)n * (size_t)m, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* Gt = G + (size_t)tid * (size_t)n * (size_t)m;
        double* work = (double*)malloc(sizeof(double) * (size_t)n * (size_t)(m + 1));
        double* e = (double*)malloc(sizeof(double) * (size_t)n);
        double beta[32];
        int32_t cols[32];
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 64)
#endif
        for (int64_t f = 0; f < total; ++f) {
            int32_t c = (int32_t)(f / half);
            uint64_t comp = (uint64_t)(f % half);
            uint64_t S = (comp & ((1ull << c) - 1ull)) | ((comp >> c) << (c + 1));
            double wf = w[(int64_t)c * half + (int64_t)oracle_compress(S, c)];
            if (wf == 0.0) continue;
            int32_t k = 0;
            for (int32_t v = 0; v < m; ++v) {
                if (!((S >> v) & 1ull)) continue;
                cols[k] = v;
                for (int64_t t = 0; t < n; ++t) work[(int64_t)k * n + t] = Xc[t * m + v];
                ++k;
            }
            double* y = work + (int64_t)k * n;
            for (int64_t t = 0; t < n; ++t) y[t] = Xc[t * m + c];
            householder_inplace(work, n, k + 1, k);
            /* back substitution R beta = (Q^T y)(0:k) */
            for (int32_t i = k - 1; i >= 0; --i) {
                double s = y[i];
                for (int32_t j = i + 1; j < k; ++j) s -= work[(int64_t)j * n + i] * beta[j];
                double rii = work[(int64_t)i * n + i];
                beta[i] = (rii != 0.0) ? s / rii : 0.0;
            }
            double rss = 0.0;
            for (int64_t t = 0; t < n; ++t) {
                double fit = 0.0;
                for (int32_t j = 0; j < k; ++j) fit += Xc[t * m + cols[j]] * beta[j];
                e[t] = Xc[t * m + c] - fit;
                rss += e[t] * e[t];
            }
            if (rss <= 0.0) continue; /* exact fit: score is -inf, no finite gradient */
            double coef = wf * (double)n / rss;
            for (int64_t t = 0; t < n; ++t) {
                Gt[t * m + c] += coef * 2.0 * e[t];
                for (int32_t j = 0; j < k; ++j) Gt[t * m + cols[j]] -= coef * 2.0 * beta[j] * e[t];
            }
        }
        free(e);
        free(work);
    }
    for (int64_t i = 0; i < n * m; ++i) {
        double s = 0.0;
        for (int t = 0; t < nt; ++t) s += G[(size_t)t * (size_t)n * (size_t)m + (size_t)i];
        gX[i] = s;
    }
    /* centring adjoint: d/dX of X - 1 mean(X) is (I - 11^T/n) */
    for (int32_t j = 0; j < m; ++j) {
        double s = 0.0;
        for (int64_t t = 0; t < n; ++t) s += gX[t * m + j];
        double mu = s / (double)n;
        for (int64_t t = 0; t < n; ++t) gX[t * m + j] -= mu;
    }
    free(G);
    free(Xc);
    return 0;
}
