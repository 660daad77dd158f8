/*
 * pcv_oracle.c -- plain, slow, FP64 CPU oracle for parallel cross-validation
 * of Gaussian-process models (Gerber & Nychka, arXiv 1912.13132).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark do.  It shares no code, header, table or constant with
 * the CUDA path.
 *
 * Every routine is the textbook definition written out, in the paper's order:
 *   - covariance:  c(s1, s2, theta) = exp(-||s1 - s2|| / theta), Euclidean norm
 *     (Sec. 3, exponential model);
 *   - model matrix: Sigma(theta) + lambda I with lambda = tau / sigma^2, the
 *     nugget only on the diagonal (Eq. 1 and Eq. 3, second line);
 *   - simple kriging predictor: yhat_P = Sigma_p^T (Sigma + lambda I)^{-1} y
 *     (Eq. 3), with a "literal" variant that keeps sigma^2 and tau apart
 *     (Eq. 3, first line) so the sigma^2-invariance can be checked;
 *   - factorisation: unpivoted Cholesky, column by column (Cholesky-Crout),
 *     followed by forward and back substitution;
 *   - loss: SSPE = sum_i (yhat_V[i] - y_V[i])^2 in index order (Eq. 4);
 *   - two times the negative log-likelihood (Eq. 2).
 * No blocking, no reordering, no fusion.  Compiled with -ffp-contract=off so
 * that x86 and Arm hosts give identical results.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_NOT_SPD 6
#define ORACLE_OOM 2

/* Euclidean distance between two points given as (x, y) pairs (Sec. 3). */
static double dist2d(const double* a, const double* b) {
    double dx = a[0] - b[0];
    double dy = a[1] - b[1];
    return sqrt(dx * dx + dy * dy);
}

/* Exponential covariance function c(s1, s2, theta) (Sec. 3). */
static double cov_exp(const double* a, const double* b, double theta) {
    return exp(-dist2d(a, b) / theta);
}

/*
 * Subset selection: indices j (ascending) with role[j] == want and
 *   x0 <= x_j < x1   (x_j <= x1 when x1_incl != 0)
 *   y0 <= y_j < y1   (y_j <= y1 when y1_incl != 0).
 * Returns the count; writes the indices to out when out != NULL.
 */
int64_t oracle_select(const double* xy, const uint8_t* role, int64_t n, int want,
                      double x0, double x1, int x1_incl, double y0, double y1, int y1_incl,
                      int64_t* out) {
    int64_t c = 0;
    for (int64_t j = 0; j < n; ++j) {
        if ((int)role[j] != want) continue;
        double x = xy[2 * j], y = xy[2 * j + 1];
        if (!(x >= x0)) continue;
        if (x1_incl ? !(x <= x1) : !(x < x1)) continue;
        if (!(y >= y0)) continue;
        if (y1_incl ? !(y <= y1) : !(y < y1)) continue;
        if (out) out[c] = j;
        ++c;
    }
    return c;
}

/*
 * Unpivoted Cholesky A = L L^T of a k x k row-major matrix, in place: on return
 * the lower triangle holds L (the strict upper triangle is left untouched).
 * Column j: L_jj = sqrt(A_jj - sum_{p<j} L_jp^2), then
 *           L_ij = (A_ij - sum_{p<j} L_ip L_jp) / L_jj   for i > j.
 * Returns ORACLE_NOT_SPD when a pivot is not positive.
 */
int oracle_cholesky(double* a, int64_t k) {
    for (int64_t j = 0; j < k; ++j) {
        double* rj = a + j * k;
        double s = rj[j];
        for (int64_t p = 0; p < j; ++p) s -= rj[p] * rj[p];
        if (!(s > 0.0)) return ORACLE_NOT_SPD;
        double ljj = sqrt(s);
        rj[j] = ljj;
        for (int64_t i = j + 1; i < k; ++i) {
            double* ri = a + i * k;
            double t = ri[j];
            for (int64_t p = 0; p < j; ++p) t -= ri[p] * rj[p];
            ri[j] = t / ljj;
        }
    }
    return ORACLE_OK;
}

/* Forward substitution L w = b (L lower, row-major k x k), in place on b. */
void oracle_forward(const double* l, int64_t k, double* b) {
    for (int64_t i = 0; i < k; ++i) {
        const double* ri = l + i * k;
        double t = b[i];
        for (int64_t p = 0; p < i; ++p) t -= ri[p] * b[p];
        b[i] = t / ri[i];
    }
}

/* Back substitution L^T x = w, in place on w. */
void oracle_backward(const double* l, int64_t k, double* w) {
    for (int64_t i = k - 1; i >= 0; --i) {
        double t = w[i];
        for (int64_t p = i + 1; p < k; ++p) t -= l[p * k + i] * w[p];
        w[i] = t / l[i * k + i];
    }
}

/*
 * Assemble the k x k model matrix in row-major order (both triangles):
 *   scale * c(s_a, s_b, theta) for a != b,  scale * 1 + nugget on the diagonal.
 * With scale = 1, nugget = lambda this is Sigma + lambda I (Eq. 3, second line);
 * with scale = sigma^2, nugget = tau it is sigma^2 Sigma + tau I (Eq. 1).
 */
static void assemble(const double* sT, int64_t k, double theta, double scale, double nugget,
                     double* a) {
    for (int64_t i = 0; i < k; ++i)
        for (int64_t j = 0; j < k; ++j)
            a[i * k + j] = scale * cov_exp(sT + 2 * i, sT + 2 * j, theta) + (i == j ? nugget : 0.0);
}

static int krige_general(const double* sT, const double* yT, int64_t k, const double* sP,
                         int64_t m, double theta, double scale, double nugget, double* yhat) {
    if (k == 0) {
        for (int64_t j = 0; j < m; ++j) yhat[j] = 0.0;
        return ORACLE_OK;
    }
    double* a = (double*)malloc((size_t)k * (size_t)k * sizeof(double));
    double* alpha = (double*)malloc((size_t)k * sizeof(double));
    if (!a || !alpha) { free(a); free(alpha); return ORACLE_OOM; }
    assemble(sT, k, theta, scale, nugget, a);
    int st = oracle_cholesky(a, k);
    if (st != ORACLE_OK) {
        for (int64_t j = 0; j < m; ++j) yhat[j] = NAN;
        free(a); free(alpha);
        return st;
    }
    memcpy(alpha, yT, (size_t)k * sizeof(double));
    oracle_forward(a, k, alpha);
    oracle_backward(a, k, alpha);          /* alpha = (model matrix)^{-1} y_T */
    for (int64_t j = 0; j < m; ++j) {      /* yhat_j = sum_a cross-cov(p_j, s_a) alpha_a */
        double t = 0.0;
        for (int64_t i = 0; i < k; ++i) t += scale * cov_exp(sP + 2 * j, sT + 2 * i, theta) * alpha[i];
        yhat[j] = t;
    }
    free(a); free(alpha);
    return ORACLE_OK;
}

/* Simple kriging with the noise-to-signal ratio lambda (Eq. 3, second line). */
int oracle_krige(const double* sT, const double* yT, int64_t k, const double* sP, int64_t m,
                 double theta, double lambda, double* yhat) {
    return krige_general(sT, yT, k, sP, m, theta, 1.0, lambda, yhat);
}

/* Simple kriging keeping sigma^2 and tau apart (Eq. 3, first line). */
int oracle_krige_literal(const double* sT, const double* yT, int64_t k, const double* sP,
                         int64_t m, double sigma2, double theta, double tau, double* yhat) {
    return krige_general(sT, yT, k, sP, m, theta, sigma2, tau, yhat);
}

/* Sum of squared prediction errors, index order (Eq. 4). */
double oracle_sspe(const double* yhat, const double* yV, int64_t m) {
    double z = 0.0;
    for (int64_t j = 0; j < m; ++j) {
        double e = yhat[j] - yV[j];
        z += e * e;
    }
    return z;
}

/*
 * Two times the negative log-likelihood of (sigma^2, tau, theta) given y (Eq. 2):
 *   k log(2 pi) + log det(sigma^2 Sigma + tau I) + y^T (sigma^2 Sigma + tau I)^{-1} y,
 * with log det = 2 sum log L_jj and the quadratic form = ||L^{-1} y||^2.
 */
int oracle_neg2loglik(const double* sT, const double* yT, int64_t k, double sigma2,
                      double theta, double tau, double* out) {
    double* a = (double*)malloc((size_t)k * (size_t)k * sizeof(double) + 1);
    double* w = (double*)malloc((size_t)k * sizeof(double) + 1);
    if (!a || !w) { free(a); free(w); return ORACLE_OOM; }
    assemble(sT, k, theta, sigma2, tau, a);
    int st = oracle_cholesky(a, k);
    if (st != ORACLE_OK) { free(a); free(w); *out = NAN; return st; }
    memcpy(w, yT, (size_t)k * sizeof(double));
    oracle_forward(a, k, w);
    double logdet = 0.0, quad = 0.0;
    for (int64_t j = 0; j < k; ++j) logdet += 2.0 * log(a[j * k + j]);
    for (int64_t j = 0; j < k; ++j) quad += w[j] * w[j];
    *out = (double)k * log(2.0 * M_PI) + logdet + quad;
    free(a); free(w);
    return ORACLE_OK;
}
