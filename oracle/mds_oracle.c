/*
 * Serial FP64 CPU oracle for the truncated-normal Bayesian MDS likelihood,
 * its gradient and the HMC leapfrog built on it
 * (Holbrook et al., "Massive parallelization boosts big Bayesian
 * multidimensional scaling", arXiv:1905.04582).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference arm use it.  It shares no code, header, table or
 * constant with the CUDA library, and it is written to be checked against the
 * paper by eye: plain loops in the paper's notation, no blocking, no fusion.
 *
 * Notation (paper, section 2.1):
 *   N items, latent locations x_i in R^D (row-major N x D, FP64),
 *   observed dissimilarities y_ij, i != j, symmetric, stored as the strict
 *   upper triangle in row-major order (0,1),(0,2),...,(N-2,N-1) (FP32 values
 *   read exactly as FP64; the library rounds Y to FP32 once at ingest, so both
 *   sides see the same numbers),
 *   delta_ij = ||x_i - x_j||, sigma > 0, z_ij = delta_ij / sigma,
 *   M = N (N - 1) / 2 pairs.
 *
 * The cross-validation functions (training likelihood of a fold, lpd-hat)
 * are pinned in tests/test_oracle_cv_pins.py and the sigma update in
 * tests/test_oracle_sigma_pins.py; planted mistakes in
 * tests/test_oracle_mutations.py.
 *
 * Pinned by (tests/test_oracle_pins.py): the N = 2 closed form at 50 digits,
 * scipy's truncated-normal log density summed over pairs (Eq. 1 model),
 * central finite differences of the oracle's own log-likelihood in X and in
 * sigma, the translation / rotation / permutation invariances, brute force at
 * 50 digits on N <= 8, the large-separation limit, and for the leapfrog the
 * closed-form harmonic-oscillator map, reversibility and the O(eps^2) energy
 * error.  The Philox4x32-10 generator is pinned against cuRAND's host
 * Philox generator where that library loads, else it is "parity unpinned".
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - L includes the sigma^(-M) factor of Eq. (2) and drops (2 pi)^(-M/2).
 *   - Pairs are i < j only; the gradient runs over j != i (Eq. (9)); the
 *     diagonal of Y is never read.
 *   - Coincident points (delta_ij = 0, i != j): r_ij uses delta = 0 and the
 *     pair adds nothing to the gradient (the unit vector is undefined).
 *   - HMC uses M = I, so dx/dt = p (the factor 1/2 printed in Eq. (7) is taken
 *     as a typo: it contradicts H = U + p^T M^{-1} p / 2 of Eq. (6)).
 *   - HMC target log pi(X) = w * L(X, sigma) - (lambda / 2) ||X||_F^2 with
 *     w in {0, 1} and lambda >= 0 (lambda = 0 by default; w = 0 gives the
 *     harmonic oscillator used to pin the integrator).
 *   - Cross-validation (section 2.4): a fold holds out a set of pairs; the
 *     training likelihood is Eq. (2) over the kept pairs only (M = their
 *     count), and the Monte Carlo estimate of the log pointwise predictive
 *     density is, over held-out pairs,
 *       lpd-hat = sum_ij log( (1/S) sum_s p(y_ij | X_s, sigma_s) ),
 *     p the truncated-normal density of Eq. (1).  The printed estimator also
 *     multiplies each term by the posterior density of the draw; with draws
 *     taken from that posterior the plain average is the standard estimate,
 *     which is the one computed here.
 *   - sigma update: the paper takes "Gibbs steps" for sigma^2 with the prior
 *     sigma^-2 ~ Gamma(s0, r0) (shape, rate), but the Phi term of Eq. (2)
 *     makes that full conditional non-standard, so the update here is a
 *     random-walk Metropolis step on log sigma (prior and Jacobian included).
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define MDSO_OK 0
#define MDSO_BAD_ARG 1
#define MDSO_OOM 2

/* ---------------------------------------------------------------------- */
/* Neumaier-compensated summation (improved Kahan-Babuska).                */
/* ---------------------------------------------------------------------- */
typedef struct {
    double s; /* running sum */
    double c; /* running compensation */
} nsum_t;

static void nsum_add(nsum_t *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum_t *a) { return a->s + a->c; }

/* ---------------------------------------------------------------------- */
/* Index of y_ij (i < j) in the packed strict upper triangle.              */
/* Row i starts after rows 0..i-1, which hold (N-1) + (N-2) + ... + (N-i)  */
/* entries = i N - i (i + 1) / 2.                                          */
/* ---------------------------------------------------------------------- */
static int64_t packed_index(int64_t n, int64_t i, int64_t j) {
    return i * n - i * (i + 1) / 2 + (j - i - 1);
}

/* y_ij for any i != j (Y symmetric, section 2.2: "symmetric dissimilarity
 * matrix"); the strict upper triangle is authoritative. */
static double y_at(const float *yp, int64_t n, int64_t i, int64_t j) {
    if (i < j) return (double)yp[packed_index(n, i, j)];
    return (double)yp[packed_index(n, j, i)];
}

/* delta_ij = ||x_i - x_j|| (section 2.1). */
static double distance(const double *x, int d, int64_t i, int64_t j) {
    double s = 0.0;
    for (int k = 0; k < d; ++k) {
        double t = x[i * d + k] - x[j * d + k];
        s += t * t;
    }
    return sqrt(s);
}

/* Standard normal CDF Phi(z) = 1 - erfc(z / sqrt 2) / 2, and its log
 * log Phi(z) = log1p(-erfc(z / sqrt 2) / 2), accurate where Phi -> 1.
 * z = delta / sigma >= 0 here, so Phi is in [1/2, 1). */
static double std_normal_cdf(double z) { return 1.0 - 0.5 * erfc(z / sqrt(2.0)); }
static double log_std_normal_cdf(double z) { return log1p(-0.5 * erfc(z / sqrt(2.0))); }

/* Standard normal density phi(z). */
static double std_normal_pdf(double z) { return exp(-0.5 * z * z) / sqrt(2.0 * M_PI); }

/* r_ij of Eq. (2): (y - delta)^2 / (2 sigma^2) + log Phi(delta / sigma). */
static double r_term(double y, double delta, double sigma) {
    double e = y - delta;
    return e * e / (2.0 * sigma * sigma) + log_std_normal_cdf(delta / sigma);
}

/* Scalar factor of the gradient contribution in Eq. (9):
 * (delta - y) / sigma^2 + phi(delta / sigma) / (sigma Phi(delta / sigma)). */
static double grad_factor(double y, double delta, double sigma) {
    double z = delta / sigma;
    return (delta - y) / (sigma * sigma) + std_normal_pdf(z) / (sigma * std_normal_cdf(z));
}

/* -d r_ij / d sigma, obtained by differentiating Eq. (2) in sigma:
 * (y - delta)^2 / sigma^3 + phi(z) delta / (sigma^2 Phi(z)). */
static double neg_dr_dsigma(double y, double delta, double sigma) {
    double z = delta / sigma;
    double e = y - delta;
    return e * e / (sigma * sigma * sigma) +
           std_normal_pdf(z) * delta / (sigma * sigma * std_normal_cdf(z));
}

/* keep[] (one byte per packed pair, NULL = all pairs): does pair (i, j)
 * belong to the training data? */
static int pair_kept(const unsigned char *keep, int64_t n, int64_t i, int64_t j) {
    if (!keep) return 1;
    return i < j ? keep[packed_index(n, i, j)] != 0 : keep[packed_index(n, j, i)] != 0;
}

/* Number of training pairs. */
static double kept_pairs(const unsigned char *keep, int64_t n) {
    if (!keep) return 0.5 * (double)n * (double)(n - 1);
    double m = 0.0;
    for (int64_t k = 0; k < n * (n - 1) / 2; ++k) m += keep[k] != 0;
    return m;
}

/* Sum over kept pairs i < j of r_ij, with the pairs of row i summed first
 * (per-row Neumaier sums), rows then summed in order.  Rows are independent,
 * so `nthreads` > 1 splits them over OpenMP threads; the result does not
 * depend on the thread count. */
static int sum_r_rows(int64_t n, int d, const float *yp, const unsigned char *keep, const double *x,
                      double sigma, int nthreads, double *out) {
    double *row = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    if (!row) return MDSO_OOM;
    int64_t i;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (i = 0; i < n; ++i) {
        nsum_t s = {0.0, 0.0};
        for (int64_t j = i + 1; j < n; ++j)
            if (pair_kept(keep, n, i, j))
                nsum_add(&s, r_term((double)yp[packed_index(n, i, j)], distance(x, d, i, j), sigma));
        row[i] = nsum_get(&s);
    }
    (void)nthreads;
    nsum_t tot = {0.0, 0.0};
    for (i = 0; i < n; ++i) nsum_add(&tot, row[i]);
    free(row);
    *out = nsum_get(&tot);
    return MDSO_OK;
}

/* Log-likelihood, Eq. (2) and the last line of Algorithm 1:
 *   log p(Y | X, sigma) = -M log sigma - sum_{i<j} r_ij
 * ((sigma^2)^(N(1-N)/4) = sigma^(-M)).  Also returns sum_{i<j} r_ij. */
int mdso_loglik_kept(int64_t n, int d, const float *yp, const unsigned char *keep, const double *x,
                     double sigma, int nthreads, double *sum_r, double *loglik) {
    if (n < 2 || d < 1 || !(sigma > 0.0) || !yp || !x) return MDSO_BAD_ARG;
    double sr = 0.0;
    int st = sum_r_rows(n, d, yp, keep, x, sigma, nthreads, &sr);
    if (st) return st;
    double m = kept_pairs(keep, n);
    if (sum_r) *sum_r = sr;
    if (loglik) *loglik = -m * log(sigma) - sr;
    return MDSO_OK;
}

int mdso_loglik(int64_t n, int d, const float *yp, const double *x, double sigma,
                int nthreads, double *sum_r, double *loglik) {
    return mdso_loglik_kept(n, d, yp, NULL, x, sigma, nthreads, sum_r, loglik);
}

/* Gradient of the log-likelihood with respect to x_i, Eq. (9):
 *   d/dx_i log p = - sum_{j != i} grad_factor(y_ij, delta_ij) (x_i - x_j) / delta_ij
 * for the rows listed in `rows` (all rows when rows == NULL, nrows ignored).
 * grad is nrows x D (or N x D).  absterm (optional, same shape) receives
 * S_ik = sum_{j != i} |term_ijk| and sqterm (optional) sqrt(sum_{j != i}
 * term_ijk^2): the scales used to judge cancellation and rounding when a
 * lower-precision result is compared with this one. */
int mdso_gradient_rows_kept(int64_t n, int d, const float *yp, const unsigned char *keep,
                            const double *x, double sigma, const int64_t *rows, int64_t nrows,
                            int nthreads, double *grad, double *absterm, double *sqterm) {
    if (n < 2 || d < 1 || d > 16 || !(sigma > 0.0) || !yp || !x || !grad) return MDSO_BAD_ARG;
    int64_t count = rows ? nrows : n;
    int64_t r;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (r = 0; r < count; ++r) {
        int64_t i = rows ? rows[r] : r;
        nsum_t g[16];
        nsum_t a[16];
        nsum_t q[16];
        for (int k = 0; k < d; ++k) {
            g[k].s = g[k].c = 0.0;
            a[k].s = a[k].c = 0.0;
            q[k].s = q[k].c = 0.0;
        }
        if (i >= 0 && i < n) {
            for (int64_t j = 0; j < n; ++j) {
                if (j == i || !pair_kept(keep, n, i, j)) continue;
                double delta = distance(x, d, i, j);
                if (delta == 0.0) continue; /* coincident points add nothing */
                double w = grad_factor(y_at(yp, n, i, j), delta, sigma);
                for (int k = 0; k < d; ++k) {
                    double term = w * (x[i * d + k] - x[j * d + k]) / delta;
                    nsum_add(&g[k], -term);
                    nsum_add(&a[k], fabs(term));
                    nsum_add(&q[k], term * term);
                }
            }
        }
        for (int k = 0; k < d; ++k) {
            grad[r * d + k] = nsum_get(&g[k]);
            if (absterm) absterm[r * d + k] = nsum_get(&a[k]);
            if (sqterm) sqterm[r * d + k] = sqrt(nsum_get(&q[k]));
        }
    }
    (void)nthreads;
    return MDSO_OK;
}

int mdso_gradient_rows(int64_t n, int d, const float *yp, const double *x, double sigma,
                       const int64_t *rows, int64_t nrows, int nthreads,
                       double *grad, double *absterm, double *sqterm) {
    return mdso_gradient_rows_kept(n, d, yp, NULL, x, sigma, rows, nrows, nthreads, grad, absterm, sqterm);
}

/* Derivative of the log-likelihood in sigma (not printed in the paper;
 * obtained by differentiating Eq. (2), including its sigma^(-M) factor):
 *   d/dsigma log p = -M / sigma + sum_{i<j} neg_dr_dsigma(y_ij, delta_ij),
 * over the kept pairs. */
int mdso_dsigma_kept(int64_t n, int d, const float *yp, const unsigned char *keep, const double *x,
                     double sigma, int nthreads, double *dsigma) {
    if (n < 2 || d < 1 || !(sigma > 0.0) || !yp || !x || !dsigma) return MDSO_BAD_ARG;
    double *row = (double *)malloc(sizeof(double) * (size_t)n);
    if (!row) return MDSO_OOM;
    int64_t i;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads > 0 ? nthreads : 1)
#endif
    for (i = 0; i < n; ++i) {
        nsum_t s = {0.0, 0.0};
        for (int64_t j = i + 1; j < n; ++j)
            if (pair_kept(keep, n, i, j))
                nsum_add(&s, neg_dr_dsigma((double)yp[packed_index(n, i, j)], distance(x, d, i, j), sigma));
        row[i] = nsum_get(&s);
    }
    (void)nthreads;
    nsum_t tot = {0.0, 0.0};
    for (i = 0; i < n; ++i) nsum_add(&tot, row[i]);
    free(row);
    double m = kept_pairs(keep, n);
    *dsigma = -m / sigma + nsum_get(&tot);
    return MDSO_OK;
}

int mdso_dsigma(int64_t n, int d, const float *yp, const double *x, double sigma,
                int nthreads, double *dsigma) {
    return mdso_dsigma_kept(n, d, yp, NULL, x, sigma, nthreads, dsigma);
}

/* ---------------------------------------------------------------------- */
/* HMC target and leapfrog (section 2.3, "Hamiltonian Monte Carlo").        */
/* ---------------------------------------------------------------------- */

/* log pi(X) = w L(X, sigma) - lambda/2 ||X||^2 and its gradient (N x D). */
static int target(int64_t n, int d, const float *yp, const unsigned char *keep, const double *x,
                  double sigma, double w, double lambda, int nthreads, double *logpi, double *grad) {
    int64_t nd = n * d;
    double ll = 0.0;
    if (w != 0.0) {
        int st = mdso_loglik_kept(n, d, yp, keep, x, sigma, nthreads, NULL, &ll);
        if (st) return st;
        if (grad) {
            st = mdso_gradient_rows_kept(n, d, yp, keep, x, sigma, NULL, 0, nthreads, grad, NULL, NULL);
            if (st) return st;
            for (int64_t k = 0; k < nd; ++k) grad[k] *= w;
        }
    } else if (grad) {
        for (int64_t k = 0; k < nd; ++k) grad[k] = 0.0;
    }
    nsum_t sq = {0.0, 0.0};
    for (int64_t k = 0; k < nd; ++k) {
        nsum_add(&sq, x[k] * x[k]);
        if (grad) grad[k] -= lambda * x[k];
    }
    if (logpi) *logpi = w * ll - 0.5 * lambda * nsum_get(&sq);
    return MDSO_OK;
}

/* Kinetic energy p^T M^{-1} p / 2 with M = I (Eq. (6)). */
static double kinetic(int64_t nd, const double *p) {
    nsum_t s = {0.0, 0.0};
    for (int64_t k = 0; k < nd; ++k) nsum_add(&s, 0.5 * p[k] * p[k]);
    return nsum_get(&s);
}

/* Leapfrog integration of dx/dt = p, dp/dt = grad log pi(x) (Eq. (7) with
 * M = I), n_steps steps of size eps, each
 *   p <- p + eps/2 grad log pi(x);  x <- x + eps p;  p <- p + eps/2 grad log pi(x).
 * x and p (N x D) are advanced in place.  H0 / H1 receive the energy
 * H = -log pi(x) + p^T p / 2 (Eq. (6)) before and after. */
int mdso_leapfrog_kept(int64_t n, int d, const float *yp, const unsigned char *keep, double *x,
                       double *p, double sigma, double w, double lambda, double eps, int n_steps,
                       int nthreads, double *h0, double *h1) {
    if (n < 2 || d < 1 || n_steps < 0 || !x || !p || (w != 0.0 && (!yp || !(sigma > 0.0))))
        return MDSO_BAD_ARG;
    int64_t nd = n * d;
    double *g = (double *)malloc(sizeof(double) * (size_t)nd);
    if (!g) return MDSO_OOM;
    double lp = 0.0;
    int st = target(n, d, yp, keep, x, sigma, w, lambda, nthreads, &lp, g);
    if (st) { free(g); return st; }
    if (h0) *h0 = -lp + kinetic(nd, p);
    for (int s = 0; s < n_steps; ++s) {
        for (int64_t k = 0; k < nd; ++k) p[k] += 0.5 * eps * g[k];
        for (int64_t k = 0; k < nd; ++k) x[k] += eps * p[k];
        st = target(n, d, yp, keep, x, sigma, w, lambda, nthreads, &lp, g);
        if (st) { free(g); return st; }
        for (int64_t k = 0; k < nd; ++k) p[k] += 0.5 * eps * g[k];
    }
    if (h1) *h1 = -lp + kinetic(nd, p);
    free(g);
    return MDSO_OK;
}

int mdso_leapfrog(int64_t n, int d, const float *yp, double *x, double *p, double sigma,
                  double w, double lambda, double eps, int n_steps, int nthreads,
                  double *h0, double *h1) {
    return mdso_leapfrog_kept(n, d, yp, NULL, x, p, sigma, w, lambda, eps, n_steps, nthreads, h0, h1);
}

/* Truncated-normal density of one observation (Eq. (1): y ~ N(delta,
 * sigma^2) restricted to y > 0), on the log scale:
 *   log p(y | delta, sigma) = -log(sqrt(2 pi) sigma) - (y - delta)^2 / (2 sigma^2)
 *                             - log Phi(delta / sigma). */
static double log_density(double y, double delta, double sigma) {
    double e = y - delta;
    return -log(sqrt(2.0 * M_PI) * sigma) - e * e / (2.0 * sigma * sigma) - log_std_normal_cdf(delta / sigma);
}

/* Log pointwise predictive density estimate of section 2.4 over the held-out
 * pairs (pairs[2 k], pairs[2 k + 1]), k < npairs, from S posterior draws
 * (locations xs[s] (N x D) and sigmas[s]):
 *   lpd-hat = sum_k log( (1/S) sum_s p(y_k | X_s, sigma_s) ),
 * each log-mean evaluated as m + log(sum_s exp(l_s - m)) - log S with
 * m = max_s l_s (the same number, without underflow of exp(l_s)). */
int mdso_lpd(int64_t n, int d, const float *yp, int64_t npairs, const int64_t *pairs, int S,
             const double *xs, const double *sigmas, double *lpd) {
    if (n < 2 || d < 1 || npairs < 0 || S < 1 || !yp || !xs || !sigmas || !lpd || (npairs > 0 && !pairs))
        return MDSO_BAD_ARG;
    double *l = (double *)malloc(sizeof(double) * (size_t)S);
    if (!l) return MDSO_OOM;
    nsum_t tot = {0.0, 0.0};
    for (int64_t k = 0; k < npairs; ++k) {
        int64_t i = pairs[2 * k], j = pairs[2 * k + 1];
        if (i < 0 || j < 0 || i >= n || j >= n || i == j) { free(l); return MDSO_BAD_ARG; }
        double m = -INFINITY;
        for (int s = 0; s < S; ++s) {
            if (!(sigmas[s] > 0.0)) { free(l); return MDSO_BAD_ARG; }
            l[s] = log_density(y_at(yp, n, i, j), distance(xs + (int64_t)s * n * d, d, i, j), sigmas[s]);
            if (l[s] > m) m = l[s];
        }
        double e = 0.0;
        for (int s = 0; s < S; ++s) e += exp(l[s] - m);
        nsum_add(&tot, m + log(e) - log((double)S));
    }
    free(l);
    *lpd = nsum_get(&tot);
    return MDSO_OK;
}

/* HMC (section 2.3): n_iter iterations, each drawing momentum p (supplied
 * by the caller in p_all, n_iter x N x D, standard normal), running
 * n_steps leapfrog steps, and accepting the proposal when
 * log u < H(x0, p0) - H(x*, p*), i.e. with probability
 * min(1, exp(-H(x*,p*)) / exp(-H(x0,p0))) (Eq. (8)); u_all[t] in (0,1).
 * x (N x D) is updated in place.  accepted[t] (0/1) and dh[t] = H1 - H0 are
 * returned per iteration. */
int mdso_hmc_kept(int64_t n, int d, const float *yp, const unsigned char *keep, double *x, double sigma,
                  double w, double lambda, double eps, int n_steps, int n_iter, const double *p_all,
                  const double *u_all, int nthreads, int *accepted, double *dh) {
    if (n < 2 || d < 1 || n_iter < 0 || !x || !p_all || !u_all) return MDSO_BAD_ARG;
    int64_t nd = n * d;
    double *x1 = (double *)malloc(sizeof(double) * (size_t)nd);
    double *p = (double *)malloc(sizeof(double) * (size_t)nd);
    if (!x1 || !p) { free(x1); free(p); return MDSO_OOM; }
    for (int t = 0; t < n_iter; ++t) {
        memcpy(x1, x, sizeof(double) * (size_t)nd);
        memcpy(p, p_all + (int64_t)t * nd, sizeof(double) * (size_t)nd);
        double h0 = 0.0, h1 = 0.0;
        int st = mdso_leapfrog_kept(n, d, yp, keep, x1, p, sigma, w, lambda, eps, n_steps, nthreads, &h0, &h1);
        if (st) { free(x1); free(p); return st; }
        int acc = log(u_all[t]) < h0 - h1;
        if (accepted) accepted[t] = acc;
        if (dh) dh[t] = h1 - h0;
        if (acc) memcpy(x, x1, sizeof(double) * (size_t)nd);
    }
    free(x1);
    free(p);
    return MDSO_OK;
}

int mdso_hmc(int64_t n, int d, const float *yp, double *x, double sigma, double w,
             double lambda, double eps, int n_steps, int n_iter, const double *p_all,
             const double *u_all, int nthreads, int *accepted, double *dh) {
    return mdso_hmc_kept(n, d, yp, NULL, x, sigma, w, lambda, eps, n_steps, n_iter, p_all, u_all, nthreads,
                         accepted, dh);
}

/* ---------------------------------------------------------------------- */
/* Philox4x32-10 counter-based generator (Salmon, Moraes, Dror and Shaw,   */
/* "Parallel random numbers: as easy as 1, 2, 3", SC'11), used to draw the  */
/* HMC momenta and uniforms when they are not supplied by the caller.       */
/* ---------------------------------------------------------------------- */
static void philox_round(uint32_t c[4], const uint32_t k[2]) {
    uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c[1] ^ k[0];
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c[3] ^ k[1];
    uint32_t n3 = lo0;
    c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
}

/* out = Philox4x32-10(counter, key). */
void mdso_philox4x32_10(const uint32_t counter[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t c[4] = {counter[0], counter[1], counter[2], counter[3]};
    uint32_t k[2] = {key[0], key[1]};
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k[0] += 0x9E3779B9u;
            k[1] += 0xBB67AE85u;
        }
        philox_round(c, k);
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* Uniform in (0, 1) from 32 random bits: (b + 1/2) / 2^32. */
static double bits_to_open_unit(uint32_t b) { return ((double)b + 0.5) * (1.0 / 4294967296.0); }

/* Momentum and uniform draws of HMC iteration `iter` for a chain whose
 * stream key is (seed_lo, seed_hi):
 *   element e of p (0 <= e < count) uses counter (e / 4, iter, chain, 0);
 *   words (0,1) give normals 4q, 4q+1 and words (2,3) give 4q+2, 4q+3 by the
 *   Box-Muller transform z0 = sqrt(-2 ln u1) cos(2 pi u2),
 *   z1 = sqrt(-2 ln u1) sin(2 pi u2);
 *   the Metropolis uniform uses counter (0, iter, chain, 1), word 0. */
void mdso_draw_momentum(uint32_t seed_lo, uint32_t seed_hi, uint32_t chain, uint32_t iter,
                        int64_t count, double *p, double *u) {
    uint32_t key[2] = {seed_lo, seed_hi};
    for (int64_t q = 0; 4 * q < count; ++q) {
        uint32_t ctr[4] = {(uint32_t)q, iter, chain, 0u};
        uint32_t o[4];
        mdso_philox4x32_10(ctr, key, o);
        for (int h = 0; h < 2; ++h) {
            double u1 = bits_to_open_unit(o[2 * h]);
            double u2 = bits_to_open_unit(o[2 * h + 1]);
            double rad = sqrt(-2.0 * log(u1));
            double th = 2.0 * M_PI * u2;
            int64_t e0 = 4 * q + 2 * h;
            if (e0 < count) p[e0] = rad * cos(th);
            if (e0 + 1 < count) p[e0 + 1] = rad * sin(th);
        }
    }
    if (u) {
        uint32_t ctr[4] = {0u, iter, chain, 1u};
        uint32_t o[4];
        mdso_philox4x32_10(ctr, key, o);
        *u = bits_to_open_unit(o[0]);
    }
}

/* ---------------------------------------------------------------------- */
/* Update of sigma given X (the sigma^2 step of the paper's Gibbs scheme,  */
/* section 3; prior sigma^-2 ~ Gamma(s0, r0), section 2.2).  The Phi term   */
/* of Eq. (2) makes the full conditional non-standard, so the update is a   */
/* random-walk Metropolis step on tau = log sigma.                          */
/* ---------------------------------------------------------------------- */

/* Draws of sigma update `iter`: counter (0, iter, chain, 2); words (0, 1)
 * give z = sqrt(-2 ln u1) cos(2 pi u2), word 2 gives the uniform. */
void mdso_sigma_draws(uint32_t seed_lo, uint32_t seed_hi, uint32_t chain, uint32_t iter, double *z, double *u) {
    uint32_t key[2] = {seed_lo, seed_hi};
    uint32_t ctr[4] = {0u, iter, chain, 2u};
    uint32_t o[4];
    mdso_philox4x32_10(ctr, key, o);
    double u1 = bits_to_open_unit(o[0]);
    double u2 = bits_to_open_unit(o[1]);
    *z = sqrt(-2.0 * log(u1)) * cos(2.0 * M_PI * u2);
    *u = bits_to_open_unit(o[2]);
}

/* log density of tau = log sigma under the prior sigma^-2 ~ Gamma(s0, r0)
 * (shape s0, rate r0): with lambda = sigma^-2 = exp(-2 tau) and
 * |d lambda / d tau| = 2 lambda,
 *   log p(tau) = (s0 - 1) log lambda - r0 lambda + log(2 lambda) + const
 *              = s0 log lambda - r0 lambda + const. */
static double log_prior_tau(double sigma, double s0, double r0) {
    double lambda = 1.0 / (sigma * sigma);
    return s0 * log(lambda) - r0 * lambda;
}

/* n_iter updates of *sigma: tau' = tau + step z_t, accepted iff
 *   log u_t < [w L(X, sigma') + log p(tau')] - [w L(X, sigma) + log p(tau)]
 * (L over the kept pairs; w in {0, 1}, w = 0 samples the prior).  z_all and
 * u_all hold the draws; accepted[t] (optional) receives the decisions. */
int mdso_sigma_mh(int64_t n, int d, const float *yp, const unsigned char *keep, const double *x, double *sigma,
                  double w, int n_iter, double step, double s0, double r0, const double *z_all,
                  const double *u_all, int nthreads, int *accepted) {
    if (n < 2 || d < 1 || n_iter < 0 || !x || !sigma || !(*sigma > 0.0) || !z_all || !u_all ||
        !(s0 > 0.0) || !(r0 > 0.0) || (w != 0.0 && !yp))
        return MDSO_BAD_ARG;
    double s = *sigma, ll = 0.0;
    if (w != 0.0) {
        int st = mdso_loglik_kept(n, d, yp, keep, x, s, nthreads, NULL, &ll);
        if (st) return st;
    }
    double cur = w * ll + log_prior_tau(s, s0, r0);
    for (int t = 0; t < n_iter; ++t) {
        double s1 = exp(log(s) + step * z_all[t]);
        double ll1 = 0.0;
        if (w != 0.0) {
            int st = mdso_loglik_kept(n, d, yp, keep, x, s1, nthreads, NULL, &ll1);
            if (st) return st;
        }
        double prop = w * ll1 + log_prior_tau(s1, s0, r0);
        int acc = log(u_all[t]) < prop - cur;
        if (acc) {
            s = s1;
            cur = prop;
        }
        if (accepted) accepted[t] = acc;
    }
    *sigma = s;
    return MDSO_OK;
}

/* ---------------------------------------------------------------------- */
/* Single-item random-walk Metropolis: the prior-art sampler of section    */
/* 2.3 (a low-dimensional random-walk kernel applied to one x_i at a time). */
/* Moving x_i changes only the N - 1 terms r_ij, j != i, so a proposal     */
/* costs O(N D) instead of a full O(N^2 D) evaluation.                      */
/* ---------------------------------------------------------------------- */

/* sum_{j != i} r_ij with x_i taken as xi (a D-vector), the other rows of X
 * as they are. */
static double row_r(int64_t n, int d, const float *yp, const double *x, int64_t i, const double *xi,
                    double sigma) {
    nsum_t s = {0.0, 0.0};
    for (int64_t j = 0; j < n; ++j) {
        if (j == i) continue;
        double dd = 0.0;
        for (int k = 0; k < d; ++k) {
            double t = xi[k] - x[j * d + k];
            dd += t * t;
        }
        nsum_add(&s, r_term(y_at(yp, n, i, j), sqrt(dd), sigma));
    }
    return nsum_get(&s);
}

/* n_prop proposals; proposal t moves item items[t] to x_i + step z_t
 * (z_all: n_prop x D) and is accepted iff log u_t < log pi(X') - log pi(X),
 * log pi = w L(X, sigma) - (lambda/2) ||X||^2, where
 *   L(X') - L(X) = sum_{j != i} r_ij(x_i) - sum_{j != i} r_ij(x_i')
 * (the -M log sigma of Eq. (2) cancels).  x is updated in place;
 * accepted[t] and dlogpi[t] (optional) receive the decision and the
 * log-target difference. */
int mdso_rwmh(int64_t n, int d, const float *yp, double *x, double sigma, double w, double lambda, double step,
              int n_prop, const int64_t *items, const double *z_all, const double *u_all, int *accepted,
              double *dlogpi) {
    if (n < 2 || d < 1 || d > 16 || n_prop < 0 || !x || !items || !z_all || !u_all || !(sigma > 0.0) ||
        (w != 0.0 && !yp))
        return MDSO_BAD_ARG;
    for (int t = 0; t < n_prop; ++t) {
        int64_t i = items[t];
        if (i < 0 || i >= n) return MDSO_BAD_ARG;
        double xi[16];
        double sq0 = 0.0, sq1 = 0.0;
        for (int k = 0; k < d; ++k) {
            xi[k] = x[i * d + k] + step * z_all[(int64_t)t * d + k];
            sq0 += x[i * d + k] * x[i * d + k];
            sq1 += xi[k] * xi[k];
        }
        double dl = 0.0;
        if (w != 0.0) dl = w * (row_r(n, d, yp, x, i, x + i * d, sigma) - row_r(n, d, yp, x, i, xi, sigma));
        double a = dl - 0.5 * lambda * (sq1 - sq0);
        int acc = log(u_all[t]) < a;
        if (acc)
            for (int k = 0; k < d; ++k) x[i * d + k] = xi[k];
        if (accepted) accepted[t] = acc;
        if (dlogpi) dlogpi[t] = a;
    }
    return MDSO_OK;
}

/* Draws of random-walk proposal `iter` of a chain keyed (seed_lo, seed_hi):
 * counter (iter, 0, chain, 3): item = floor(word0 * N / 2^32), u from
 * word 1; counters (iter, 1 + q, chain, 3) give z components 4q..4q+3 by
 * Box-Muller from words (0, 1) and (2, 3), as the momenta. */
void mdso_rwmh_draws(uint32_t seed_lo, uint32_t seed_hi, uint32_t chain, uint32_t iter, int64_t n, int d,
                     int64_t *item, double *z, double *u) {
    uint32_t key[2] = {seed_lo, seed_hi};
    uint32_t ctr[4] = {iter, 0u, chain, 3u};
    uint32_t o[4];
    mdso_philox4x32_10(ctr, key, o);
    *item = (int64_t)(((uint64_t)o[0] * (uint64_t)n) >> 32);
    *u = bits_to_open_unit(o[1]);
    for (int q = 0; 4 * q < d; ++q) {
        uint32_t c2[4] = {iter, 1u + (uint32_t)q, chain, 3u};
        mdso_philox4x32_10(c2, key, o);
        for (int h = 0; h < 2; ++h) {
            double u1 = bits_to_open_unit(o[2 * h]);
            double u2 = bits_to_open_unit(o[2 * h + 1]);
            double rad = sqrt(-2.0 * log(u1));
            double th = 2.0 * M_PI * u2;
            int e0 = 4 * q + 2 * h;
            if (e0 < d) z[e0] = rad * cos(th);
            if (e0 + 1 < d) z[e0 + 1] = rad * sin(th);
        }
    }
}
