// kl_bayes.cpp -- the surrogate model behind the tuner's Bayesian-optimisation
// strategy.  The paper tunes with Kernel Tuner's Bayesian optimisation next to
// random search (Sec. 5.3, Fig. 3); here the same idea lives in the library:
// a Gaussian-process regression of log(kernel time) over the encoded
// configurations, and the expected improvement of an unevaluated candidate as
// the acquisition.  Host code only (no CUDA).
//
// Model (standard GP regression, e.g. Rasmussen & Williams 2006, Alg. 2.1):
//  - observations y are standardised to zero mean and unit (population)
//    variance; prior variance 1, noise variance `noise`, both in those units;
//  - covariance Matern 5/2 of the Euclidean distance r between feature rows:
//    k(r) = (1 + a + a^2/3) exp(-a), a = sqrt(5) r / l;
//  - the length scale l, unless given, maximises the log marginal likelihood
//    over kLengthGrid;
//  - posterior mean m(x) = k_x^T (K + noise I)^-1 y, latent variance
//    v(x) = 1 - k_x^T (K + noise I)^-1 k_x, both mapped back to y's units.
// Expected improvement (minimisation) over the best observed value b, with
// margin xi: EI = (b - m - xi) Phi(z) + s phi(z), z = (b - m - xi) / s,
// s = sqrt(v); EI = max(b - m - xi, 0) where s = 0.
// Pending candidates (already chosen, not yet measured) enter as observations
// equal to their posterior mean ("kriging believer"), with the hyperparameters
// of the fit on the real observations, so that one batch spreads out.

#include "kl_internal.h"

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

namespace kl {

namespace {

const double kLengthGrid[] = {0.05, 0.1, 0.2, 0.3, 0.5, 0.75, 1.0, 1.5, 2.0, 3.0};
const double kDefaultNoise = 1e-4;

double matern52(double r, double ls)
{
    double a = std::sqrt(5.0) * r / ls;
    return (1.0 + a + a * a / 3.0) * std::exp(-a);
}

double dist(const double *a, const double *b, int d)
{
    double s = 0;
    for (int q = 0; q < d; ++q) {
        double t = a[q] - b[q];
        s += t * t;
    }
    return std::sqrt(s);
}

struct Gp {
    int n = 0, d = 0;
    std::vector<double> X;       // n x d, row major
    std::vector<double> ys;      // standardised observations
    std::vector<double> L;       // n x n lower Cholesky factor of K + noise I
    std::vector<double> alpha;   // (K + noise I)^-1 ys
    double mean = 0, scale = 1, ls = 1, noise = kDefaultNoise;
};

// in-place Cholesky of the n x n matrix A (lower part); false if not positive definite
bool cholesky(std::vector<double> &A, int n)
{
    for (int j = 0; j < n; ++j) {
        double s = A[(size_t)j * n + j];
        for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
        if (!(s > 0)) return false;
        double ljj = std::sqrt(s);
        A[(size_t)j * n + j] = ljj;
        for (int i = j + 1; i < n; ++i) {
            double t = A[(size_t)i * n + j];
            for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
            A[(size_t)i * n + j] = t / ljj;
        }
        for (int i = 0; i < j; ++i) A[(size_t)i * n + j] = 0;
    }
    return true;
}

// solve L z = b (forward), then L^T x = z (backward) when `both`
void tri_solve(const std::vector<double> &L, int n, std::vector<double> &b, bool both)
{
    for (int i = 0; i < n; ++i) {
        double t = b[i];
        for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * b[k];
        b[i] = t / L[(size_t)i * n + i];
    }
    if (!both) return;
    for (int i = n; i-- > 0;) {
        double t = b[i];
        for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * b[k];
        b[i] = t / L[(size_t)i * n + i];
    }
}

// factor K + noise I for the current X, ys and length scale; false if singular
bool factor(Gp &g)
{
    int n = g.n;
    g.L.assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            double k = matern52(dist(&g.X[(size_t)i * g.d], &g.X[(size_t)j * g.d], g.d), g.ls);
            if (i == j) k += g.noise;
            g.L[(size_t)i * n + j] = k;
            g.L[(size_t)j * n + i] = k;
        }
    if (!cholesky(g.L, n)) return false;
    g.alpha = g.ys;
    tri_solve(g.L, n, g.alpha, true);
    return true;
}

double log_marginal(const Gp &g)
{
    double s = 0;
    for (int i = 0; i < g.n; ++i) s += g.ys[i] * g.alpha[i];
    double ld = 0;
    for (int i = 0; i < g.n; ++i) ld += std::log(g.L[(size_t)i * g.n + i]);
    return -0.5 * s - ld - 0.5 * g.n * std::log(2.0 * M_PI);
}

// fit to n observations; ls <= 0 selects the length scale by marginal likelihood
bool fit(int n, int d, const double *X, const double *y, double ls, double noise, Gp *g)
{
    g->n = n;
    g->d = d;
    g->X.assign(X, X + (size_t)n * d);
    double m = 0;
    for (int i = 0; i < n; ++i) m += y[i];
    m /= n;
    double v = 0;
    for (int i = 0; i < n; ++i) v += (y[i] - m) * (y[i] - m);
    v /= n;
    g->mean = m;
    g->scale = v > 1e-300 ? std::sqrt(v) : 1.0;
    g->ys.resize(n);
    for (int i = 0; i < n; ++i) g->ys[i] = (y[i] - m) / g->scale;
    g->noise = noise > 0 ? noise : kDefaultNoise;
    if (ls > 0) {
        g->ls = ls;
        return factor(*g);
    }
    double best = -INFINITY, best_ls = 0;
    for (double c : kLengthGrid) {
        g->ls = c;
        if (!factor(*g)) continue;
        double lml = log_marginal(*g);
        if (lml > best) {
            best = lml;
            best_ls = c;
        }
    }
    if (best_ls <= 0) return false;
    g->ls = best_ls;
    return factor(*g);
}

// posterior mean and latent variance at x, in y's units
void predict(const Gp &g, const double *x, double *mu, double *var)
{
    std::vector<double> k(g.n);
    for (int i = 0; i < g.n; ++i) k[i] = matern52(dist(&g.X[(size_t)i * g.d], x, g.d), g.ls);
    double m = 0;
    for (int i = 0; i < g.n; ++i) m += k[i] * g.alpha[i];
    tri_solve(g.L, g.n, k, false);
    double q = 0;
    for (int i = 0; i < g.n; ++i) q += k[i] * k[i];
    *mu = g.mean + g.scale * m;
    *var = g.scale * g.scale * std::max(1.0 - q, 0.0);
}

// append one observation (standardised value ys_new) with the current
// hyperparameters: one new row of L, then alpha again (O(n^2))
bool extend(Gp &g, const double *x, double ys_new)
{
    int n = g.n, n1 = n + 1;
    std::vector<double> k(n);
    for (int i = 0; i < n; ++i) k[i] = matern52(dist(&g.X[(size_t)i * g.d], x, g.d), g.ls);
    tri_solve(g.L, n, k, false);
    double s = 1.0 + g.noise;
    for (int i = 0; i < n; ++i) s -= k[i] * k[i];
    if (!(s > 0)) return false;
    std::vector<double> L((size_t)n1 * n1, 0.0);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) L[(size_t)i * n1 + j] = g.L[(size_t)i * n + j];
    for (int j = 0; j < n; ++j) L[(size_t)n * n1 + j] = k[j];
    L[(size_t)n * n1 + n] = std::sqrt(s);
    g.L.swap(L);
    g.X.insert(g.X.end(), x, x + g.d);
    g.ys.push_back(ys_new);
    g.n = n1;
    g.alpha = g.ys;
    tri_solve(g.L, n1, g.alpha, true);
    return true;
}

double expected_improvement(double mu, double var, double best, double xi)
{
    double imp = best - mu - xi;
    double s = std::sqrt(var);
    if (!(s > 1e-300)) return std::max(imp, 0.0);
    double z = imp / s;
    double cdf = 0.5 * std::erfc(-z / std::sqrt(2.0));
    double pdf = std::exp(-0.5 * z * z) / std::sqrt(2.0 * M_PI);
    return imp * cdf + s * pdf;
}

bool all_finite(const double *p, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

}  // namespace

int bo_suggest(int n, int d, const double *X, const double *y, int np, const double *P, int m,
               const double *C, double xi, double ls, double noise, double *ls_used,
               std::vector<double> *ei, std::string *err)
{
    Gp g;
    if (!fit(n, d, X, y, ls, noise, &g)) {
        *err = "surrogate: covariance matrix is not positive definite";
        return -1;
    }
    if (ls_used) *ls_used = g.ls;
    double best = *std::min_element(y, y + n);
    for (int p = 0; p < np; ++p) {
        double mu, var;
        predict(g, P + (size_t)p * d, &mu, &var);
        if (!extend(g, P + (size_t)p * d, (mu - g.mean) / g.scale)) {
            // a pending point on top of an observation adds nothing new
            continue;
        }
    }
    ei->assign(m, 0.0);
    int arg = 0;
    for (int c = 0; c < m; ++c) {
        double mu, var;
        predict(g, C + (size_t)c * d, &mu, &var);
        (*ei)[c] = expected_improvement(mu, var, best, xi);
        if ((*ei)[c] > (*ei)[arg]) arg = c;
    }
    return arg;
}

}  // namespace kl

using namespace kl;

extern "C" {

kl_status kl_bo_posterior(int32_t n, int32_t d, const double *X, const double *y, int32_t m,
                          const double *Xq, double length_scale, double noise, double *mean,
                          double *var, double *ls_used)
{
    if (n < 1 || d < 1 || m < 0) return fail(KL_ERR_INVALID_ARG, "bo: need n >= 1, d >= 1, m >= 0");
    if (!X || !y || (m > 0 && (!Xq || !mean || !var)))
        return fail(KL_ERR_INVALID_ARG, "bo: NULL argument");
    if (!all_finite(X, (size_t)n * d) || !all_finite(y, n) || (m > 0 && !all_finite(Xq, (size_t)m * d)))
        return fail(KL_ERR_INVALID_ARG, "bo: non-finite input");
    Gp g;
    if (!fit(n, d, X, y, length_scale, noise, &g))
        return fail(KL_ERR_INVALID_ARG, "bo: covariance matrix is not positive definite");
    if (ls_used) *ls_used = g.ls;
    for (int q = 0; q < m; ++q) predict(g, Xq + (size_t)q * d, &mean[q], &var[q]);
    return KL_OK;
}

kl_status kl_bo_suggest(int32_t n, int32_t d, const double *X, const double *y, int32_t np,
                        const double *P, int32_t m, const double *C, double xi, double length_scale,
                        double noise, int32_t *choice, double *ei)
{
    if (n < 1 || d < 1 || np < 0 || m < 1)
        return fail(KL_ERR_INVALID_ARG, "bo: need n >= 1, d >= 1, np >= 0, m >= 1");
    if (!X || !y || !C || !choice || (np > 0 && !P)) return fail(KL_ERR_INVALID_ARG, "bo: NULL argument");
    if (!all_finite(X, (size_t)n * d) || !all_finite(y, n) || !all_finite(C, (size_t)m * d) ||
        (np > 0 && !all_finite(P, (size_t)np * d)) || !std::isfinite(xi))
        return fail(KL_ERR_INVALID_ARG, "bo: non-finite input");
    std::vector<double> e;
    std::string err;
    int c = bo_suggest(n, d, X, y, np, P, m, C, xi, length_scale, noise, nullptr, &e, &err);
    if (c < 0) return fail(KL_ERR_INVALID_ARG, "bo: " + err);
    *choice = c;
    if (ei) std::copy(e.begin(), e.end(), ei);
    return KL_OK;
}

}  // extern "C"
