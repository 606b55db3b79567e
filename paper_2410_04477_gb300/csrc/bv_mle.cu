// bv_mle.cu -- maximum-likelihood driver over the block-Vecchia log-likelihood.
//
// The paper estimates theta with the derivative-free BOBYQA optimiser (Sec. 3.2); this
// library uses the derivative-free Nelder-Mead simplex method (Nelder and Mead 1965) with
// the standard coefficients (reflection 1, expansion 2, contraction 1/2, shrink 1/2).
// Coordinates: log(sigma^2 / beta^(2 nu)), log beta, log tau^2 (the free ones).  For the
// Matern model sigma^2 and beta are poorly identified separately but their combination
// sigma^2 / beta^(2 nu) is well identified, so the likelihood surface has a long ridge in
// (log sigma^2, log beta) that this change of variables straightens.  Points outside the
// box [lo, hi] score -inf.  After convergence the simplex is rebuilt once around the best
// point and the search resumed (a standard guard against premature collapse).  Every
// objective value is one device evaluation of ell (bv_loglik); a non-positive-definite
// point also scores -inf and is rejected.  With BV_MIXED the search runs in mixed
// precision and is finished by a short FP64 search from its optimum, so the returned
// estimate and ell are FP64.
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "bv_internal.h"

namespace {

struct Space {
    bv_theta base;
    uint32_t mask;
    int dim;
    double lo[3], hi[3];  // log-box of sigma^2, range, nugget (in that order, all three)
    double two_nu;
};

// Internal coordinates x -> theta.  x holds, for the free parameters in order:
// u = log sigma^2 - 2 nu log beta (if sigma^2 free), log beta (if range free), log tau^2.
bool to_theta(const Space& S, const double* x, bv_theta* t) {
    *t = S.base;
    int k = 0;
    double lsig = log(S.base.sigma2), lbeta = log(S.base.range[0]), ltau = log(S.base.nugget > 0 ? S.base.nugget : 1e-300);
    double u = 0.0;
    const bool fs = S.mask & BV_FREE_SIGMA2, fr = S.mask & BV_FREE_RANGE, fn = S.mask & BV_FREE_NUGGET;
    if (fs) u = x[k++];
    if (fr) lbeta = x[k++];
    if (fn) ltau = x[k++];
    if (fs) lsig = u + S.two_nu * lbeta;
    if (lsig < S.lo[0] || lsig > S.hi[0] || lbeta < S.lo[1] || lbeta > S.hi[1] || ltau < S.lo[2] || ltau > S.hi[2])
        return false;
    t->sigma2 = exp(lsig);
    const double f = exp(lbeta) / S.base.range[0];
    for (int j = 0; j < 3; ++j) t->range[j] = S.base.range[j] * f;
    if (fn) t->nugget = exp(ltau);
    return true;
}

void from_theta(const Space& S, const bv_theta& t, double* x) {
    int k = 0;
    const double lb = log(t.range[0]);
    if (S.mask & BV_FREE_SIGMA2) x[k++] = log(t.sigma2) - S.two_nu * lb;
    if (S.mask & BV_FREE_RANGE) x[k++] = lb;
    if (S.mask & BV_FREE_NUGGET) x[k++] = log(t.nugget);
}

// One Nelder-Mead search from x0 with initial step `step`; returns the best point and
// value (of f = -ell) and adds the evaluations used to *evals.
int nelder_mead(bv_ctx* c, const Space& S, int prec, std::vector<double> x0, double step, double ftol, double xtol,
                int max_evals, int* evals, std::vector<double>* xbest, double* fbest) {
    const int n = S.dim;
    int hard_error = BV_OK;
    auto f = [&](const std::vector<double>& x) -> double {
        bv_theta t;
        if (!to_theta(S, x.data(), &t)) return INFINITY;
        double ll = -INFINITY;
        ++*evals;
        const int st = bv_loglik(c, &t, prec, &ll, nullptr);
        if (st != BV_OK && st != BV_ENOTPD) hard_error = st;
        return (st == BV_OK && std::isfinite(ll)) ? -ll : INFINITY;
    };
    std::vector<std::vector<double>> X(n + 1, x0);
    for (int j = 0; j < n; ++j) X[j + 1][j] += step;
    std::vector<double> F(n + 1);
    for (int j = 0; j <= n; ++j) {
        F[j] = f(X[j]);
        if (hard_error) return hard_error;
    }
    std::vector<int> idx(n + 1);
    std::vector<double> xc(n), xr(n), xe(n), xk(n);
    while (*evals < max_evals) {
        std::iota(idx.begin(), idx.end(), 0);
        std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return F[a] < F[b]; });
        {
            std::vector<std::vector<double>> X2(n + 1);
            std::vector<double> F2(n + 1);
            for (int j = 0; j <= n; ++j) {
                X2[j] = X[idx[j]];
                F2[j] = F[idx[j]];
            }
            X.swap(X2);
            F.swap(F2);
        }
        double xs = 0.0;
        for (int j = 1; j <= n; ++j)
            for (int q = 0; q < n; ++q) xs = std::max(xs, fabs(X[j][q] - X[0][q]));
        if (std::isfinite(F[n]) && F[n] - F[0] <= ftol * fabs(F[0]) && xs <= xtol) break;
        for (int q = 0; q < n; ++q) {
            xc[q] = 0.0;
            for (int j = 0; j < n; ++j) xc[q] += X[j][q];
            xc[q] /= n;
        }
        for (int q = 0; q < n; ++q) xr[q] = xc[q] + (xc[q] - X[n][q]);
        const double fr = f(xr);
        if (hard_error) return hard_error;
        if (fr < F[0]) {
            for (int q = 0; q < n; ++q) xe[q] = xc[q] + 2.0 * (xc[q] - X[n][q]);
            const double fe = f(xe);
            if (hard_error) return hard_error;
            if (fe < fr) {
                X[n] = xe;
                F[n] = fe;
            } else {
                X[n] = xr;
                F[n] = fr;
            }
        } else if (fr < F[n - 1]) {
            X[n] = xr;
            F[n] = fr;
        } else {
            const bool outside = fr < F[n];
            for (int q = 0; q < n; ++q)
                xk[q] = outside ? xc[q] + 0.5 * (xr[q] - xc[q]) : xc[q] + 0.5 * (X[n][q] - xc[q]);
            const double fk = f(xk);
            if (hard_error) return hard_error;
            if (fk < (outside ? fr : F[n])) {
                X[n] = xk;
                F[n] = fk;
            } else {
                for (int j = 1; j <= n; ++j) {
                    for (int q = 0; q < n; ++q) X[j][q] = X[0][q] + 0.5 * (X[j][q] - X[0][q]);
                    F[j] = f(X[j]);
                    if (hard_error) return hard_error;
                }
            }
        }
    }
    int best = 0;
    for (int j = 1; j <= n; ++j)
        if (F[j] < F[best]) best = j;
    *xbest = X[best];
    *fbest = F[best];
    return BV_OK;
}

}  // namespace

extern "C" int bv_mle(bv_ctx* c, const bv_theta* theta0, const bv_theta* lo, const bv_theta* hi,
                      uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat, double* loglik_hat,
                      int32_t* n_evals) {
    if (!c || !theta0 || !lo || !hi || !opts || !theta_hat) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    if ((free_mask & ~7u) != 0 || free_mask == 0) return BV_EINVAL;
    if (opts->max_evals < 1 || opts->init_step <= 0.0) return BV_EINVAL;
    if (opts->precision != BV_FP64 && opts->precision != BV_MIXED) return BV_EINVAL;
    Space S;
    S.base = *theta0;
    S.mask = free_mask;
    S.two_nu = 2.0 * theta0->nu;
    const double vals[3] = {theta0->sigma2, theta0->range[0], theta0->nugget};
    const double los[3] = {lo->sigma2, lo->range[0], lo->nugget}, his[3] = {hi->sigma2, hi->range[0], hi->nugget};
    S.dim = 0;
    for (int j = 0; j < 3; ++j) {
        if (!(free_mask & (1u << j))) {  // fixed parameters are never checked against the box
            S.lo[j] = -1e300;
            S.hi[j] = 1e300;
            continue;
        }
        if (!(los[j] > 0.0) || !(his[j] >= los[j]) || !(vals[j] > 0.0)) return BV_EINVAL;
        S.lo[j] = log(los[j]);
        S.hi[j] = log(his[j]);
        ++S.dim;
    }
    // start inside the box
    bv_theta t0 = *theta0;
    t0.sigma2 = std::min(his[0], std::max(los[0], t0.sigma2));
    if (free_mask & BV_FREE_RANGE) {
        const double r0 = std::min(his[1], std::max(los[1], t0.range[0]));
        const double f = r0 / t0.range[0];
        for (int j = 0; j < 3; ++j) t0.range[j] *= f;
    }
    if (free_mask & BV_FREE_NUGGET) t0.nugget = std::min(his[2], std::max(los[2], t0.nugget));
    S.base = t0;
    std::vector<double> x(S.dim), xb;
    from_theta(S, t0, x.data());
    int evals = 0;
    double fb = INFINITY;
    const int prec = opts->precision;
    // search, then one restart around the optimum (smaller step)
    BV_TRY(nelder_mead(c, S, prec, x, opts->init_step, opts->ftol_rel, opts->xtol, opts->max_evals, &evals, &xb, &fb));
    BV_TRY(nelder_mead(c, S, prec, xb, std::max(opts->init_step * 0.1, 20.0 * opts->xtol), opts->ftol_rel, opts->xtol,
                       opts->max_evals, &evals, &xb, &fb));
    if (prec == BV_MIXED && std::isfinite(fb)) {
        // FP64 finish from the mixed-precision optimum
        BV_TRY(nelder_mead(c, S, BV_FP64, xb, std::max(opts->init_step * 0.02, 20.0 * opts->xtol), opts->ftol_rel,
                           opts->xtol, opts->max_evals, &evals, &xb, &fb));
    }
    bv_theta th;
    if (!to_theta(S, xb.data(), &th)) return BV_EINTERNAL;
    *theta_hat = th;
    if (loglik_hat) *loglik_hat = -fb;
    if (n_evals) *n_evals = evals;
    return std::isfinite(fb) ? BV_OK : BV_ENOTPD;
}
