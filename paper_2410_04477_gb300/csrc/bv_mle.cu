// bv_mle.cu -- maximum-likelihood driver over the block-Vecchia log-likelihood.
//
// The paper estimates theta with the derivative-free BOBYQA optimiser (Sec. 3.2); this
// library uses the derivative-free Nelder-Mead simplex method (Nelder and Mead 1965) with
// the standard coefficients (reflection 1, expansion 2, contraction 1/2, shrink 1/2) on
// the logarithms of the free parameters, projected onto the box [lo, hi].  Every
// objective value is one device evaluation of ell (bv_loglik); a non-positive-definite
// point scores -inf and is rejected by the simplex.
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
    double lo[3], hi[3];
};

bv_theta to_theta(const Space& S, const double* x) {
    bv_theta t = S.base;
    int k = 0;
    if (S.mask & BV_FREE_SIGMA2) t.sigma2 = exp(x[k++]);
    if (S.mask & BV_FREE_RANGE) {
        const double f = exp(x[k++]) / S.base.range[0];
        for (int j = 0; j < 3; ++j) t.range[j] = S.base.range[j] * f;
    }
    if (S.mask & BV_FREE_NUGGET) t.nugget = exp(x[k++]);
    return t;
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
    Space S;
    S.base = *theta0;
    S.mask = free_mask;
    S.dim = 0;
    auto add = [&](double v0, double l, double h) -> bool {
        if (!(l > 0.0) || !(h >= l) || !(v0 > 0.0)) return false;
        S.lo[S.dim] = log(l);
        S.hi[S.dim] = log(h);
        ++S.dim;
        return true;
    };
    if ((free_mask & BV_FREE_SIGMA2) && !add(theta0->sigma2, lo->sigma2, hi->sigma2)) return BV_EINVAL;
    if ((free_mask & BV_FREE_RANGE) && !add(theta0->range[0], lo->range[0], hi->range[0])) return BV_EINVAL;
    if ((free_mask & BV_FREE_NUGGET) && !add(theta0->nugget, lo->nugget, hi->nugget)) return BV_EINVAL;
    const int n = S.dim;
    int evals = 0;
    auto clampv = [&](std::vector<double>& x) {
        for (int j = 0; j < n; ++j) x[j] = std::min(S.hi[j], std::max(S.lo[j], x[j]));
    };
    int hard_error = BV_OK;
    auto f = [&](std::vector<double>& x) -> double {
        clampv(x);
        const bv_theta t = to_theta(S, x.data());
        double ll = -INFINITY;
        ++evals;
        const int st = bv_loglik(c, &t, opts->precision, &ll, nullptr);
        if (st != BV_OK && st != BV_ENOTPD) hard_error = st;
        return (st == BV_OK && std::isfinite(ll)) ? -ll : INFINITY;
    };
    // initial simplex
    std::vector<std::vector<double>> X(n + 1, std::vector<double>(n));
    {
        int k = 0;
        if (free_mask & BV_FREE_SIGMA2) X[0][k++] = log(theta0->sigma2);
        if (free_mask & BV_FREE_RANGE) X[0][k++] = log(theta0->range[0]);
        if (free_mask & BV_FREE_NUGGET) X[0][k++] = log(theta0->nugget);
        clampv(X[0]);
        for (int j = 0; j < n; ++j) {
            X[j + 1] = X[0];
            double step = opts->init_step;
            if (X[0][j] + step > S.hi[j]) step = -step;  // stay inside the box
            X[j + 1][j] += step;
        }
    }
    std::vector<double> F(n + 1);
    for (int j = 0; j <= n; ++j) {
        F[j] = f(X[j]);
        if (hard_error) return hard_error;
    }
    std::vector<int> idx(n + 1);
    std::vector<double> xc(n), xr(n), xe(n), xk(n);
    while (evals < opts->max_evals) {
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
        // convergence: value spread and simplex size
        double xs = 0.0;
        for (int j = 1; j <= n; ++j)
            for (int q = 0; q < n; ++q) xs = std::max(xs, fabs(X[j][q] - X[0][q]));
        const double fs = F[n] - F[0];
        if (std::isfinite(F[n]) && fs <= opts->ftol_rel * fabs(F[0]) && xs <= opts->xtol) break;
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
    *theta_hat = to_theta(S, X[best].data());
    if (loglik_hat) *loglik_hat = -F[best];
    if (n_evals) *n_evals = evals;
    return std::isfinite(F[best]) ? BV_OK : BV_ENOTPD;
}
