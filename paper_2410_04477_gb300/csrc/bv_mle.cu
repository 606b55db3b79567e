// bv_mle.cu -- maximum-likelihood driver over the block-Vecchia log-likelihood.
//
// The paper estimates theta with the derivative-free BOBYQA optimiser (Sec. 3.2), a
// trust-region method on interpolated quadratic models; this library runs trust-region
// Newton iterations on central-difference quadratic models (with newton_first, the
// default of the Python binding) and falls back to the derivative-free Nelder-Mead
// simplex method (Nelder and Mead 1965, the standard coefficients: reflection 1,
// expansion 2, contraction 1/2, shrink 1/2).
//
// Profile likelihood.  Write the covariance as sigma^2 (R_beta + eta I) with eta =
// tau^2 / sigma^2.  Every block's kriging weights depend on (beta, eta) only and its
// conditional covariance is sigma^2 times that at sigma^2 = 1, so with Q and D the
// quadratic form and log-determinant of Eq. 4 at sigma^2 = 1,
//     ell(sigma^2, beta, eta) = -(Q / sigma^2 + D + n log sigma^2 + n log 2 pi) / 2,
// which is concave in log sigma^2 with its maximum at sigma^2 = Q / n.  When sigma^2 is
// free (and the nugget is free or zero) the search therefore runs over (log beta,
// log eta) only, each point costing one evaluation at sigma^2 = 1 that returns Q and ell
// (bv_loglik_terms), and sigma^2 is set in closed form: Q / n clamped to the part of the
// box that keeps sigma^2 and tau^2 = eta sigma^2 inside [lo, hi].  Otherwise the search
// runs over log(sigma^2 / beta^(2 nu)), log beta, log tau^2 (the free ones); for the
// Matern model sigma^2 and beta are poorly identified separately but that combination is
// well identified, so the change of variables straightens the ridge of the surface.
//
// Points outside the box score -inf, and so does a non-positive-definite point.  With
// newton_first, trust-region Newton iterations run from the start point: in FP64 to the
// caller's tolerances; in mixed precision to coarse ones (step 1e-3 in log-parameters,
// relative ell change ten times the measured mixed error) with wide difference steps,
// then an FP64 polish.  Where they fail, or without newton_first, the search runs in two
// stages.  A coarse Nelder-Mead search (in the requested precision) stops at a simplex of
// diameter 1e-3 in log-parameters; the simplex is then rebuilt once around the best point
// and the search resumed (a standard guard against premature collapse).  An FP64 Newton
// polish on a central-difference quadratic model then takes the estimate to the caller's
// xtol in a few evaluations; where the model is not convex or a step fails to improve
// (e.g. an optimum on the box boundary), an FP64 Nelder-Mead search with the caller's
// tolerances finishes instead.  The returned estimate is the best FP64-scored point, and
// ell is its FP64 value.
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <condition_variable>
#include <mutex>
#include <thread>
#include <numeric>
#include <vector>

#include "bv_internal.h"

namespace {

struct Space {
    bv_theta base;
    uint32_t mask;
    int dim;
    double lo[4], hi[4];  // log-box of sigma^2, range, nugget, smoothness (in that order)
    bool profile;         // sigma^2 profiled out; coordinates (log beta, log nu, log eta)
    double n;             // number of observations
};

// Profile coordinates x -> the sigma^2 = 1 point (range, eta) it stands for.
bool to_unit_theta(const Space& S, const double* x, bv_theta* t, double* leta) {
    *t = S.base;
    int k = 0;
    double lbeta = log(S.base.range[0]), lnu = log(S.base.nu);
    *leta = -INFINITY;  // eta = 0 when the nugget is fixed at zero
    if (S.mask & BV_FREE_RANGE) lbeta = x[k++];
    if (S.mask & BV_FREE_NU) lnu = x[k++];
    if (S.mask & BV_FREE_NUGGET) *leta = x[k++];
    if (lbeta < S.lo[1] || lbeta > S.hi[1] || lnu < S.lo[3] || lnu > S.hi[3]) return false;
    t->sigma2 = 1.0;
    if (S.mask & BV_FREE_NU) t->nu = exp(lnu);
    if (S.mask & BV_FREE_RANGE) {
        const double f = exp(lbeta) / S.base.range[0];
        for (int j = 0; j < 3; ++j) t->range[j] = S.base.range[j] * f;
    }
    t->nugget = (S.mask & BV_FREE_NUGGET) ? exp(*leta) : 0.0;
    return true;
}

// The profile maximiser of ell over sigma^2 inside the box, given Q and log eta: Q / n,
// or, in logs, clamped to [lo, hi] of sigma^2 intersected with that of tau^2 - log eta.
bool profile_sigma2(const Space& S, double Q, double leta, double* s2, double* lsig) {
    double a = S.lo[0], b = S.hi[0];
    if (S.mask & BV_FREE_NUGGET) {
        a = std::max(a, S.lo[2] - leta);
        b = std::min(b, S.hi[2] - leta);
    }
    if (!(a <= b) || !(Q > 0.0)) return false;
    *s2 = Q / S.n;
    *lsig = log(*s2);
    if (*lsig < a || *lsig > b) {
        *lsig = std::min(b, std::max(a, *lsig));
        *s2 = exp(*lsig);
    }
    return true;
}

// Internal coordinates x -> theta.  x holds, for the free parameters in order:
// u = log sigma^2 - 2 nu log beta (if sigma^2 free), log beta (if range free), log nu (if
// the smoothness is free), log tau^2.
bool to_theta(const Space& S, const double* x, bv_theta* t) {
    *t = S.base;
    int k = 0;
    double lsig = log(S.base.sigma2), lbeta = log(S.base.range[0]), ltau = log(S.base.nugget > 0 ? S.base.nugget : 1e-300);
    double lnu = log(S.base.nu);
    double u = 0.0;
    const bool fs = S.mask & BV_FREE_SIGMA2, fr = S.mask & BV_FREE_RANGE, fn = S.mask & BV_FREE_NUGGET,
               fv = S.mask & BV_FREE_NU;
    if (fs) u = x[k++];
    if (fr) lbeta = x[k++];
    if (fv) lnu = x[k++];
    if (fn) ltau = x[k++];
    if (fs) lsig = u + 2.0 * exp(lnu) * lbeta;
    if (lsig < S.lo[0] || lsig > S.hi[0] || lbeta < S.lo[1] || lbeta > S.hi[1] || ltau < S.lo[2] || ltau > S.hi[2] ||
        lnu < S.lo[3] || lnu > S.hi[3])
        return false;
    if (fs) t->sigma2 = exp(lsig);
    if (fv) t->nu = exp(lnu);
    if (fr) {
        const double f = exp(lbeta) / S.base.range[0];
        for (int j = 0; j < 3; ++j) t->range[j] = S.base.range[j] * f;
    }
    if (fn) t->nugget = exp(ltau);
    return true;
}

void from_theta(const Space& S, const bv_theta& t, double* x) {
    int k = 0;
    const double lb = log(t.range[0]);
    if (S.profile) {
        if (S.mask & BV_FREE_RANGE) x[k++] = lb;
        if (S.mask & BV_FREE_NU) x[k++] = log(t.nu);
        if (S.mask & BV_FREE_NUGGET) x[k++] = log(t.nugget) - log(t.sigma2);
        return;
    }
    if (S.mask & BV_FREE_SIGMA2) x[k++] = log(t.sigma2) - 2.0 * t.nu * lb;
    if (S.mask & BV_FREE_RANGE) x[k++] = lb;
    if (S.mask & BV_FREE_NU) x[k++] = log(t.nu);
    if (S.mask & BV_FREE_NUGGET) x[k++] = log(t.nugget);
}

// One log-likelihood evaluation for a search: (ell, and with want_q the quadratic form
// Q) at theta in the given precision; returns a bv_status.
struct Evaluator {
    virtual int eval(const bv_theta& t, int prec, bool want_q, double* ll, double* Q) = 0;
    virtual ~Evaluator() = default;
};

// A single-dataset context: direct synchronous calls.
struct DirectEval : Evaluator {
    bv_ctx* c;
    explicit DirectEval(bv_ctx* ctx) : c(ctx) {}
    int eval(const bv_theta& t, int prec, bool want_q, double* ll, double* Q) override {
        if (want_q) return bv_loglik_terms(c, &t, prec, ll, Q, nullptr);
        return bv_loglik(c, &t, prec, ll, nullptr);
    }
};

// The objective f = -ell at internal coordinates x, one device evaluation per call.
// Remembers the best full theta it has scored (reset() between precisions).
struct Objective {
    Evaluator* ev;
    const Space* S;
    int prec = BV_FP64;
    int evals = 0;
    int hard_error = BV_OK;
    double fbest = INFINITY;
    bv_theta tbest{};
    std::vector<double> xbest;

    void reset(int p) {
        prec = p;
        fbest = INFINITY;
    }
    double operator()(const std::vector<double>& x) {
        bv_theta t;
        double ll = -INFINITY;
        if (S->profile) {
            double leta, Q = 0.0;
            if (!to_unit_theta(*S, x.data(), &t, &leta)) return INFINITY;
            ++evals;
            const int st = ev->eval(t, prec, true, &ll, &Q);
            if (st != BV_OK && st != BV_ENOTPD) hard_error = st;
            double s2, lsig;
            if (st != BV_OK || !std::isfinite(ll) || !profile_sigma2(*S, Q, leta, &s2, &lsig)) return INFINITY;
            // ell at sigma^2 from ell at 1:  + (Q - Q / sigma^2 - n log sigma^2) / 2
            ll += 0.5 * (Q - Q / s2 - S->n * lsig);
            t.sigma2 = s2;
            if (S->mask & BV_FREE_NUGGET) t.nugget = exp(leta + lsig);
        } else {
            if (!to_theta(*S, x.data(), &t)) return INFINITY;
            ++evals;
            double Qd = 0.0;
            const int st = ev->eval(t, prec, false, &ll, &Qd);
            if (st != BV_OK && st != BV_ENOTPD) hard_error = st;
            if (st != BV_OK || !std::isfinite(ll)) return INFINITY;
        }
        if (-ll < fbest) {
            fbest = -ll;
            tbest = t;
            xbest = x;
        }
        return -ll;
    }
};

// One Nelder-Mead search from x0 with initial step `step` (`step_last` for a free
// nugget's coordinate, the last one); returns the best point and value of f.
int nelder_mead(Objective& f, const Space& S, std::vector<double> x0, double step, double step_last,
                double ftol, double xtol, int max_evals, std::vector<double>* xbest, double* fbest) {
    const int n = S.dim;
    int& hard_error = f.hard_error;
    int* evals = &f.evals;
    std::vector<std::vector<double>> X(n + 1, x0);
    // the nugget, when free, is the last coordinate and may take its own step
    for (int j = 0; j < n; ++j) X[j + 1][j] += (j == n - 1 && (S.mask & BV_FREE_NUGGET)) ? step_last : step;
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

// Cholesky solve of the n x n (n <= 3) system H p = -g; false unless H is positive definite.
bool newton_step(std::vector<double> H, const std::vector<double>& g, int n, std::vector<double>* p) {
    for (int j = 0; j < n; ++j) {
        for (int k = 0; k < j; ++k) H[j * n + j] -= H[j * n + k] * H[j * n + k];
        if (!(H[j * n + j] > 0.0)) return false;
        H[j * n + j] = sqrt(H[j * n + j]);
        for (int i = j + 1; i < n; ++i) {
            for (int k = 0; k < j; ++k) H[i * n + j] -= H[i * n + k] * H[j * n + k];
            H[i * n + j] /= H[j * n + j];
        }
    }
    std::vector<double> w(n);
    for (int i = 0; i < n; ++i) {
        double v = -g[i];
        for (int k = 0; k < i; ++k) v -= H[i * n + k] * w[k];
        w[i] = v / H[i * n + i];
    }
    p->assign(n, 0.0);
    for (int i = n - 1; i >= 0; --i) {
        double v = w[i];
        for (int k = i + 1; k < n; ++k) v -= H[k * n + i] * (*p)[k];
        (*p)[i] = v / H[i * n + i];
    }
    return true;
}

// Newton polish of f from x (f(x) = fx) on a central-difference quadratic model with
// step h: gradient and Hessian from 1 + 2n + n(n-1)/2 evaluations, a Newton step (at
// most `cap` in the sup norm), repeated while it improves f (at most `iters` times).  True when the last step was
// within xtol or the model's predicted decrease g^T H^-1 g / 2 was within ftol |f| (the
// rounding floor of f bounds how well a weakly identified direction can be resolved);
// false when the model was not convex, a point left the box, a step did not improve f,
// or the iterations ran out (the caller then falls back to Nelder-Mead).
bool newton_polish(Objective& f, const Space& S, std::vector<double>* x, double* fx, double h, double xtol,
                   double ftol, int max_evals, double cap = 0.1, int iters = 4) {
    const int n = S.dim;
    std::vector<double> H(n * n), g(n), fp(n), fm(n), p, y;
    for (int it = 0; it < iters; ++it) {
        if (f.evals + 2 + n * (n + 3) / 2 > max_evals) return false;
        for (int i = 0; i < n; ++i) {
            y = *x;
            y[i] += h;
            fp[i] = f(y);
            y[i] = (*x)[i] - h;
            fm[i] = f(y);
            if (f.hard_error || !std::isfinite(fp[i]) || !std::isfinite(fm[i])) return false;
            g[i] = (fp[i] - fm[i]) / (2.0 * h);
            H[i * n + i] = (fp[i] - 2.0 * *fx + fm[i]) / (h * h);
        }
        for (int i = 0; i < n; ++i)
            for (int j = i + 1; j < n; ++j) {
                y = *x;
                y[i] += h;
                y[j] += h;
                const double fij = f(y);
                if (f.hard_error || !std::isfinite(fij)) return false;
                H[i * n + j] = H[j * n + i] = (fij - fp[i] - fp[j] + *fx) / (h * h);
            }
        if (!newton_step(H, g, n, &p)) return false;
        double len = 0.0, pred = 0.0;
        for (int i = 0; i < n; ++i) {
            len = std::max(len, fabs(p[i]));
            pred -= 0.5 * g[i] * p[i];
        }
        const double sc = len > cap ? cap / len : 1.0;
        y = *x;
        for (int i = 0; i < n; ++i) y[i] += sc * p[i];
        const double fy = f(y);
        if (f.hard_error) return false;
        const bool improved = fy < *fx;
        if (improved) {
            *x = y;
            *fx = fy;
        }
        if (len <= xtol || pred <= ftol * fabs(*fx)) return true;
        if (!improved) return false;
    }
    return false;
}

// Central-difference gradient and Hessian of f at x (f(x) = fx) with step h: 2n + n(n-1)/2
// evaluations.  False when a point is not finite (outside the box, not positive definite).
bool fd_model(Objective& f, const std::vector<double>& x, double fx, double h, std::vector<double>* g,
              std::vector<double>* H) {
    const int n = (int)x.size();
    std::vector<double> fp(n), y;
    g->assign(n, 0.0);
    H->assign((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) {
        y = x;
        y[i] += h;
        fp[i] = f(y);
        y[i] = x[i] - h;
        const double fm = f(y);
        if (f.hard_error || !std::isfinite(fp[i]) || !std::isfinite(fm)) return false;
        (*g)[i] = (fp[i] - fm) / (2.0 * h);
        (*H)[i * n + i] = (fp[i] - 2.0 * fx + fm) / (h * h);
    }
    for (int i = 0; i < n; ++i)
        for (int j = i + 1; j < n; ++j) {
            y = x;
            y[i] += h;
            y[j] += h;
            const double fij = f(y);
            if (f.hard_error || !std::isfinite(fij)) return false;
            (*H)[i * n + j] = (*H)[j * n + i] = (fij - fp[i] - fp[j] + fx) / (h * h);
        }
    return true;
}

// Trust-region Newton iteration (the basic trust-region algorithm of Nocedal and Wright,
// Numerical Optimization, Alg. 4.1, with a sup-norm radius) on the central-difference
// model of fd_model.  Each iteration builds the model at x, solves H p = -g (H shifted by
// a multiple of the identity where it is not positive definite, the Levenberg-Marquardt
// remedy), truncates p to the radius and evaluates the step; the ratio of the actual to
// the model's decrease grows the radius (ratio > 3/4 at a truncated step) or shrinks it
// (ratio < 1/4: a quarter of the step taken).  A step that does not lower f is retried
// at the smaller radius on the same model, at most three times.  Returns true when the
// unshifted Newton step is within xtol or its predicted decrease g^T H^-1 g / 2 within
// ftol |f|; false when the iterations or evaluations run out or no retry lowers f (the
// caller then falls back to the simplex search).
bool trust_newton(Objective& f, const Space& S, std::vector<double>* x, double* fx, double h, double xtol,
                  double ftol, int max_evals, double rad, int iters, int* accepted = nullptr) {
    const int n = S.dim;
    const bool log = getenv("BV_LOG_MLE") && atoi(getenv("BV_LOG_MLE")) >= 2;
    if (accepted) *accepted = 0;
    std::vector<double> g, H, Hs, p, st(n), y;
    double maxdiag = 0.0;
    for (int it = 0; it < iters; ++it) {
        if (f.evals + 2 + n * (n + 3) / 2 + 3 > max_evals) return false;
        if (!fd_model(f, *x, *fx, h, &g, &H)) return false;
        maxdiag = 0.0;
        for (int i = 0; i < n; ++i) maxdiag = std::max(maxdiag, fabs(H[i * n + i]));
        double lam = 0.0;
        Hs = H;
        while (!newton_step(Hs, g, n, &p)) {
            lam = lam > 0.0 ? 4.0 * lam : 1e-3 * maxdiag + 1e-300;
            if (!(lam < 1e6 * maxdiag + 1.0)) return false;
            Hs = H;
            for (int i = 0; i < n; ++i) Hs[i * n + i] += lam;
        }
        double len = 0.0, pred_full = 0.0;
        for (int i = 0; i < n; ++i) {
            len = std::max(len, fabs(p[i]));
            pred_full -= 0.5 * g[i] * p[i];
        }
        bool improved = false;
        for (int tr = 0; tr < 4 && !improved; ++tr) {
            const double sc = len > rad ? rad / len : 1.0;
            double pred = 0.0;
            for (int i = 0; i < n; ++i) st[i] = sc * p[i];
            for (int i = 0; i < n; ++i) {
                double hs = 0.0;
                for (int j = 0; j < n; ++j) hs += H[i * n + j] * st[j];
                pred -= g[i] * st[i] + 0.5 * st[i] * hs;
            }
            y = *x;
            for (int i = 0; i < n; ++i) y[i] += st[i];
            const double fy = f(y);
            if (f.hard_error) return false;
            const double ratio = pred > 0.0 && std::isfinite(fy) ? (*fx - fy) / pred : -1.0;
            if (ratio > 0.75 && sc < 1.0) rad = std::min(2.0 * rad, 4.0);
            else if (ratio < 0.25) rad = 0.25 * sc * len;
            if (log)
                fprintf(stderr, "bv_mle:   it %d try %d: f %.9g -> %.9g, predicted %.3g, full step %.3g (lambda %.3g), "
                        "radius %.3g\n", it, tr, *fx, fy, pred, len, lam, rad);
            if (fy < *fx) {
                *x = y;
                *fx = fy;
                improved = true;
                if (accepted) ++*accepted;
            }
        }
        if (lam == 0.0 && (len <= xtol || pred_full <= ftol * fabs(*fx))) return true;
        if (!improved) return false;
    }
    return false;
}

}  // namespace

// The mixed-precision search stage scores points for an FP64 polish that fixes the final
// estimate, so it evaluates without the mixed path's FP64 check (its error sets the stage's
// tolerance instead, see mle_search); the caller's setting is restored on return.
struct UncheckedMixed {
    bv_ctx* c;
    double old;
    explicit UncheckedMixed(bv_ctx* ctx) : c(ctx), old(ctx->mixed_tol) { bv_set_mixed_tolerance(c, 0.0); }
    ~UncheckedMixed() { bv_set_mixed_tolerance(c, old); }
};

// The search of one dataset with n observations: checks, start point, the stages.
static int mle_search(bv_ctx* c, Evaluator* ev, double n_obs, const bv_theta* theta0, const bv_theta* lo,
                      const bv_theta* hi, uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat,
                      double* loglik_hat, int32_t* n_evals) {
    if (!c || !lo || !hi || !opts || !theta_hat || !theta0) return BV_EINVAL;

    if ((free_mask & ~15u) != 0 || free_mask == 0) return BV_EINVAL;
    if (opts->max_evals < 1 || opts->init_step <= 0.0) return BV_EINVAL;
    if (opts->precision != BV_FP64 && opts->precision != BV_MIXED) return BV_EINVAL;
    Space S;
    S.base = *theta0;
    S.mask = free_mask;
    const double vals[4] = {theta0->sigma2, theta0->range[0], theta0->nugget, theta0->nu};
    const double los[4] = {lo->sigma2, lo->range[0], lo->nugget, lo->nu};
    const double his[4] = {hi->sigma2, hi->range[0], hi->nugget, hi->nu};
    if ((free_mask & BV_FREE_NU) && !(his[3] <= BV_NU_MAX)) return BV_EINVAL;
    S.dim = 0;
    for (int j = 0; j < 4; ++j) {
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
    if (free_mask & BV_FREE_NU) t0.nu = std::min(his[3], std::max(los[3], t0.nu));
    S.base = t0;
    S.n = n_obs;
    S.profile = (free_mask & BV_FREE_SIGMA2) && ((free_mask & BV_FREE_NUGGET) || t0.nugget == 0.0);
    if (S.profile) --S.dim;
    std::vector<double> x(S.dim), xb;
    from_theta(S, t0, x.data());
    Objective obj{ev, &S};
    double fb = INFINITY;
    const int prec = opts->precision;
    if (S.dim == 0) {
        // only sigma^2 free (nugget zero): the closed form is the estimate
        obj.reset(BV_FP64);
        fb = obj(x);
        BV_TRY(obj.hard_error);
    } else {
        // Coarse search: Nelder-Mead to a simplex of diameter 1e-3 and relative ell spread
        // 1e-7 (in mixed precision no tighter than 1e-6 or ten times its measured error at
        // the start point), restarted once around the optimum; then, in FP64, a Newton polish
        // to xtol, or, if that fails, the Nelder-Mead search and restart to the caller's
        // tolerances.
        const double s0 = opts->init_step, sn = opts->init_step_nugget > 0.0 ? opts->init_step_nugget : s0;
        double ftol_c = std::max(opts->ftol_rel, 1e-7);
        const double xtol_c = std::max(opts->xtol, 1e-3);
        if (prec == BV_MIXED) {
            obj.reset(BV_FP64);
            const double f64 = obj(x);
            BV_TRY(obj.hard_error);
            obj.reset(BV_MIXED);
            const double f32 = obj(x);
            BV_TRY(obj.hard_error);
            const double err = (std::isfinite(f64) && std::isfinite(f32)) ? fabs(f32 - f64) / fabs(f64) : 1e-6;
            // no finer than the mixed path resolves ell: ten times its error at the start,
            // and at least its stated relative accuracy (1e-6): between nearby points its
            // FP32 rounding moves ell by about that much, more than at any single point
            ftol_c = std::max(ftol_c, std::max(10.0 * err, 1e-6));
        }
        obj.reset(prec);
        // Newton first: trust-region steps on a central-difference model from the start
        // point; in FP64 straight to the caller's tolerances, in mixed precision to the
        // coarse ones with difference steps of 0.02 (FP32 rounding of ell, about 1e-8 of
        // it, would swamp difference quotients over 1e-3).  The simplex search runs only
        // if the steps fail, from the best point they reached.
        bool near = false, done = false;
        if (opts->newton_first) {
            const bool fp64 = prec == BV_FP64;
            double fx = obj(x);
            BV_TRY(obj.hard_error);
            std::vector<double> xn = x;
            int acc = 0;
            near = std::isfinite(fx) && trust_newton(obj, S, &xn, &fx, fp64 ? 1e-3 : 2e-2, fp64 ? opts->xtol : xtol_c,
                                                     fp64 ? opts->ftol_rel : ftol_c, opts->max_evals, 0.5, 40, &acc);
            BV_TRY(obj.hard_error);
            // in mixed precision, iterations that moved and then stalled have reached the
            // FP32 rounding floor of ell near the optimum: the FP64 polish takes over there
            if (!near && !fp64 && acc > 0 && std::isfinite(fx)) {
                near = true;
                if (getenv("BV_LOG_MLE")) fprintf(stderr, "bv_mle: Newton-first stalled after %d steps\n", acc);
            }
            if (near) {
                xb = xn;
                fb = fx;
                done = fp64;
            } else if (!obj.xbest.empty()) {
                x = obj.xbest;
                obj.reset(prec);
            }
            if (getenv("BV_LOG_MLE"))
                fprintf(stderr, "bv_mle: Newton-first %s after %d evals\n", near ? "converged" : "failed",
                        obj.evals);
        }
        if (!near) {
            BV_TRY(nelder_mead(obj, S, x, s0, sn, ftol_c, xtol_c, opts->max_evals, &xb, &fb));
            const double s1 = std::max(s0 * 0.1, 20.0 * xtol_c);
            BV_TRY(nelder_mead(obj, S, xb, s1, s1, ftol_c, xtol_c, opts->max_evals, &xb, &fb));
        }
        if (std::isfinite(fb) && !done) {
            obj.reset(BV_FP64);
            fb = obj(xb);
            BV_TRY(obj.hard_error);
            const int coarse = obj.evals;
            done = std::isfinite(fb) && (opts->newton_first
                                             ? trust_newton(obj, S, &xb, &fb, 1e-3, opts->xtol, opts->ftol_rel,
                                                            opts->max_evals, 0.1, 8)
                                             : newton_polish(obj, S, &xb, &fb, 1e-3, opts->xtol, opts->ftol_rel,
                                                             opts->max_evals));
            BV_TRY(obj.hard_error);
            if (getenv("BV_LOG_MLE"))
                fprintf(stderr, "bv_mle: coarse search %d evals, Newton polish %s after %d\n", coarse,
                        done ? "converged" : "fell back", obj.evals - coarse);
            if (!done) {
                xb = obj.xbest;
                const double s2 = std::max(s0 * 0.02, 20.0 * opts->xtol);
                BV_TRY(nelder_mead(obj, S, xb, s2, s2, opts->ftol_rel, opts->xtol, opts->max_evals, &xb, &fb));
                const double s3 = std::max(s0 * 0.01, 20.0 * opts->xtol);
                BV_TRY(nelder_mead(obj, S, xb, s3, s3, opts->ftol_rel, opts->xtol, opts->max_evals, &xb, &fb));
            }
        }
    }
    if (!std::isfinite(obj.fbest)) {
        *theta_hat = t0;
        if (loglik_hat) *loglik_hat = -INFINITY;
        if (n_evals) *n_evals = obj.evals;
        return BV_ENOTPD;
    }
    *theta_hat = obj.tbest;
    if (loglik_hat) *loglik_hat = -obj.fbest;
    if (n_evals) *n_evals = obj.evals;
    return BV_OK;
}

// Geometric centre of the box (the warm start's input when no start is given).
static bv_theta box_centre(const bv_theta* lo, const bv_theta* hi) {
    bv_theta mid = *lo;
    mid.sigma2 = sqrt(lo->sigma2 * hi->sigma2);
    for (int j = 0; j < 3; ++j) mid.range[j] = sqrt(lo->range[j] * hi->range[j]);
    mid.nugget = sqrt(lo->nugget * hi->nugget);
    mid.nu = sqrt(lo->nu * hi->nu);
    return mid;
}

extern "C" int bv_mle(bv_ctx* c, const bv_theta* theta0, const bv_theta* lo, const bv_theta* hi,
                      uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat, double* loglik_hat,
                      int32_t* n_evals) {
    if (!c || !lo || !hi || !opts || !theta_hat) return BV_EINVAL;
    if (c->ndata != 1) return c->ndata == 0 ? BV_ESTATE : BV_EINVAL;
    if (!c->have_nn) return BV_ESTATE;
    bv_theta warm;
    if (!theta0) {
        // learned warm start from the centre of the box (the smoothness and the range
        // ratios are taken from it; the network sets sigma^2, the range and tau^2)
        if (!c->have_mlp) return BV_ESTATE;
        bv_theta mid = box_centre(lo, hi);
        if (free_mask & BV_FREE_NU) mid.nu = 0.0;  // start from the network's smoothness class
        BV_TRY(bv_warmstart_predict(c, &mid, &warm));
        if (free_mask & BV_FREE_NU) warm.nu = std::min(hi->nu, std::max(lo->nu, warm.nu));
        theta0 = &warm;
    }
    UncheckedMixed unchecked(c);
    DirectEval ev(c);
    return mle_search(c, &ev, (double)c->n_tot, theta0, lo, hi, free_mask, opts, theta_hat, loglik_hat, n_evals);
}

// ------------------------------------------------------------------------------------
// Test support: bv_mle's search on a synthetic likelihood evaluated on the host, so that
// the optimizer's logic (profiling, trust-region Newton, simplex fallback, the box) runs
// without a device.  With u = log(beta / beta0), v = log(eta / eta0), eta = tau^2 / sigma^2:
//     Q = n exp(c_q u),  D = n (a u^2 + b v^2 + c_uv u v + k (u^4 + v^4)),
//     ell = -(Q / sigma^2 + D + n log sigma^2 + n log 2 pi) / 2,
// the profile form of Eq. 4's sum; a mixed-precision evaluation adds the deterministic
// perturbation n * 1e-7 * sin(1e3 (u + 2 v)) (a stand-in for FP32 rounding).
// ------------------------------------------------------------------------------------
namespace {
struct SyntheticEval : Evaluator {
    double n, lb0, le0, cq, a, b, cuv, k;
    int eval(const bv_theta& t, int prec, bool, double* ll, double* Q) override {
        if (!(t.sigma2 > 0.0) || !(t.range[0] > 0.0) || !(t.nugget > 0.0)) return BV_ENOTPD;
        const double u = log(t.range[0]) - lb0, v = log(t.nugget / t.sigma2) - le0;
        const double q = n * exp(cq * u);
        const double D = n * (a * u * u + b * v * v + cuv * u * v + k * (u * u * u * u + v * v * v * v));
        double l = -0.5 * (q / t.sigma2 + D + n * log(t.sigma2) + n * kLog2PiHost);
        if (prec == BV_MIXED) l += n * 1e-7 * sin(1e3 * (u + 2.0 * v));
        *ll = l;
        *Q = q / t.sigma2;  // the quadratic form at this sigma^2
        return BV_OK;
    }
    static constexpr double kLog2PiHost = 1.8378770664093454835606594728112;
};
}  // namespace

extern "C" int bv_mle_check(const double* model, const bv_theta* theta0, const bv_theta* lo, const bv_theta* hi,
                            uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat, double* loglik_hat,
                            int32_t* n_evals) {
    if (!model || !theta0) return BV_EINVAL;
    SyntheticEval ev;
    ev.n = model[0];
    ev.lb0 = log(model[1]);
    ev.le0 = log(model[2]);
    ev.cq = model[3];
    ev.a = model[4];
    ev.b = model[5];
    ev.cuv = model[6];
    ev.k = model[7];
    if (!(ev.n > 0.0) || !(model[1] > 0.0) || !(model[2] > 0.0)) return BV_EINVAL;
    bv_ctx* dummy = reinterpret_cast<bv_ctx*>(&ev);  // mle_search uses the context only as a non-null handle
    return mle_search(dummy, &ev, ev.n, theta0, lo, hi, free_mask, opts, theta_hat, loglik_hat, n_evals);
}

// ------------------------------------------------------------------------------------
// Many datasets at once.  Each dataset's search runs unchanged in its own host thread;
// its evaluations meet at a barrier, and when every unfinished search is waiting one
// batched evaluation (one graph launch over all datasets, per precision requested) scores
// them all.  Datasets without a pending request are evaluated at their last point.
// ------------------------------------------------------------------------------------
namespace {

struct Batch {
    bv_ctx* c;
    int nd;
    std::mutex mu;
    std::condition_variable cv;
    int active = 0, waiting = 0;
    uint64_t generation = 0;
    std::vector<bv_theta> th, last;
    std::vector<int> prec;
    std::vector<char> pending;
    std::vector<double> ll, Q;
    std::vector<int> st;
    int batches = 0;

    int request(int ds, const bv_theta& t, int p, double* oll, double* oQ) {
        std::unique_lock<std::mutex> lk(mu);
        th[ds] = t;
        last[ds] = t;
        prec[ds] = p;
        pending[ds] = 1;
        ++waiting;
        const uint64_t gen = generation;
        if (waiting == active) run_locked();
        else cv.wait(lk, [&] { return generation != gen; });
        *oll = ll[ds];
        *oQ = Q[ds];
        return st[ds];
    }
    void finish() {
        std::unique_lock<std::mutex> lk(mu);
        --active;
        if (active > 0 && waiting == active) run_locked();
    }
    void run_locked() {
        std::vector<bv_theta> ths(nd);
        std::vector<double> l(nd), q(nd);
        for (int p : {(int)BV_FP64, (int)BV_MIXED}) {
            bool any = false;
            for (int k = 0; k < nd; ++k) any = any || (pending[k] && prec[k] == p);
            if (!any) continue;
            for (int k = 0; k < nd; ++k) ths[k] = (pending[k] && prec[k] == p) ? th[k] : last[k];
            const int s = bv_loglik_terms_multi(c, ths.data(), p, l.data(), q.data());
            ++batches;
            for (int k = 0; k < nd; ++k)
                if (pending[k] && prec[k] == p) {
                    ll[k] = l[k];
                    Q[k] = q[k];
                    st[k] = (s == BV_OK || s == BV_ENOTPD) ? (std::isfinite(l[k]) ? BV_OK : BV_ENOTPD) : s;
                }
        }
        for (int k = 0; k < nd; ++k) pending[k] = 0;
        waiting = 0;
        ++generation;
        cv.notify_all();
    }
};

struct BatchEval : Evaluator {
    Batch* b;
    int ds;
    int eval(const bv_theta& t, int prec, bool, double* ll, double* Q) override {
        return b->request(ds, t, prec, ll, Q);
    }
};

}  // namespace

extern "C" int bv_mle_multi(bv_ctx* c, const bv_theta* theta0, const bv_theta* lo, const bv_theta* hi,
                            uint32_t free_mask, const bv_mle_opts* opts, bv_theta* theta_hat, double* loglik_hat,
                            int32_t* n_evals, int32_t* status, int32_t* n_batches) {
    if (!c || !lo || !hi || !opts || !theta_hat) return BV_EINVAL;
    if (c->ndata < 1) return BV_ESTATE;
    if (!c->have_nn) return BV_ESTATE;
    const int nd = c->ndata;
    std::vector<bv_theta> start(nd);
    if (theta0) {
        for (int k = 0; k < nd; ++k) start[k] = theta0[k];
    } else {
        if (!c->have_mlp) return BV_ESTATE;
        std::vector<bv_theta> mid(nd, box_centre(lo, hi));
        if (free_mask & BV_FREE_NU)
            for (auto& t : mid) t.nu = 0.0;  // start from the network's smoothness class
        BV_TRY(bv_warmstart_predict_multi(c, mid.data(), start.data()));
        if (free_mask & BV_FREE_NU)
            for (auto& t : start) t.nu = std::min(hi->nu, std::max(lo->nu, t.nu));
    }
    UncheckedMixed unchecked(c);
    Batch b;
    b.c = c;
    b.nd = nd;
    b.active = nd;
    b.th = start;
    b.last = start;
    b.prec.assign(nd, BV_FP64);
    b.pending.assign(nd, 0);
    b.ll.assign(nd, -INFINITY);
    b.Q.assign(nd, 0.0);
    b.st.assign(nd, BV_OK);
    std::vector<int> res(nd, BV_OK);
    std::vector<double> llh(nd, -INFINITY);
    std::vector<int32_t> ne(nd, 0);
    std::vector<std::thread> pool;
    pool.reserve(nd);
    for (int k = 0; k < nd; ++k) {
        pool.emplace_back([&, k] {
            BatchEval ev;
            ev.b = &b;
            ev.ds = k;
            const double n_obs = (double)(c->pt_off[k + 1] - c->pt_off[k]);
            res[k] = mle_search(c, &ev, n_obs, &start[k], lo, hi, free_mask, opts, &theta_hat[k], &llh[k], &ne[k]);
            b.finish();
        });
    }
    for (auto& t : pool) t.join();
    int worst = BV_OK;
    for (int k = 0; k < nd; ++k) {
        if (loglik_hat) loglik_hat[k] = llh[k];
        if (n_evals) n_evals[k] = ne[k];
        if (status) status[k] = res[k];
        if (res[k] != BV_OK && res[k] != BV_ENOTPD) worst = res[k];
    }
    if (n_batches) *n_batches = b.batches;
    return worst;
}
