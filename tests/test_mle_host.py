"""The MLE driver's search (bv_mle's stages: sigma^2 profiled out, trust-region Newton
first or the simplex first, the FP64 polish, the box) on a synthetic likelihood evaluated
on the host (bv_mle_check), against the optimum of the same closed form found by SciPy.
No device: this checks the optimizer's logic, which the GPU tests exercise only through
the block-Vecchia likelihood."""
import numpy as np
import pytest
from scipy.optimize import minimize

from paper_2410_04477_gb300 import bv

# n, beta0, eta0, c_q, a, b, c_uv, k
MODEL = np.array([2.0e4, 0.05, 3e-3, 0.3, 2.0, 0.5, 0.3, 0.05])


def _profile_optimum(model):
    # ell profiled over sigma^2 (at sigma^2 = Q / n): -(n log(Q / n) + n + D + n log 2 pi) / 2,
    # with n log(Q / n) = n c_q u: -(n + n f(u, v) + n log 2 pi) / 2
    n, _, _, cq, a, b, cuv, k = model
    f = lambda x: cq * x[0] + a * x[0] ** 2 + b * x[1] ** 2 + cuv * x[0] * x[1] + k * (x[0] ** 4 + x[1] ** 4)
    r = minimize(f, [0.0, 0.0], method="BFGS", options=dict(gtol=1e-12))
    u, v = r.x
    s2 = np.exp(cq * u)
    ell = -0.5 * (n + n * f(r.x) + n * np.log(2 * np.pi))
    return u, v, s2, ell


def _ell(model, s2, beta, tau2):
    n, b0, e0, cq, a, b, cuv, k = model
    u, v = np.log(beta / b0), np.log(tau2 / s2 / e0)
    q = n * np.exp(cq * u)
    d = n * (a * u * u + b * v * v + cuv * u * v + k * (u ** 4 + v ** 4))
    return -0.5 * (q / s2 + d + n * np.log(s2) + n * np.log(2 * np.pi))


LO, HI = bv.theta(0.01, 0.001, 1.5, 1e-6), bv.theta(100.0, 3.0, 1.5, 10.0)


@pytest.mark.parametrize("newton_first", [True, False])
@pytest.mark.parametrize("prec_name", ["BV_FP64", "BV_MIXED"])
@pytest.mark.parametrize("start", [(1.0, 0.1, 1e-2), (0.8, 0.06, 2e-3), (5.0, 0.5, 1.0)])
def test_search_reaches_the_profile_optimum(prec_name, newton_first, start):
    u, v, s2, ell = _profile_optimum(MODEL)
    th0 = bv.theta(start[0], start[1], 1.5, start[2])
    th, ll, ne, st = bv.mle_check(MODEL, th0, LO, HI, precision=getattr(bv, prec_name), ftol_rel=1e-13,
                                  xtol=1e-8, newton_first=newton_first)
    assert st == 0
    beta_hat, s2_hat = th.range[0], th.sigma2
    eta_hat = th.nugget / s2_hat
    assert abs(np.log(beta_hat / MODEL[1]) - u) < 1e-5
    assert abs(np.log(eta_hat / MODEL[2]) - v) < 1e-5
    assert abs(s2_hat / s2 - 1) < 1e-5
    # the returned ell is the (FP64) value at the returned theta, and the maximum
    assert ll == pytest.approx(_ell(MODEL, s2_hat, beta_hat, th.nugget), rel=1e-13, abs=1e-9)
    assert abs(ll - ell) <= 1e-10 * abs(ell)
    assert 0 < ne < 2000


def test_newton_first_needs_fewer_evaluations():
    th0 = bv.theta(1.0, 0.1, 1.5, 1e-2)
    _, _, ne_n, _ = bv.mle_check(MODEL, th0, LO, HI, ftol_rel=1e-12, xtol=1e-7, newton_first=True)
    _, _, ne_s, _ = bv.mle_check(MODEL, th0, LO, HI, ftol_rel=1e-12, xtol=1e-7, newton_first=False)
    assert ne_n < 0.6 * ne_s, (ne_n, ne_s)


def test_sigma2_bound_holds():
    # an upper bound on sigma^2 below the optimum's Q / n: the estimate sits on the bound,
    # the search still ends (Newton fails at the kink, the simplex finishes)
    _, _, s2, _ = _profile_optimum(MODEL)
    hi = bv.theta(0.9 * s2, 3.0, 1.5, 10.0)
    th, ll, ne, st = bv.mle_check(MODEL, bv.theta(0.5, 0.1, 1.5, 1e-2), LO, hi, ftol_rel=1e-12, xtol=1e-7)
    assert st == 0
    assert th.sigma2 <= 0.9 * s2 * (1 + 1e-12)
    assert th.sigma2 == pytest.approx(0.9 * s2, rel=1e-6)
    # no better point nearby inside the box
    for k in range(3):
        for sgn in (-1, 1):
            v = [th.sigma2, th.range[0], th.nugget]
            v[k] *= np.exp(sgn * 1e-3)
            if v[0] <= 0.9 * s2:
                assert _ell(MODEL, *v) <= ll + 1e-9 * abs(ll)


def test_fixed_nugget_searches_without_profiling():
    # nugget fixed (not free): the direct search over log(sigma^2 / beta^(2 nu)) and log beta
    tau2 = 5e-3
    th0 = bv.theta(1.0, 0.1, 1.5, tau2)
    th, ll, ne, st = bv.mle_check(MODEL, th0, LO, HI, free_mask=bv.BV_FREE_SIGMA2 | bv.BV_FREE_RANGE,
                                  ftol_rel=1e-13, xtol=1e-8)
    assert st == 0 and th.nugget == tau2
    f = lambda x: -_ell(MODEL, np.exp(x[0]), np.exp(x[1]), tau2)
    r = minimize(f, [np.log(th.sigma2), np.log(th.range[0])], method="Nelder-Mead",
                 options=dict(xatol=1e-10, fatol=1e-12, maxiter=4000))
    assert ll >= -r.fun - 1e-9 * abs(r.fun)
    np.testing.assert_allclose([np.log(th.sigma2), np.log(th.range[0])], r.x, atol=1e-4)
