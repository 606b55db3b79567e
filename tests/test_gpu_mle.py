"""GPU maximum likelihood (Sec. 3.2) and the two terms of ell it profiles with: the
quadratic form against the oracle, the returned ell against the oracle at the returned
theta, the closed-form sigma^2 = Q / n, and local optimality of the estimate."""
import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bv():
    import torch
    assert torch.cuda.is_available()
    from paper_2410_04477_gb300 import bv as _bv
    return _bv


def _problem(n=3000, nu=1.5, s2=1.4, beta=0.06, tau2=5e-3, seed=31, bc=300, m=40):
    locs = synth.locs_uniform(n, 2, seed)
    y = oracle.exact_draw(oracle.theta(s2, beta, nu, tau2), locs, synth.normal(seed, 20, n))
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=seed, iters=20)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
    return locs, y, (bp, pi, nnp, nni), bc, m, seed


def _ctx(bv, locs, y, bc, m, seed, ostruct):
    ctx = bv.Context()
    ctx.set_data(locs, y)
    g = ctx.build_blocks(bc, seed=seed, iters=20) + ctx.select_neighbors(m)
    for a, b in zip(g, ostruct):
        np.testing.assert_array_equal(a, b)
    return ctx


def _oracle_ell(th, locs, y, st):
    return oracle.loglik(oracle.theta(th.sigma2, th.range[0], th.nu, th.nugget), locs, y, *st)[0]


def test_loglik_terms_match_oracle(bv):
    locs, y, st, bc, m, seed = _problem()
    n = len(y)
    with _ctx(bv, locs, y, bc, m, seed, st) as ctx:
        th = bv.theta(1.1, 0.05, 1.5, 4e-3)
        ll, Q, D = ctx.loglik_terms(th)
        assert ll == ctx.loglik(th)
    l1 = oracle.loglik(oracle.theta(1.1, 0.05, 1.5, 4e-3), locs, y, *st)[0]
    l2 = oracle.loglik(oracle.theta(2.2, 0.05, 1.5, 8e-3), locs, y, *st)[0]
    Q_o = 2.0 * (n * np.log(2.0) - 2.0 * (l1 - l2))   # l1 - l2 = -(Q - Q/2 - n log 2) / 2
    assert abs(ll - l1) <= 1e-10 * abs(l1)
    assert abs(Q - Q_o) <= 1e-8 * Q_o, (Q, Q_o)
    assert ll == pytest.approx(-0.5 * (Q + D + n * np.log(2 * np.pi)), rel=1e-13)


@pytest.mark.parametrize("newton_first", [True, False])
@pytest.mark.parametrize("prec_name", ["BV_FP64", "BV_MIXED"])
def test_profile_mle_is_a_stationary_maximum(bv, prec_name, newton_first):
    # both search orders: trust-region Newton first (the default) and the simplex first
    locs, y, st, bc, m, seed = _problem()
    n = len(y)
    nu = 1.5
    lo, hi = bv.theta(0.01, 0.001, nu, 1e-6), bv.theta(100.0, 3.0, nu, 10.0)
    with _ctx(bv, locs, y, bc, m, seed, st) as ctx:
        th, ll, ne = ctx.mle(bv.theta(1.0, 0.1, nu, 1e-2), lo, hi, precision=getattr(bv, prec_name),
                             ftol_rel=1e-13, xtol=1e-7, newton_first=newton_first)
        print(f"{prec_name} newton_first={newton_first}: {ne} evaluations")
        assert 0 < ne < 2000
        # the returned ell is the FP64 ell at the returned theta
        assert ll == pytest.approx(ctx.loglik(th), rel=1e-11)
        # sigma^2 is the closed-form profile maximiser Q / n at (beta, tau^2 / sigma^2)
        _, Q1, _ = ctx.loglik_terms(bv.theta(1.0, th.range[0], nu, th.nugget / th.sigma2))
        assert th.sigma2 == pytest.approx(Q1 / n, rel=1e-12)
        # a small move of any log-parameter lowers ell
        for k in range(3):
            for sgn in (-1, 1):
                v = [th.sigma2, th.range[0], th.nugget]
                v[k] *= np.exp(sgn * 1e-3)
                assert ctx.loglik(bv.theta(v[0], v[1], nu, v[2])) < ll
    assert abs(ll - _oracle_ell(th, locs, y, st)) <= 1e-10 * abs(ll)


def test_profile_mle_paths_without_a_free_nugget(bv):
    locs, y, st, bc, m, seed = _problem(tau2=0.0, nu=0.5, beta=0.1, n=2000, bc=200, m=30, seed=32)
    n = len(y)
    nu = 0.5
    lo, hi = bv.theta(0.01, 0.001, nu, 1e-6), bv.theta(100.0, 3.0, nu, 10.0)
    with _ctx(bv, locs, y, bc, m, seed, st) as ctx:
        # sigma^2 alone, nugget zero: closed form, one evaluation
        th, ll, ne = ctx.mle(bv.theta(1.0, 0.1, nu, 0.0), lo, hi, free_mask=bv.BV_FREE_SIGMA2)
        assert ne == 1
        _, Q1, _ = ctx.loglik_terms(bv.theta(1.0, 0.1, nu, 0.0))
        assert th.sigma2 == pytest.approx(Q1 / n, rel=1e-14) and th.range[0] == 0.1 and th.nugget == 0.0
        assert ll == pytest.approx(ctx.loglik(th), rel=1e-11)
        # sigma^2 and range, nugget zero: a one-dimensional search
        th, ll, ne = ctx.mle(bv.theta(1.0, 0.2, nu, 0.0), lo, hi,
                             free_mask=bv.BV_FREE_SIGMA2 | bv.BV_FREE_RANGE, ftol_rel=1e-13, xtol=1e-7)
        assert th.nugget == 0.0
        for k in range(2):
            for sgn in (-1, 1):
                v = [th.sigma2, th.range[0]]
                v[k] *= np.exp(sgn * 1e-3)
                assert ctx.loglik(bv.theta(v[0], v[1], nu, 0.0)) < ll
        # nugget fixed away from zero: no profiling, the direct search over sigma^2 and beta
        th2, ll2, _ = ctx.mle(bv.theta(1.0, 0.2, nu, 1e-3), lo, hi,
                              free_mask=bv.BV_FREE_SIGMA2 | bv.BV_FREE_RANGE, ftol_rel=1e-13, xtol=1e-7)
        assert th2.nugget == 1e-3
        for k in range(2):
            for sgn in (-1, 1):
                v = [th2.sigma2, th2.range[0]]
                v[k] *= np.exp(sgn * 1e-3)
                assert ctx.loglik(bv.theta(v[0], v[1], nu, 1e-3)) < ll2
    assert abs(ll - _oracle_ell(th, locs, y, st)) <= 1e-10 * abs(ll)


def test_profile_respects_the_box(bv):
    # an upper bound on sigma^2 below Q / n: the estimate sits on the bound
    locs, y, st, bc, m, seed = _problem(n=2000, bc=200, m=30, seed=33)
    nu = 1.5
    with _ctx(bv, locs, y, bc, m, seed, st) as ctx:
        lo, hi = bv.theta(0.01, 0.001, nu, 1e-6), bv.theta(0.5, 3.0, nu, 10.0)
        th, ll, _ = ctx.mle(bv.theta(0.3, 0.1, nu, 1e-2), lo, hi, ftol_rel=1e-12, xtol=1e-7)
        assert th.sigma2 <= 0.5 * (1 + 1e-12)
        assert 1e-6 * (1 - 1e-12) <= th.nugget <= 10.0 * (1 + 1e-12)
        assert 0.001 <= th.range[0] <= 3.0
        assert ll == pytest.approx(ctx.loglik(th), rel=1e-11)


def test_mle_with_all_earlier_points_is_the_exact_mle(bv):
    # With m >= n every conditioning set holds all earlier points, so the block-Vecchia
    # likelihood is the exact one (Eq. 2-3) and its maximiser is the exact MLE; here that
    # is found independently by SciPy's Nelder-Mead on the oracle's Eq. 1.
    from scipy.optimize import minimize
    n, nu = 400, 1.5
    locs = synth.locs_uniform(n, 2, 34)
    y = oracle.exact_draw(oracle.theta(1.2, 0.08, nu, 2e-2), locs, synth.normal(34, 20, n))

    def negll(x):
        return -oracle.exact_loglik(oracle.theta(*np.exp(x[:2]), nu, np.exp(x[2])), locs, y)

    r = minimize(negll, np.log([1.0, 0.1, 1e-2]), method="Nelder-Mead",
                 options=dict(xatol=1e-9, fatol=1e-12, maxiter=4000, maxfev=4000))
    r = minimize(negll, r.x, method="Nelder-Mead", options=dict(xatol=1e-10, fatol=1e-13, maxfev=4000))
    lo, hi = bv.theta(0.01, 0.001, nu, 1e-6), bv.theta(100.0, 3.0, nu, 10.0)
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        ctx.build_blocks(40, seed=34)
        ctx.select_neighbors(10**5)
        th, ll, _ = ctx.mle(bv.theta(1.0, 0.1, nu, 1e-2), lo, hi, ftol_rel=1e-13, xtol=1e-8)
    assert abs(ll + r.fun) <= 1e-10 * abs(r.fun), (ll, -r.fun)
    np.testing.assert_allclose([np.log(th.sigma2), np.log(th.range[0]), np.log(th.nugget)], r.x, atol=2e-3)


def test_mle_with_free_smoothness(bv):
    # nu free (Sec. 3.2 estimates it): a stationary maximum in all four log-parameters,
    # at least as high as the maximum with nu held at its true value
    locs, y, st, bc, m, seed = _problem(n=4000, nu=1.2, s2=1.1, beta=0.06, tau2=5e-3, seed=35, bc=400, m=40)
    lo, hi = bv.theta(0.01, 0.001, 0.2, 1e-6), bv.theta(100.0, 3.0, 5.0, 10.0)
    free = bv.BV_FREE_SIGMA2 | bv.BV_FREE_RANGE | bv.BV_FREE_NUGGET | bv.BV_FREE_NU
    with _ctx(bv, locs, y, bc, m, seed, st) as ctx:
        th, ll, ne = ctx.mle(bv.theta(1.0, 0.1, 0.8, 1e-2), lo, hi, free_mask=free, ftol_rel=1e-13, xtol=1e-7)
        _, ll_fix, _ = ctx.mle(bv.theta(1.0, 0.1, 1.2, 1e-2), lo, hi, ftol_rel=1e-13, xtol=1e-7)
        assert ll >= ll_fix - 1e-9 * abs(ll)
        assert abs(th.nu - 1.2) < 0.3, th.nu
        assert ll == pytest.approx(ctx.loglik(th), rel=1e-11)
        for k in range(4):
            for sgn in (-1, 1):
                v = [th.sigma2, th.range[0], th.nugget, th.nu]
                v[k] *= np.exp(sgn * 1e-3)
                assert ctx.loglik(bv.theta(v[0], v[1], v[3], v[2])) < ll
    assert abs(ll - _oracle_ell(th, locs, y, st)) <= 1e-10 * abs(ll)


def test_batched_mle_over_datasets(bv):
    # several datasets, one context: every dataset's search issues its evaluations into
    # shared batched launches; each result matches the same dataset fitted alone
    sizes = [1500, 2200, 1800, 2600, 1200, 2000]
    truths = [(1.2, 0.05, 1e-3), (0.8, 0.08, 5e-3), (1.5, 0.04, 2e-3), (1.0, 0.06, 1e-2), (0.6, 0.1, 3e-3),
              (1.3, 0.07, 4e-3)]
    nu = 1.5
    locs, ys = [], []
    for k, (n, (s2, beta, tau2)) in enumerate(zip(sizes, truths)):
        l = synth.locs_uniform(n, 2, 400 + k)
        locs.append(l)
        ys.append(oracle.exact_draw(oracle.theta(s2, beta, nu, tau2), l, synth.normal(400 + k, 20, n)))
    lo, hi = bv.theta(0.01, 0.001, nu, 1e-6), bv.theta(100.0, 3.0, nu, 10.0)
    starts = [bv.theta(1.0, 0.1, nu, 1e-2)] * len(sizes)
    with bv.Context() as ctx:
        ctx.set_datasets(locs, ys)
        ctx.build_blocks_multi([n // 10 for n in sizes], seed=500)
        ctx.select_neighbors(30)
        ths, lls, nes, sts, nb = ctx.mle_multi(starts, lo, hi, ftol_rel=1e-13, xtol=1e-7)
    assert np.all(sts == 0) and nb < nes.sum()
    for k, n in enumerate(sizes):
        with bv.Context() as ctx:
            ctx.set_data(locs[k], ys[k])
            ctx.build_blocks(n // 10, seed=500 + k)
            ctx.select_neighbors(30)
            th, ll, _ = ctx.mle(starts[k], lo, hi, ftol_rel=1e-13, xtol=1e-7)
            assert ctx.loglik(ths[k]) == pytest.approx(lls[k], rel=1e-11)
        assert abs(lls[k] - ll) <= 1e-9 * abs(ll), (k, lls[k], ll)
