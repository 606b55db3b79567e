"""General smoothness nu (Eq. 5 with any nu > 0): the device's K_nu-based Matern against
SciPy's Bessel function, and the log-likelihood, exact likelihood, sampler and
prediction at non-half-integer nu against the oracle (whose K_nu is an independent
quadrature)."""
import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth
from tests import _ref

pytestmark = pytest.mark.gpu

NUS = [0.2, 0.3, 0.5, 0.77, 1.0, 1.2, 1.5, 2.0, 2.5, 3.3, 5.0, 7.2, 12.5]


@pytest.fixture(scope="module")
def bv():
    import torch
    assert torch.cuda.is_available()
    from paper_2410_04477_gb300 import bv as _bv
    return _bv


@pytest.mark.parametrize("nu", NUS)
def test_device_matern_matches_scipy(bv, nu):
    x = np.concatenate([[0.0], np.logspace(-8, np.log10(60.0), 400), [1.999999, 2.0, 2.000001]])
    got = bv.matern_check(nu, x)
    want = _ref.matern_kv(nu, x)
    np.testing.assert_allclose(got, want, rtol=2e-13, atol=1e-300)
    # the per-evaluation octave table of the log-likelihood kernels, out to 600
    xt = np.concatenate([x, np.logspace(np.log10(60.0), np.log10(600.0), 50), [1e-13, 2.0 ** -40, 511.9, 512.0]])
    tab = bv.matern_check(nu, xt, tabulated=True)
    np.testing.assert_allclose(tab, _ref.matern_kv(nu, xt), rtol=5e-13, atol=1e-300)


@pytest.mark.parametrize("nu,beta,tau2", [(0.3, 0.1, 1e-3), (0.8, 0.08, 1e-4), (1.2, 0.05, 1e-3),
                                          (2.0, 0.04, 1e-2), (3.7, 0.03, 1e-2)])
def test_loglik_general_nu_matches_oracle(bv, nu, beta, tau2):
    n = 1500
    locs = synth.locs_uniform(n, 2, 100)
    th = oracle.theta(1.1, beta, nu, tau2)
    y = oracle.exact_draw(th, locs, synth.normal(100, 20, n))
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        bp, pi = ctx.build_blocks(150, seed=1)
        nnp, nni = ctx.select_neighbors(40)
        ll, per, _ = ctx.loglik(bv.theta(1.1, beta, nu, tau2), per_block=True)
        llm = ctx.loglik(bv.theta(1.1, beta, nu, tau2), bv.BV_MIXED)
        ll_half = ctx.loglik(bv.theta(1.1, beta, 1.5, tau2))     # switch back to a closed form
        lx, _, _ = ctx.exact_loglik(bv.theta(1.1, beta, nu, tau2))
    ll_o, per_o, _ = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    assert abs(ll - ll_o) <= 1e-10 * abs(ll_o), (ll, ll_o)
    np.testing.assert_allclose(per, per_o, rtol=1e-9, atol=1e-9)
    assert abs(llm - ll_o) <= 1e-6 * abs(ll_o), (llm, ll_o, abs(llm - ll_o))
    assert ll_half == pytest.approx(oracle.loglik(oracle.theta(1.1, beta, 1.5, tau2), locs, y, bp, pi, nnp, nni)[0],
                                    rel=1e-10)
    want_x = oracle.exact_loglik(th, locs, y)
    assert abs(lx - want_x) <= 1e-10 * abs(want_x)


def test_sampler_and_prediction_general_nu(bv):
    n = 1200
    locs = synth.locs_uniform(n + 100, 2, 101)
    lo, ls = locs[:n], locs[n:]
    th = oracle.theta(0.9, 0.07, 1.3, 1e-2)
    z = synth.normal(101, 20, n)
    with bv.Context() as ctx:
        ctx.set_data(lo)
        bp, pi = ctx.build_blocks(120, seed=2)
        nnp, nni = ctx.select_neighbors(30)
        y = ctx.simulate(bv.theta(0.9, 0.07, 1.3, 1e-2), z)
        ctx.set_pred_locations(ls)
        pbp, ppi = ctx.build_pred_blocks(10, seed=3)
        ctx.select_pred_neighbors(50)
        mean, var, _ = ctx.predict(bv.theta(0.9, 0.07, 1.3, 1e-2))
    y_o = oracle.bv_draw(th, lo, bp, pi, nnp, nni, z)
    np.testing.assert_allclose(y, y_o, rtol=1e-9, atol=1e-9)
    obp, opi, oce = oracle.build_pred_blocks(ls, 10, seed=3)
    onnp, onni = oracle.select_pred_neighbors(lo, oce, 50)
    om, ov, _ = oracle.predict(th, lo, y_o, ls, obp, opi, onnp, onni)
    np.testing.assert_allclose(mean, om, rtol=1e-8, atol=1e-9)
    np.testing.assert_allclose(var, ov, rtol=1e-8, atol=1e-10)
