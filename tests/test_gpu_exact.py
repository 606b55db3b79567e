"""GPU exact log-likelihood (Eq. 1, dense tiled Cholesky) and the KL divergence of the
block-Vecchia approximation (Eq. 7) against the FP64 oracle."""
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


@pytest.mark.parametrize("n,d,nu,tau2", [(500, 2, 0.5, 1e-3), (639, 2, 1.5, 1e-2), (1000, 3, 2.5, 1e-2),
                                          (63, 2, 1.5, 1e-3), (1, 2, 0.5, 0.0)])
def test_exact_loglik_matches_oracle(bv, n, d, nu, tau2):
    locs = synth.locs_uniform(n, d, 90 + n)
    th = oracle.theta(1.2, 0.1, nu, tau2)
    y = oracle.exact_draw(th, locs, synth.normal(90 + n, 20, n)) if n > 1 else np.array([0.7])
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        ll, q, ld = ctx.exact_loglik(bv.theta(1.2, 0.1, nu, tau2))
        l0, q0, ld0 = ctx.exact_loglik(bv.theta(1.2, 0.1, nu, tau2), use_y=False)
    want = oracle.exact_loglik(th, locs, y)
    assert abs(ll - want) <= 1e-10 * max(1.0, abs(want)), (ll, want)
    assert q0 == 0.0 and ld0 == ld
    w0 = oracle.exact_loglik(th, locs, np.zeros(n))
    assert abs(l0 - w0) <= 1e-10 * max(1.0, abs(w0))


def test_kl_divergence_matches_oracle(bv):
    n = 1200
    locs = synth.locs_uniform(n, 2, 91)
    th = oracle.theta(1.0, 0.052537, 1.5, 1e-4)
    zero = np.zeros(n)
    l0 = oracle.exact_loglik(th, locs, zero)
    for m, order in ((10, "random"), (30, "maxmin"), (30, "hilbert"), (10**5, "random")):
        with bv.Context() as ctx:
            ctx.set_data(locs)
            ctx.build_blocks(120, seed=5)
            ctx.order_blocks(order, seed=6)
            ctx.select_neighbors(m)
            kl, d0, da = ctx.kl_divergence(bv.theta(1.0, 0.052537, 1.5, 1e-4))
        bp, pi, ce = oracle.build_blocks(locs, 120, seed=5)
        bp, pi, ce = oracle.apply_block_order(bp, pi, ce, oracle.order_blocks(ce, order, seed=6))
        nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
        la = oracle.loglik(th, locs, zero, bp, pi, nnp, nni)[0]
        want = l0 - la
        assert abs(kl - want) <= 1e-9 * abs(l0), (m, order, kl, want)
        assert kl >= -1e-9 * abs(l0)
        if m >= n:
            assert abs(kl) <= 1e-9 * abs(l0)


def test_exact_not_positive_definite(bv):
    locs = synth.locs_uniform(200, 2, 92)
    locs[7] = locs[3]
    with bv.Context() as ctx:
        ctx.set_data(locs, np.ones(200))
        with pytest.raises(bv.BVError):
            ctx.exact_loglik(bv.theta(1.0, 0.1, 0.5, 0.0))
