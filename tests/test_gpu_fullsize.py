"""Full-size parity at the batched plain-FP64 configuration (n = 200,000 uniform points,
bc = 20,000 K-means blocks, m = 60, Matern nu = 1.5, beta = 0.05, nugget 1e-4), in the
benchmark's launch configuration: the oracle builds its own blocks, neighbours and draw;
the GPU builds its own; blocks and neighbour sets must agree bit for bit, every per-block
term to 1e-9 and the total to 1e-10 relative.  (A block-Vecchia draw at m = 30 supplies y:
the draw's m does not enter the evaluation's parity.)"""
import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth

pytestmark = pytest.mark.gpu


def test_config2_full_size():
    from paper_2410_04477_gb300 import bv
    n, bc, m = 200_000, 20_000, 60
    locs = synth.locs_uniform(n, 2, 1)
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=1, iters=20)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
    gnp, gni = oracle.select_neighbors(locs, bp, pi, ce, 30)
    th = oracle.theta(1.0, 0.05, 1.5, 1e-4)
    y = oracle.bv_draw(th, locs, bp, pi, gnp, gni, synth.normal(1, 20, n))
    ll_o, per_o, st = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    assert st == 0
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        gbp, gpi = ctx.build_blocks(bc, seed=1, iters=20)
        gnnp, gnni = ctx.select_neighbors(m)
        _, _, gce = ctx.blocks()
        np.testing.assert_array_equal(gbp, bp)
        np.testing.assert_array_equal(gpi, pi)
        assert gce.tobytes() == ce.tobytes()
        np.testing.assert_array_equal(gnnp, nnp)
        np.testing.assert_array_equal(gnni, nni)
        ctx.autotune(bv.BV_FP64)
        ll, per, st = ctx.loglik(bv.theta(1.0, 0.05, 1.5, 1e-4), bv.BV_FP64, per_block=True)
        llm = ctx.loglik(bv.theta(1.0, 0.05, 1.5, 1e-4), bv.BV_MIXED)
    assert abs(ll - ll_o) <= 1e-10 * abs(ll_o), (ll, ll_o)
    np.testing.assert_allclose(per, per_o, rtol=1e-9, atol=1e-9)
    print(f"config 2 full size, mixed: |dl| {abs(llm - ll_o):.3e} rel {abs(llm - ll_o) / abs(ll_o):.2e}")
    assert abs(llm - ll_o) <= 1e-6 * abs(ll_o), (llm, ll_o)
