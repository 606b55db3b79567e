"""Edge cases of the GPU path against the oracle: one-dimensional locations, a single
point, two points, one block holding everything (the global-memory kernel; exact by
Eq. 1), strongly ragged block sizes from clustered locations, and a multi-dataset
context with a tiny dataset."""
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


def _run(bv, locs, y, bc, m, th, seed=0):
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        bp, pi = ctx.build_blocks(bc, seed=seed)
        nnp, nni = ctx.select_neighbors(m)
        ll = ctx.loglik(bv.theta(*th))
        llm = ctx.loglik(bv.theta(*th), bv.BV_MIXED)
    obp, opi, oce = oracle.build_blocks(locs, bc, seed=seed)
    onnp, onni = oracle.select_neighbors(locs, obp, opi, oce, m)
    for a, b in ((bp, obp), (pi, opi), (nnp, onnp), (nni, onni)):
        np.testing.assert_array_equal(a, b)
    lo = oracle.loglik(oracle.theta(*th), locs, y, obp, opi, onnp, onni)[0]
    return ll, llm, lo


def test_one_dimensional_locations(bv):
    n = 1000
    locs = synth.locs_uniform(n, 1, 120)
    th = (1.2, 0.05, 1.5, 1e-3)
    y = oracle.exact_draw(oracle.theta(*th), locs, synth.normal(120, 20, n))
    ll, llm, lo = _run(bv, locs, y, 100, 20, th)
    assert abs(ll - lo) <= 1e-10 * abs(lo)
    assert abs(llm - lo) <= 1e-6 * abs(lo), (llm, lo, abs(llm - lo))


@pytest.mark.parametrize("n,bc,m", [(1, 1, 5), (2, 2, 1), (3, 1, 0), (5, 5, 10)])
def test_tiny_problems(bv, n, bc, m):
    locs = synth.locs_uniform(n, 2, 121 + n)
    th = (0.9, 0.2, 0.5, 1e-2)
    y = synth.normal(121 + n, 20, n)
    ll, llm, lo = _run(bv, locs, y, bc, m, th)
    assert abs(ll - lo) <= 1e-12 * max(1.0, abs(lo))
    assert abs(llm - lo) <= 1e-6 * max(1.0, abs(lo)), (llm, lo, abs(llm - lo))
    if n == 1:
        v = 0.9 + 1e-2
        assert lo == pytest.approx(-0.5 * (np.log(2 * np.pi * v) + y[0] ** 2 / v), rel=1e-13)


def test_single_block_is_exact_through_the_global_kernel(bv):
    n = 400                                   # N = 400: above both shared-memory limits
    locs = synth.locs_uniform(n, 2, 122)
    th = (1.0, 0.1, 2.5, 1e-2)
    y = oracle.exact_draw(oracle.theta(*th), locs, synth.normal(122, 20, n))
    ll, llm, lo = _run(bv, locs, y, 1, 0, th)
    exact = oracle.exact_loglik(oracle.theta(*th), locs, y)
    assert abs(lo - exact) <= 1e-10 * abs(exact)
    assert abs(ll - exact) <= 1e-10 * abs(exact)
    assert abs(llm - exact) <= 1e-6 * abs(exact)


def test_ragged_blocks_from_clustered_locations(bv):
    # three tight clusters and a sparse background: K-means blocks of very uneven sizes
    rng_u = synth.uniform01(123, 1, 2 * 1800).reshape(1800, 2)
    centres = np.array([[0.2, 0.3], [0.7, 0.8], [0.5, 0.1]])
    locs = rng_u.copy()
    for k in range(3):
        locs[400 * k:400 * (k + 1)] = centres[k] + 0.01 * (rng_u[400 * k:400 * (k + 1)] - 0.5)
    th = (1.0, 0.05, 1.5, 1e-2)
    y = synth.normal(123, 20, len(locs))
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        bp, _ = ctx.build_blocks(60, seed=4)
    sizes = np.diff(bp)
    assert sizes.max() >= 8 * np.median(sizes)
    ll, llm, lo = _run(bv, locs, y, 60, 120, th, seed=4)
    assert abs(ll - lo) <= 1e-10 * abs(lo)
    assert abs(llm - lo) <= 1e-6 * abs(lo), (llm, lo, abs(llm - lo))


def test_multi_dataset_with_a_tiny_dataset(bv):
    sizes = [900, 3, 1500]
    locs = [synth.locs_uniform(n, 2, 130 + k) for k, n in enumerate(sizes)]
    ths = [(1.0, 0.1, 0.5, 1e-2), (2.0, 0.3, 1.5, 1e-1), (0.7, 0.05, 2.5, 1e-3)]
    ys = [synth.normal(130 + k, 20, n) for k, n in enumerate(sizes)]
    bcs = [90, 1, 150]
    with bv.Context() as ctx:
        ctx.set_datasets(locs, ys)
        ctx.build_blocks_multi(bcs, seed=7)
        ctx.select_neighbors(25)
        out = ctx.loglik_multi([bv.theta(*t) for t in ths])
    for k in range(3):
        bp, pi, ce = oracle.build_blocks(locs[k], bcs[k], seed=7 + k)
        nnp, nni = oracle.select_neighbors(locs[k], bp, pi, ce, 25)
        lo = oracle.loglik(oracle.theta(*ths[k]), locs[k], ys[k], bp, pi, nnp, nni)[0]
        assert abs(out[k] - lo) <= 1e-10 * max(1.0, abs(lo)), (k, out[k], lo)
