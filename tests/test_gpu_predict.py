"""GPU prediction parity (Sec. 2.4, Algorithm 2): prediction blocks and their
conditioning sets bit-exact against the oracle; conditional means, variances and block
covariances against the oracle's FP64 solves; conditional-simulation intervals and
coverage against the oracle's draws of the same counter-based generator."""
import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth
from tests import _ref

pytestmark = pytest.mark.gpu

Z95 = 1.959963984540054


@pytest.fixture(scope="module")
def bv():
    import torch
    assert torch.cuda.is_available()
    from paper_2410_04477_gb300 import bv as _bv
    return _bv


def _data(n, n_star, d, seed, s2, beta, nu, tau2, ranges=None):
    locs = synth.locs_uniform(n + n_star, d, seed)
    th = oracle.theta(s2, beta, nu, tau2, ranges)
    y_all = oracle.exact_draw(th, locs, synth.normal(seed, 20, n + n_star))
    return locs[:n], y_all[:n], locs[n:], y_all[n:], th


def _gpu(bv, lo, y, ls, yt, bc, m, th_args, seed=0, packed=False):
    with bv.Context() as ctx:
        ctx.set_data(lo, y)
        ctx.set_pred_locations(ls, yt)
        bp, pi = ctx.build_pred_blocks(bc, seed=seed)
        nnp, nni = ctx.select_pred_neighbors(m)
        mean, var, cov = ctx.predict(bv.theta(*th_args), packed_cov=packed)
        lo_b, up_b, covered = ctx.cond_sim(1000, seed=5, z_crit=Z95)
    return (bp, pi, nnp, nni), mean, var, cov, (lo_b, up_b, covered)


CASES = [  # n_obs, n_star, d, bc, m, (sigma2, beta, nu, tau2)
    (2000, 300, 2, 30, 40, (1.0, 0.1, 0.5, 1e-3)),
    (1500, 257, 2, 25, 97, (1.4, 0.05, 1.5, 1e-2)),
    (1200, 160, 3, 16, 60, (0.8, 0.2, 2.5, 1e-3)),
    (300, 90, 2, 9, 10**5, (1.2, 0.08, 1.5, 5e-3)),   # all observations: global-memory path
]


@pytest.mark.parametrize("n,ns,d,bc,m,th", CASES)
def test_prediction_matches_oracle(bv, n, ns, d, bc, m, th):
    lo, y, ls, yt, oth = _data(n, ns, d, 50 + n, *th)
    (bp, pi, nnp, nni), mean, var, cov, (lb, ub, covered) = _gpu(bv, lo, y, ls, yt, bc, m, th, seed=7, packed=True)
    obp, opi, oce = oracle.build_pred_blocks(ls, bc, seed=7)
    onnp, onni = oracle.select_pred_neighbors(lo, oce, m)
    for a, b in ((bp, obp), (pi, opi), (nnp, onnp), (nni, onni)):
        np.testing.assert_array_equal(a, b)
    omean, ovar, ocov = oracle.predict(oth, lo, y, ls, obp, opi, onnp, onni, packed_cov=True)
    scale = th[0] + th[3]
    np.testing.assert_allclose(mean, omean, rtol=1e-9, atol=1e-10 * scale)
    np.testing.assert_allclose(var, ovar, rtol=1e-9, atol=1e-10 * scale)
    np.testing.assert_allclose(cov, ocov, rtol=1e-9, atol=1e-10 * scale)
    # intervals: the GPU's from its own moments, the oracle's from the oracle's
    olb, oub, ocovered = oracle.cond_sim(omean, ovar, 1000, 5, Z95, yt)
    np.testing.assert_allclose(lb, olb, rtol=1e-9, atol=1e-9 * scale)
    np.testing.assert_allclose(ub, oub, rtol=1e-9, atol=1e-9 * scale)
    near = np.sum((np.abs(yt - olb) < 1e-8 * scale) | (np.abs(yt - oub) < 1e-8 * scale))
    assert abs(covered - ocovered) <= near, (covered, ocovered, near)


def test_lattice_ties_and_interpolation(bv):
    # new locations on observed lattice sites, zero nugget: exact interpolation; ties in
    # the neighbour ranking are broken by index on both sides
    g = np.arange(12) / 12.0
    lo = np.array([(a, b) for a in g for b in g])
    y = synth.normal(60, 1, len(lo))
    ls = lo[[5, 40, 77, 100, 143]] + 0.0
    with bv.Context() as ctx:
        ctx.set_data(lo, y)
        ctx.set_pred_locations(ls)
        bp, pi = ctx.build_pred_blocks(5, seed=1)
        nnp, nni = ctx.select_pred_neighbors(9)
        mean, var, _ = ctx.predict(bv.theta(1.0, 0.2, 0.5, 0.0))
        _, _, covered = ctx.cond_sim(100)
    obp, opi, oce = oracle.build_pred_blocks(ls, 5, seed=1)
    onnp, onni = oracle.select_pred_neighbors(lo, oce, 9)
    np.testing.assert_array_equal(nni, onni)
    np.testing.assert_allclose(mean, y[[5, 40, 77, 100, 143]], rtol=1e-9, atol=1e-12)
    assert np.all(np.abs(var) < 1e-9)
    assert covered == -1


def test_no_neighbours_is_the_prior(bv):
    lo, y, ls, yt, oth = _data(400, 64, 2, 61, 0.9, 0.07, 1.5, 2e-2)
    with bv.Context() as ctx:
        ctx.set_data(lo, y)
        ctx.set_pred_locations(ls, yt)
        bp, pi = ctx.build_pred_blocks(8, seed=2)
        ctx.select_pred_neighbors(0)
        mean, var, cov = ctx.predict(bv.theta(0.9, 0.07, 1.5, 2e-2), packed_cov=True)
    assert np.all(mean == 0.0)
    np.testing.assert_allclose(var, 0.92, rtol=1e-15)
    blk = pi[bp[0]:bp[1]]
    C = _ref.full_cov(ls[blk], 0.9, 0.07, 1.5, 2e-2)
    np.testing.assert_allclose(cov[:len(blk) * (len(blk) + 1) // 2], C[np.tril_indices(len(blk))], rtol=1e-13)


def test_picp_at_the_papers_prediction_shape(bv):
    # Sec. 3.2: n = 20,000 in the unit square, 10% held out, 200 prediction blocks,
    # 1,000 conditional-simulation rounds; data drawn from the block-Vecchia model
    # at m = 200 (close to exact); the 95% interval should cover about 95%.
    n = 20000
    locs = synth.locs_uniform(n, 2, 62)
    th = bv.theta(1.0, 0.05, 1.5, 1e-2)
    with bv.Context() as ctx:
        ctx.set_data(locs)
        ctx.build_blocks(n // 10, seed=62)
        ctx.select_neighbors(200)
        y = ctx.simulate(th, synth.normal(62, 20, n))
    hold = np.zeros(n, bool)
    hold[synth.splitmix64(synth.stream(62, 9), np.arange(n, dtype=np.uint64)) % np.uint64(10) == 0] = True
    with bv.Context() as ctx:
        ctx.set_data(locs[~hold], y[~hold])
        ctx.set_pred_locations(locs[hold], y[hold])
        ctx.build_pred_blocks(200, seed=3)
        ctx.select_pred_neighbors(120)
        mean, var, _ = ctx.predict(th)
        lo_b, up_b, covered = ctx.cond_sim(1000, seed=4)
    picp = covered / hold.sum()
    assert 0.93 <= picp <= 0.97, picp
    assert np.all(var > 0) and np.all(up_b > lo_b)
