"""Pins for the oracle's block-Vecchia prediction (Sec. 2.4, Algorithm 2) and its
univariate conditional simulation (Sec. 2.4; PICP, Sec. 3.2).

Each check compares the oracle with something the mathematics fixes, computed by a
different route: dense kriging by library solves, SciPy's Gaussian density, brute-force
neighbour ranking, and the normal distribution's CDF."""
import math

import numpy as np
import pytest
from scipy import stats

import oracle
from paper_2410_04477_gb300 import synth
from tests import _ref


def _split(n=700, n_star=120, seed=40, d=2):
    locs = synth.locs_uniform(n + n_star, d, seed)
    return locs[:n], locs[n:]


def _draw(locs_all, s2, beta, nu, tau2, seed):
    S = _ref.full_cov(locs_all, s2, beta, nu, tau2)
    return np.linalg.cholesky(S) @ synth.normal(seed, 21, len(locs_all)), S


def test_pred_blocks_partition_and_centroids():
    _, ls = _split(n_star=300)
    bp, pi, ce = oracle.build_pred_blocks(ls, 30, seed=3)
    assert bp[0] == 0 and bp[-1] == len(ls) and np.all(np.diff(bp) > 0)
    assert np.array_equal(np.sort(pi), np.arange(len(ls)))
    label, _ = oracle.kmeans(ls, 30, seed=3)
    groups = [np.flatnonzero(label == c) for c in range(30) if np.any(label == c)]
    for i, g in enumerate(groups):                      # cluster-index order, members ascending
        np.testing.assert_array_equal(pi[bp[i]:bp[i + 1]], g)
        np.testing.assert_allclose(ce[i], ls[g].mean(axis=0), rtol=0, atol=1e-12)


def test_pred_neighbors_brute_force():
    lo, ls = _split()
    bp, pi, ce = oracle.build_pred_blocks(ls, 12, seed=4)
    for m in (0, 1, 17, 10**6):
        nnp, nni = oracle.select_pred_neighbors(lo, ce, m)
        mi = min(m, len(lo))
        assert np.array_equal(np.diff(nnp), np.full(len(ce), mi))
        for i, c in enumerate(ce):
            d2 = ((lo - c) ** 2).sum(axis=1)
            want = np.lexsort((np.arange(len(lo)), d2))[:mi]
            np.testing.assert_array_equal(nni[nnp[i]:nnp[i + 1]], want)


@pytest.mark.parametrize("nu,tau2", [(0.5, 1e-3), (1.5, 1e-2), (2.5, 0.0)])
def test_all_observations_is_exact_kriging(nu, tau2):
    # With every observation in the conditioning set, each block's conditional law is the
    # exact GP conditional of y_* given y: mean Sigma_*y Sigma_yy^-1 y, covariance
    # Sigma_** - Sigma_*y Sigma_yy^-1 Sigma_y*.
    lo, ls = _split(n=400, n_star=60, seed=41)
    n = len(lo)
    y_all, S = _draw(np.vstack([lo, ls]), 1.3, 0.1, nu, tau2 + 1e-8, 41)
    S = _ref.full_cov(np.vstack([lo, ls]), 1.3, 0.1, nu, tau2)
    y = y_all[:n]
    th = oracle.theta(1.3, 0.1, nu, tau2)
    bp, pi, ce = oracle.build_pred_blocks(ls, 8, seed=5)
    nnp, nni = oracle.select_pred_neighbors(lo, ce, 10**6)
    mean, var, packed = oracle.predict(th, lo, y, ls, bp, pi, nnp, nni, packed_cov=True)
    Syy, Sxy, Sxx = S[:n, :n], S[n:, :n], S[n:, n:]
    km = Sxy @ np.linalg.solve(Syy, y)
    kc = Sxx - Sxy @ np.linalg.solve(Syy, Sxy.T)
    np.testing.assert_allclose(mean, km, rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(var, np.diag(kc), rtol=1e-8, atol=1e-10)
    off = 0
    for i in range(len(bp) - 1):
        blk = pi[bp[i]:bp[i + 1]]
        b = len(blk)
        C = np.zeros((b, b))
        C[np.tril_indices(b)] = packed[off:off + b * (b + 1) // 2]
        C = C + np.tril(C, -1).T
        np.testing.assert_allclose(C, kc[np.ix_(blk, blk)], rtol=1e-8, atol=1e-10)
        off += b * (b + 1) // 2


def test_no_neighbours_is_the_prior():
    lo, ls = _split(n=200, n_star=50, seed=42)
    y = synth.normal(42, 22, len(lo))
    th = oracle.theta(0.9, 0.07, 1.5, 2e-2)
    bp, pi, ce = oracle.build_pred_blocks(ls, 5, seed=6)
    nnp, nni = oracle.select_pred_neighbors(lo, ce, 0)
    mean, var, packed = oracle.predict(th, lo, y, ls, bp, pi, nnp, nni, packed_cov=True)
    assert np.all(mean == 0.0)
    np.testing.assert_allclose(var, np.full(len(ls), 0.9 + 2e-2), rtol=1e-15)
    blk = pi[bp[0]:bp[1]]
    C = _ref.full_cov(ls[blk], 0.9, 0.07, 1.5, 2e-2)
    np.testing.assert_allclose(packed[:len(blk) * (len(blk) + 1) // 2], C[np.tril_indices(len(blk))],
                               rtol=1e-12)


def test_interpolates_observations_without_nugget():
    lo, _ = _split(n=300, n_star=1, seed=43)
    ls = lo[[5, 77, 150]].copy()
    y = synth.normal(43, 23, len(lo))
    th = oracle.theta(1.0, 0.05, 0.5, 0.0)
    bp, pi, ce = oracle.build_pred_blocks(ls, 3, seed=7)
    nnp, nni = oracle.select_pred_neighbors(lo, ls[pi], 30)   # conditioning sets contain the site
    mean, var, _ = oracle.predict(th, lo, y, ls, bp, pi, nnp, nni)
    np.testing.assert_allclose(mean, y[[5, 77, 150]], rtol=1e-9, atol=1e-12)
    assert np.all(np.abs(var) <= 1e-9)


def test_conditional_law_is_the_block_likelihood():
    # Algorithm 2's conditional law of a block is the one Algorithm 1 scores: the density
    # of y_B under N(mu, Sigma_B) equals the block's conditional log-likelihood.
    n = 500
    locs = synth.locs_uniform(n, 2, 44)
    th = oracle.theta(1.1, 0.08, 1.5, 1e-2)
    y = oracle.exact_draw(th, locs, synth.normal(44, 20, n))
    bp, pi, ce = oracle.build_blocks(locs, 50, seed=44)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 25)
    for i in (0, 7, 31, 49):
        blk, nn = pi[bp[i]:bp[i + 1]], nni[nnp[i]:nnp[i + 1]]
        mu, C = oracle.predict_block(th, locs, y, nn, locs, blk)
        ell, st = oracle.block_loglik(th, locs, y, nn, blk)
        assert st == 0
        assert ell == pytest.approx(stats.multivariate_normal(mu, C).logpdf(y[blk]), rel=1e-10, abs=1e-10)


def test_csim_normals_are_standard_normal():
    # 60 locations x 1,001 draws (an odd count: the last pair's second normal is dropped)
    z = np.array([oracle.csim_normal(9, j, 1001, r) for j in range(60) for r in range(1001)])
    assert stats.kstest(z, "norm").pvalue > 1e-3
    assert abs(z.mean()) < 4 / np.sqrt(len(z))
    assert abs(z.var() - 1.0) < 4 * np.sqrt(2.0 / len(z))
    # the two normals of a pair are independent: their correlation is within noise, and
    # the pair's squared radius is exponential with mean 2 (chi-square with 2 dof)
    a = np.array([oracle.csim_normal(9, j, 1000, 2 * k) for j in range(20) for k in range(500)])
    b = np.array([oracle.csim_normal(9, j, 1000, 2 * k + 1) for j in range(20) for k in range(500)])
    assert abs(np.corrcoef(a, b)[0, 1]) < 4 / np.sqrt(len(a))
    assert stats.kstest(a * a + b * b, "expon", args=(0, 2)).pvalue > 1e-3
    assert oracle.csim_normal(9, 0, 10, 5) != oracle.csim_normal(10, 0, 10, 5)
    assert oracle.csim_normal(9, 1, 10, 0) != oracle.csim_normal(9, 0, 10, 0)


def csim_normal_rule(seed, j, rounds, r):
    """Normal r of new location j written out from its stated rule: pair k = r // 2 of
    location j takes SplitMix64 draws 2c and 2c + 1 of the stream seed ^ "condsim_", with
    c = j ceil(R / 2) + k; u1 = 1 - (x >> 11) 2^-53, u2 = (x' >> 11) 2^-53; the even member
    is sqrt(-2 ln u1) cos(2 pi u2), the odd one the same with sin."""
    stream = seed ^ 0x636F6E6473696D5F          # the ASCII bytes of "condsim_"
    c = j * ((rounds + 1) // 2) + r // 2
    u1 = 1.0 - (oracle.splitmix64(stream, 2 * c) >> 11) * 2.0 ** -53
    u2 = (oracle.splitmix64(stream, 2 * c + 1) >> 11) * 2.0 ** -53
    rho = math.sqrt(-2.0 * math.log(u1))
    return rho * (math.cos(2.0 * math.pi * u2) if r % 2 == 0 else math.sin(2.0 * math.pi * u2))


@pytest.mark.parametrize("rounds", [1000, 1001, 2])
def test_csim_normal_follows_its_stated_rule(rounds):
    # every draw of the first and of a later location, and the location offsets: draws
    # of different locations never share a pair
    for seed, j in ((9, 0), (9, 1), (12345, 777)):
        for r in list(range(min(rounds, 40))) + [rounds - 2, rounds - 1]:
            want = csim_normal_rule(seed, j, rounds, r)
            assert oracle.csim_normal(seed, j, rounds, r) == pytest.approx(want, rel=1e-14, abs=1e-15)


def test_cond_sim_interval_and_coverage():
    rng_mean = synth.normal(45, 1, 20000)
    sd = np.exp(synth.uniform01(45, 2, 20000) - 0.5)
    truth = rng_mean + sd * synth.normal(45, 3, 20000)       # held-out values from the same law
    R = 1000
    lo, up, covered = oracle.cond_sim(rng_mean, sd ** 2, R, 11, 1.959963984540054, truth)
    mid, half = 0.5 * (lo + up), 0.5 * (up - lo)
    # sample mean within 5 standard errors; sample sd within 5 standard errors of sd
    assert np.all(np.abs(mid - rng_mean) <= 5 * sd / np.sqrt(R))
    assert np.all(np.abs(half / 1.959963984540054 - sd) <= 5 * sd / np.sqrt(2 * (R - 1)))
    picp = covered / 20000
    assert abs(picp - 0.95) < 4 * np.sqrt(0.95 * 0.05 / 20000) + 0.003
    assert covered == int(np.sum((truth >= lo) & (truth <= up)))
    # zero variance: the interval collapses onto the mean
    lo0, up0, _ = oracle.cond_sim(rng_mean[:10], np.zeros(10), 50, 1, 1.96)
    np.testing.assert_allclose(lo0, rng_mean[:10], rtol=1e-14)
    np.testing.assert_allclose(up0, rng_mean[:10], rtol=1e-14)
