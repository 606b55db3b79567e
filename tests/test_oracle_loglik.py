"""Pins for the oracle's block-Vecchia log-likelihood (Eq. 1-4, Algorithm 1) and draws.

Each check compares the oracle with something the paper and the mathematics fix,
computed by a different route (dense matrices, library solves, SciPy's Bessel K_nu)."""
import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth
from tests import _ref


def _setup(n=300, d=2, bc=30, m=20, seed=0, nu=1.5, beta=0.1, sigma2=1.3, nugget=1e-2,
           ranges=None):
    locs = synth.locs_uniform(n, d, seed)
    th = oracle.theta(sigma2, beta, nu, nugget, ranges)
    S = _ref.full_cov(locs, sigma2, beta, nu, nugget, ranges)
    z = synth.normal(seed, 20, n)
    y = np.linalg.cholesky(S) @ z
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=seed + 1)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
    return locs, th, S, y, (bp, pi, nnp, nni)


def test_one_block_is_exact_eq1():
    locs, th, S, y, _ = _setup(n=250)
    bp = np.array([0, len(y)])
    pi = np.arange(len(y), dtype=np.int32)
    ll, per, st = oracle.loglik(th, locs, y, bp, pi, np.array([0, 0]), np.zeros(0, np.int32))
    assert st == 0
    assert ll == pytest.approx(_ref.exact_loglik(S, y), rel=1e-12)
    assert oracle.exact_loglik(th, locs, y) == pytest.approx(_ref.exact_loglik(S, y), rel=1e-12)


@pytest.mark.parametrize("nu,seed", [(0.5, 1), (1.5, 2), (2.5, 3)])
def test_all_previous_points_is_exact(nu, seed):
    # Eq. 2-3: with every earlier point in the conditioning set the product of
    # conditionals is the joint density, for any partition and any block order.
    locs, th, S, y, (bp, pi, nnp, nni) = _setup(n=240, bc=24, m=10**6, seed=seed, nu=nu,
                                               nugget=5e-2)
    ll, _, st = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    assert st == 0
    assert ll == pytest.approx(_ref.exact_loglik(S, y), rel=1e-10)


def test_singleton_blocks_no_neighbours_closed_form():
    n = 200
    locs, th, S, y, _ = _setup(n=n)
    bp = np.arange(n + 1, dtype=np.int64)
    pi = np.arange(n, dtype=np.int32)
    ll, _, _ = oracle.loglik(th, locs, y, bp, pi, np.zeros(n + 1, np.int64), np.zeros(0, np.int32))
    v = 1.3 + 1e-2
    want = np.sum(-0.5 * (np.log(2 * np.pi) + np.log(v) + y ** 2 / v))
    assert ll == pytest.approx(want, rel=1e-13)


def test_singleton_blocks_is_classic_vecchia():
    # bc = n: block Vecchia reduces to the classic univariate Vecchia approximation.
    n = 260
    locs = synth.locs_uniform(n, 2, 4)
    th = oracle.theta(1.0, 0.08, 0.5, 1e-3)
    S = _ref.full_cov(locs, 1.0, 0.08, 0.5, 1e-3)
    y = np.linalg.cholesky(S) @ synth.normal(4, 21, n)
    bp, pi, ce = oracle.build_blocks(locs, n, seed=9, iters=3)
    assert len(bp) - 1 == n
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 15)
    ll, per, _ = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    want = 0.0
    for i in range(n):
        j = pi[i]
        c = nni[nnp[i]:nnp[i + 1]].astype(np.int64)
        if len(c):
            w = np.linalg.solve(S[np.ix_(c, c)], S[c, j])
            mu, var = w @ y[c], S[j, j] - S[c, j] @ w
        else:
            mu, var = 0.0, S[j, j]
        li = -0.5 * (np.log(2 * np.pi) + np.log(var) + (y[j] - mu) ** 2 / var)
        assert per[i] == pytest.approx(li, rel=1e-10, abs=1e-12)
        want += li
    assert ll == pytest.approx(want, rel=1e-11)


def test_classic_vecchia_structure():
    # singleton blocks in a random order: a permutation; each singleton's query point is
    # the point itself, so its neighbours are the m earlier points nearest to it
    n = 300
    locs = synth.locs_uniform(n, 2, 5)
    bp, pi, ce = oracle.build_singletons(locs, seed=3)
    np.testing.assert_array_equal(bp, np.arange(n + 1))
    assert np.array_equal(np.sort(pi), np.arange(n)) and not np.array_equal(pi, np.arange(n))
    assert np.array_equal(ce, locs[pi])
    bp2, pi2, _ = oracle.build_singletons(locs, seed=4)
    assert not np.array_equal(pi, pi2)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 12)
    for i in range(n):
        cand = pi[:i].astype(np.int64)
        d2 = ((locs[cand] - locs[pi[i]]) ** 2).sum(axis=1)
        np.testing.assert_array_equal(nni[nnp[i]:nnp[i + 1]], cand[np.lexsort((cand, d2))][:12])


def test_classic_vecchia_loglik_by_kriging():
    # Sec. 1: classic Vecchia, each point conditioned on its m nearest earlier points, by
    # the univariate kriging formula sigma_j^2 = C_jj - c^T C^-1 c
    n = 240
    locs = synth.locs_uniform(n, 2, 6)
    th = oracle.theta(1.1, 0.06, 1.5, 2e-3)
    S = _ref.full_cov(locs, 1.1, 0.06, 1.5, 2e-3)
    y = np.linalg.cholesky(S) @ synth.normal(6, 21, n)
    bp, pi, ce = oracle.build_singletons(locs, seed=7)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 10)
    ll, per, _ = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    want = 0.0
    for i in range(n):
        j, c = pi[i], nni[nnp[i]:nnp[i + 1]].astype(np.int64)
        if len(c):
            w = np.linalg.solve(S[np.ix_(c, c)], S[c, j])
            mu, var = w @ y[c], S[j, j] - S[c, j] @ w
        else:
            mu, var = 0.0, S[j, j]
        want += -0.5 * (np.log(2 * np.pi) + np.log(var) + (y[j] - mu) ** 2 / var)
    assert ll == pytest.approx(want, rel=1e-11)


@pytest.mark.parametrize("d,ranges,nu", [(2, None, 0.5), (3, [0.1, 0.15, 0.3], 0.5), (2, None, 1.2),
                                         (2, None, 3.7)])
def test_dense_implied_precision(d, ranges, nu):
    # Eq. 4 defines a joint Gaussian with precision A^T D^{-1} A; its log density at y
    # equals the sum of the per-block conditionals (here also at non-half-integer nu,
    # where both sides need K_nu: the oracle's quadrature, the reference SciPy's kv).
    locs, th, S, y, (bp, pi, nnp, nni) = _setup(n=320, d=d, bc=40, m=12, seed=5, nu=nu,
                                               ranges=ranges, nugget=1e-3)
    ll, per, _ = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    P, ldP, _, _ = _ref.bv_dense_precision(S, bp, pi, nnp, nni)
    assert ll == pytest.approx(_ref.loglik_from_precision(P, ldP, y), rel=1e-10)
    for i in range(0, len(bp) - 1, 7):
        want = _ref.conditional_block_loglik(S, y, nni[nnp[i]:nnp[i + 1]], pi[bp[i]:bp[i + 1]])
        assert per[i] == pytest.approx(want, rel=1e-10)


def test_vecchia_trace_identity_and_kl_bounds():
    # tr(P S) = n for the implied precision P, so by Eq. 7 the KL divergence is
    # l_0(theta; 0) - l_a(theta; 0) >= 0, decreasing as nested conditioning sets grow.
    n = 240
    locs = synth.locs_uniform(n, 2, 7)
    th = oracle.theta(1.0, 0.1, 1.5, 1e-3)
    S = _ref.full_cov(locs, 1.0, 0.1, 1.5, 1e-3)
    bp, pi, ce = oracle.build_blocks(locs, 24, seed=2)
    y0 = np.zeros(n)
    l0 = oracle.exact_loglik(th, locs, y0)
    kls = []
    for m in [0, 3, 8, 20, 60, 10**6]:
        nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
        la, _, _ = oracle.loglik(th, locs, y0, bp, pi, nnp, nni)
        if m == 8:
            P, _, _, _ = _ref.bv_dense_precision(S, bp, pi, nnp, nni)
            assert np.trace(P @ S) == pytest.approx(n, rel=1e-9)
        kls.append(l0 - la)
    assert all(k >= -1e-9 for k in kls)
    assert all(a >= b - 1e-9 for a, b in zip(kls, kls[1:]))
    assert abs(kls[-1]) < 1e-8 * abs(l0)


def test_scaling_identity():
    locs, th, S, y, (bp, pi, nnp, nni) = _setup(n=200, seed=8)
    c = 3.7
    th2 = oracle.theta(1.3 * c, 0.1, 1.5, 1e-2 * c)
    l1, _, _ = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    l2, _, _ = oracle.loglik(th2, locs, np.sqrt(c) * y, bp, pi, nnp, nni)
    assert l2 == pytest.approx(l1 - 0.5 * len(y) * np.log(c), rel=1e-12)


def test_profile_form_in_sigma2():
    # Scaling sigma^2 and tau^2 together by s leaves every kriging weight unchanged and
    # scales every conditional covariance by s, so ell(s) = a - Q / (2 s) - (n / 2) log s
    # for constants a, Q: two evaluations fix a and Q, a third must follow, and the
    # maximiser over s is Q / n.
    locs, th, S, y, (bp, pi, nnp, nni) = _setup(n=300, seed=10)
    n = len(y)

    def ell(s):
        return oracle.loglik(oracle.theta(1.3 * s, 0.1, 1.5, 1e-2 * s), locs, y, bp, pi, nnp, nni)[0]

    l1, l2 = ell(1.0), ell(2.0)
    Q = 2.0 * (2.0 * (l2 - l1) + n * np.log(2.0))   # from l1 - l2 = -(Q - Q/2 - n log 2) / 2
    a = l1 + 0.5 * Q
    for s in (0.3, 5.0):
        assert ell(s) == pytest.approx(a - Q / (2 * s) - 0.5 * n * np.log(s), rel=1e-12)
    s_hat = Q / n
    for f in (0.999, 1.001):
        assert ell(s_hat * f) < ell(s_hat)


def test_order_within_sets_is_immaterial():
    locs, th, S, y, (bp, pi, nnp, nni) = _setup(n=300, seed=9)
    l1, _, _ = oracle.loglik(th, locs, y, bp, pi, nnp, nni)
    rng = np.random.default_rng(0)
    pi2, nni2 = pi.copy(), nni.copy()
    for i in range(len(bp) - 1):
        rng.shuffle(pi2[bp[i]:bp[i + 1]])
        rng.shuffle(nni2[nnp[i]:nnp[i + 1]])
    l2, _, _ = oracle.loglik(th, locs, y, bp, pi2, nnp, nni2)
    assert l2 == pytest.approx(l1, rel=1e-12)


def test_not_positive_definite_reported():
    locs, th, S, y, (bp, pi, nnp, nni) = _setup(n=120, bc=12, m=10)
    locs2 = locs.copy()
    # duplicate site inside the first block (no conditioning set) and no nugget: with
    # sigma^2 = 1 the second pivot is exactly 1 - 1 = 0
    locs2[pi[bp[0] + 1]] = locs2[pi[bp[0]]]
    th0 = oracle.theta(1.0, 0.1, 1.5, 0.0)
    ll, _, st = oracle.loglik(th0, locs2, y, bp, pi, nnp, nni, check=False)
    assert st == 4 and ll == -np.inf


def test_exact_draw_and_bv_draw():
    n = 220
    locs = synth.locs_uniform(n, 2, 12)
    th = oracle.theta(1.1, 0.07, 2.5, 1e-2)
    S = _ref.full_cov(locs, 1.1, 0.07, 2.5, 1e-2)
    z = synth.normal(12, 22, n)
    y = oracle.exact_draw(th, locs, z)
    np.testing.assert_allclose(y, np.linalg.cholesky(S) @ z, rtol=1e-10, atol=1e-12)
    # one block: the block-Vecchia draw is the exact draw
    y1 = oracle.bv_draw(th, locs, np.array([0, n]), np.arange(n, dtype=np.int32),
                        np.array([0, 0]), np.zeros(0, np.int32), z)
    np.testing.assert_allclose(y1, y, rtol=1e-10, atol=1e-12)
    # many blocks: A y = blockdiag(chol(C_i)) z for the dense implied factor A
    bp, pi, ce = oracle.build_blocks(locs, 22, seed=3)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 15)
    yb = oracle.bv_draw(th, locs, bp, pi, nnp, nni, z)
    _, _, A, Db = _ref.bv_dense_precision(S, bp, pi, nnp, nni)
    lhs = A @ yb
    for blk, C in Db:
        np.testing.assert_allclose(lhs[blk], np.linalg.cholesky(C) @ z[blk], rtol=1e-9,
                                   atol=1e-10)
