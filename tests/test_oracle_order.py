"""Pins for the oracle's block orderings (Sec. 2.1: random, maxmin, Morton, KD-tree,
Hilbert), each checked through a property that characterises it rather than by
rebuilding it: adjacency of consecutive cells on a full grid for the Hilbert curve,
quadrant nesting for the Z-order, the median-split partition for the KD-tree order and
the greedy farthest-point property for maxmin."""
import itertools

import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth


def _is_perm(p, n):
    return np.array_equal(np.sort(p), np.arange(n))


@pytest.mark.parametrize("d,k", [(2, 5), (3, 3)])
def test_hilbert_visits_grid_cells_adjacently(d, k):
    # the level-k cells of a 2^k grid, placed on the 21-bit lattice, in Hilbert order:
    # every step moves to a face-adjacent cell, and the curve starts at the origin
    side = 1 << k
    cells = np.array(list(itertools.product(range(side), repeat=d)), np.uint64)
    keys = np.array([oracle.hilbert_index(c << np.uint64(21 - k)) for c in cells], dtype=np.uint64)
    assert len(np.unique(keys)) == len(keys)
    path = cells[np.argsort(keys)].astype(np.int64)
    steps = np.abs(np.diff(path, axis=0)).sum(axis=1)
    assert np.all(steps == 1)
    assert np.all(path[0] == 0)


def test_hilbert_order_of_centroids_on_a_grid():
    # centroids exactly on a 16 x 16 grid spanning the unit square map to distinct 21-bit
    # cells; the ordering visits them in grid-adjacent steps
    g = np.arange(16) / 16.0
    ce = np.array([(a, b) for a in g for b in g]) + 1.0 / 32
    perm = oracle.order_blocks(ce, "hilbert")
    assert _is_perm(perm, len(ce))
    path = np.rint(ce[perm] * 16 - 0.5).astype(int)
    assert np.all(np.abs(np.diff(path, axis=0)).sum(axis=1) == 1)


def test_morton_quadrant_nesting():
    # Z-order on a 2^k grid: at every level the sequence of sub-quadrant labels
    # (bit of axis 0 first, then axis 1) is non-decreasing within each parent cell
    k = 4
    g = (np.arange(1 << k) + 0.5) / (1 << k)
    ce = np.array([(a, b) for a in g for b in g])
    perm = oracle.order_blocks(ce, "morton")
    assert _is_perm(perm, len(ce))
    cell = np.floor(ce[perm] * (1 << k)).astype(int)
    for level in range(1, k + 1):
        parent = cell >> (k - level + 1)
        child = (cell >> (k - level)) & 1
        lab = child[:, 0] + 2 * child[:, 1]
        pid = parent[:, 0] * (1 << k) + parent[:, 1]
        for p in np.unique(pid):
            assert np.all(np.diff(lab[pid == p]) >= 0)
    assert np.all(np.diff(perm[:2]) != 0) and tuple(cell[0]) == (0, 0)


def test_kdtree_median_partition():
    ce = synth.locs_uniform(203, 2, 11)
    perm = oracle.order_blocks(ce, "kdtree")
    assert _is_perm(perm, len(ce))

    def check(seq, depth):
        if len(seq) <= 1:
            return
        ax = depth % 2
        h = len(seq) // 2
        left, right = seq[:h], seq[h:]
        kl = max((ce[p, ax], p) for p in left)
        kr = min((ce[p, ax], p) for p in right)
        assert kl < kr
        check(left, depth + 1)
        check(right, depth + 1)

    check(list(perm), 0)


def test_maxmin_greedy_property():
    ce = synth.locs_uniform(150, 2, 12)
    perm = oracle.order_blocks(ce, "maxmin")
    assert _is_perm(perm, len(ce))
    d2 = ((ce[:, None, :] - ce[None, :, :]) ** 2).sum(-1)
    mean = ce.mean(axis=0)
    to_mean = ((ce - mean) ** 2).sum(1)
    assert perm[0] == int(np.flatnonzero(to_mean == to_mean.min())[0])
    placed = [perm[0]]
    for q in range(1, len(perm)):
        rest = np.setdiff1d(np.arange(len(ce)), placed)
        dmin = d2[np.ix_(rest, placed)].min(axis=1)
        best = rest[dmin == dmin.max()].min()
        assert perm[q] == best
        placed.append(perm[q])


def test_random_order_is_a_seeded_permutation():
    ce = synth.locs_uniform(100, 2, 13)
    a, b, c = (oracle.order_blocks(ce, "random", seed=s) for s in (1, 1, 2))
    assert _is_perm(a, 100) and np.array_equal(a, b) and not np.array_equal(a, c)


def test_ordering_keeps_the_likelihood_a_valid_block_vecchia():
    # any block order with all earlier points conditioned on is exact (Eq. 3); with a
    # finite m every order still gives tr(P Sigma) = n, so KL = ell0(0) - ella(0) >= 0
    from tests import _ref
    n = 240
    locs = synth.locs_uniform(n, 2, 14)
    th = oracle.theta(1.0, 0.1, 1.5, 1e-2)
    S = _ref.full_cov(locs, 1.0, 0.1, 1.5, 1e-2)
    bp, pi, ce = oracle.build_blocks(locs, 24, seed=3)
    l0 = oracle.exact_loglik(th, locs, np.zeros(n))
    for name in oracle.ORDERS:
        nbp, npi, nce = oracle.apply_block_order(bp, pi, ce, oracle.order_blocks(ce, name, seed=5))
        nnp, nni = oracle.select_neighbors(locs, nbp, npi, nce, 10**6)
        assert oracle.loglik(th, locs, np.zeros(n), nbp, npi, nnp, nni)[0] == pytest.approx(l0, rel=1e-10)
        nnp, nni = oracle.select_neighbors(locs, nbp, npi, nce, 8)
        la = oracle.loglik(th, locs, np.zeros(n), nbp, npi, nnp, nni)[0]
        assert l0 - la >= -1e-9
