"""Pins for the oracle's preprocessing: K-means blocks, the block order and the block
nearest-neighbour sets (Sec. 2.1-2.2, Algorithm 1)."""
import math

import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth


def _d2(x, c):
    # D2 written out independently: (x0-c0)^2 + (x1-c1)^2 + ... left to right
    acc = np.zeros(x.shape[0]) if x.ndim == 2 else 0.0
    for k in range(c.shape[-1]):
        t = (x[..., k] - c[..., k])
        acc = acc + t * t
    return acc


@pytest.mark.parametrize("n,d,k", [(600, 2, 40), (500, 3, 25)])
def test_kmeans_final_assignment_is_nearest_centre(n, d, k):
    locs = synth.locs_uniform(n, d, seed=11)
    label, cent = oracle.kmeans(locs, k, seed=5, iters=20)
    D = np.stack([_d2(locs, cent[c][None, :]) for c in range(k)], axis=1)
    np.testing.assert_array_equal(label, np.argmin(D, axis=1))


def test_kmeans_matches_library_lloyd_from_same_seeding():
    sk = pytest.importorskip("sklearn.cluster")
    locs = synth.locs_uniform(800, 2, seed=2)
    k = 30
    # seeding only (0 Lloyd iterations) gives the k-means++ centres
    _, init = oracle.kmeans(locs, k, seed=9, iters=0)
    label, cent = oracle.kmeans(locs, k, seed=9, iters=15)
    km = sk.KMeans(n_clusters=k, init=init, n_init=1, max_iter=15, tol=0.0,
                   algorithm="lloyd").fit(locs)
    assert (km.labels_ == label).mean() > 0.99
    np.testing.assert_allclose(km.cluster_centers_, cent, atol=1e-9)


def test_kmeans_inertia_non_increasing():
    locs = synth.locs_uniform(700, 2, seed=4)
    prev = np.inf
    for it in range(0, 12):
        label, cent = oracle.kmeans(locs, 35, seed=1, iters=it)
        # inertia of the centres after `it` updates, with their own optimal labels
        D = np.stack([_d2(locs, cent[c][None, :]) for c in range(35)], axis=1)
        inertia = D.min(axis=1).sum()
        assert inertia <= prev * (1 + 1e-12)
        prev = inertia


def test_kmeanspp_first_centre_and_distinct_seeds():
    locs = synth.locs_uniform(300, 2, seed=8)
    _, c0 = oracle.kmeans(locs, 1, seed=77, iters=0)
    r0 = oracle.splitmix64(77 ^ 0x6B6D65616E732B2B, 0)
    first = (r0 * 300) >> 64
    np.testing.assert_array_equal(c0[0], locs[first])
    _, c = oracle.kmeans(locs, 50, seed=77, iters=0)
    # k-means++ never picks an already chosen point while unchosen points have D2 > 0
    assert len({tuple(v) for v in c}) == 50


def _ceil_log2(v):
    e = 0
    while (1 << e) < v:
        e += 1
    return e


def kmeanspp_picks(locs, k, seed):
    """The k-means++ seeding written out from its stated rule, in plain Python integers:
    the first centre is point floor(r_0 n / 2^64); centre t is drawn with probability
    proportional to D^2 on integer weights w_j = floor(D2_j 2^s), with s the largest
    exponent that keeps n (d2max 2^s) below 2^61 (d2max: squared diagonal of the bounding
    box); target = floor(r_t W / 2^64); the pick is the first j whose inclusive prefix sum
    of w exceeds the target.  r_t = SplitMix64 draw t of the stream seed ^ "kmeans++"."""
    n, d = locs.shape
    lo, hi = locs.min(axis=0), locs.max(axis=0)
    d2max = 0.0
    for a in range(d):
        d2max = d2max + (hi[a] - lo[a]) * (hi[a] - lo[a])
    s = 61 - _ceil_log2(n) - (math.frexp(d2max)[1] + 1)
    stream = seed ^ 0x6B6D65616E732B2B
    picks = [(oracle.splitmix64(stream, 0) * n) >> 64]
    D2 = _d2(locs, locs[picks[0]][None, :])
    for t in range(1, k):
        w = [int(math.ldexp(float(v), s)) for v in D2]
        W = sum(w)
        r = oracle.splitmix64(stream, t)
        if W == 0:
            pick = (r * n) >> 64
        else:
            target, pre, pick = (r * W) >> 64, 0, n - 1
            for j, wj in enumerate(w):
                pre += wj
                if pre > target:
                    pick = j
                    break
        picks.append(pick)
        D2 = np.minimum(D2, _d2(locs, locs[pick][None, :]))
    return picks


@pytest.mark.parametrize("n,d,k,seed", [(400, 2, 10, 3), (250, 3, 8, 41), (1000, 2, 6, 12345)])
def test_kmeanspp_picks_follow_the_d2_rule(n, d, k, seed):
    locs = synth.locs_uniform(n, d, seed=seed + 1)
    _, cent = oracle.kmeans(locs, k, seed=seed, iters=0)
    np.testing.assert_array_equal(cent, locs[kmeanspp_picks(locs, k, seed)])


def test_kmeanspp_second_centre_is_drawn_proportional_to_d2():
    # the law itself, independent of the integer weights: over many seeds the second
    # centre is point j with probability D2_j / sum D2, D2 to the first centre
    n, trials = 12, 6000
    locs = synth.locs_uniform(n, 2, seed=5)
    counts = np.zeros((n, n))
    for seed in range(trials):
        _, c = oracle.kmeans(locs, 2, seed=seed, iters=0)
        i = int(np.flatnonzero((locs == c[0]).all(axis=1))[0])
        j = int(np.flatnonzero((locs == c[1]).all(axis=1))[0])
        counts[i, j] += 1
    chi2, dof = 0.0, 0
    for i in range(n):
        tot = counts[i].sum()
        if tot < 200:
            continue
        p = _d2(locs, locs[i][None, :])
        p = p / p.sum()
        e = tot * p
        keep = e > 0
        chi2 += (((counts[i] - e)[keep]) ** 2 / e[keep]).sum()
        dof += int(keep.sum()) - 1
        assert counts[i, i] == 0  # a chosen point has D2 = 0
    assert dof > 20
    # chi-square with dof degrees of freedom: mean dof, sd sqrt(2 dof); allow 5 sd
    assert chi2 < dof + 5 * math.sqrt(2 * dof), (chi2, dof)


@pytest.mark.parametrize("n,d,bc", [(2000, 2, 200), (900, 3, 90)])
def test_blocks_partition_and_centroids(n, d, bc):
    locs = synth.locs_uniform(n, d, seed=0)
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=0, iters=20)
    nb = len(bp) - 1
    assert nb <= bc and nb > 0.9 * bc
    assert bp[0] == 0 and bp[-1] == n and np.all(np.diff(bp) >= 1)
    np.testing.assert_array_equal(np.sort(pi), np.arange(n))      # each point once
    for i in range(nb):
        mem = pi[bp[i]:bp[i + 1]]
        assert np.all(np.diff(mem) > 0)                            # ascending index
        np.testing.assert_allclose(ce[i], locs[mem].mean(axis=0), atol=1e-12)
    # blocks are K-means clusters: every point is nearest to its own block centroid
    D = np.stack([_d2(locs, ce[i][None, :]) for i in range(nb)], axis=1)
    own = np.empty(n, np.int64)
    for i in range(nb):
        own[pi[bp[i]:bp[i + 1]]] = i
    # the centroids here are the means of the final members, one update after the final
    # labels, so allow the few points that a last Lloyd step would still move
    assert (np.argmin(D, axis=1) == own).mean() > 0.97


def integer_mean(values, n, amax):
    """A block centroid coordinate written out from its stated rule, in Python integers:
    q = 61 - ceil(log2 n) - (e + 1), where 2^(e-1) <= max |coordinate| < 2^e over the
    dataset of n points; S = the sum of the members' x 2^q, each rounded to the nearest
    integer (ties to even); the centroid is (S / count, one rounded division) 2^-q."""
    q = 61 - _ceil_log2(n) - (math.frexp(amax)[1] + 1)
    S = sum(round(math.ldexp(float(v), q)) for v in values)
    return math.ldexp(float(S) / len(values), -q)


@pytest.mark.parametrize("n,d,bc,shift,scale", [(2000, 2, 200, 0.0, 1.0), (900, 3, 90, -0.5, 3.0),
                                                (500, 1, 50, -7.25, 0.01)])
def test_block_centroids_follow_the_integer_mean_rule(n, d, bc, shift, scale):
    # bit for bit, with negative coordinates and other magnitudes: the exponent q follows
    # the largest |coordinate|, so its choice shows in the last bits of every centroid
    locs = synth.locs_uniform(n, d, seed=5) * scale + shift
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=3, iters=20)
    amax = float(np.abs(locs).max())
    for i in range(len(bp) - 1):
        mem = pi[bp[i]:bp[i + 1]]
        for k in range(d):
            assert ce[i, k] == integer_mean(locs[mem, k], n, amax), (i, k)


def test_block_order_is_a_seeded_permutation():
    locs = synth.locs_uniform(1000, 2, seed=3)
    a = oracle.build_blocks(locs, 100, seed=1)
    b = oracle.build_blocks(locs, 100, seed=1)
    c = oracle.build_blocks(locs, 100, seed=2)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)
    assert not np.array_equal(a[1], c[1])


ZETA_STREAM = 0x7A6574615F6F7264  # the ASCII bytes of "zeta_ord"


def fisher_yates(count, seed):
    """The block permutation written out from its stated rule, in plain Python integers:
    start from the identity; for i = count - 1 down to 1 take r_i = SplitMix64 output i of
    the stream seed ^ "zeta_ord", j = floor(r_i (i + 1) / 2^64) (uniform on 0 .. i), and
    swap entries i and j."""
    perm = list(range(count))
    stream = seed ^ ZETA_STREAM
    for i in range(count - 1, 0, -1):
        j = (oracle.splitmix64(stream, i) * (i + 1)) >> 64
        perm[i], perm[j] = perm[j], perm[i]
    return perm


@pytest.mark.parametrize("n,d,bc,seed", [(1500, 2, 150, 4), (600, 3, 60, 77)])
def test_block_order_follows_the_fisher_yates_rule(n, d, bc, seed):
    # the non-empty K-means clusters in cluster-index order, shuffled by the stated rule:
    # block position p holds cluster perm[p], its points ascending
    locs = synth.locs_uniform(n, d, seed=seed + 2)
    label, _ = oracle.kmeans(locs, bc, seed, iters=20)
    clusters = [c for c in (np.flatnonzero(label == k) for k in range(bc)) if len(c)]
    bp, pi, _ = oracle.build_blocks(locs, bc, seed, iters=20)
    assert len(bp) - 1 == len(clusters)
    for p, k in enumerate(fisher_yates(len(clusters), seed)):
        np.testing.assert_array_equal(pi[bp[p]:bp[p + 1]], clusters[k])


@pytest.mark.parametrize("n,seed", [(1, 3), (2, 0), (57, 9), (1000, 123456789)])
def test_singleton_and_random_orders_follow_the_fisher_yates_rule(n, seed):
    locs = synth.locs_uniform(n, 2, seed=seed + 1)
    bp, pi, ce = oracle.build_singletons(locs, seed)
    np.testing.assert_array_equal(pi, fisher_yates(n, seed))
    np.testing.assert_array_equal(bp, np.arange(n + 1))
    np.testing.assert_array_equal(ce, locs[pi])
    np.testing.assert_array_equal(oracle.order_blocks(locs, "random", seed=seed), fisher_yates(n, seed))


def test_block_order_law_is_uniform():
    # a random block ordering makes every order equally likely: over 4,800 seeds each of
    # the 24 orders of four singletons appears about 200 times (chi-square with 23 degrees
    # of freedom within 5 sd).  A shuffle that never draws j = i (Sattolo's) yields only
    # the 6 cyclic orders, one that draws j from all positions is biased.
    locs = synth.locs_uniform(4, 2, seed=1)
    counts = {}
    for seed in range(4800):
        key = tuple(oracle.build_singletons(locs, seed)[1].tolist())
        counts[key] = counts.get(key, 0) + 1
    assert len(counts) == 24
    e = 4800 / 24
    chi2 = sum((v - e) ** 2 / e for v in counts.values())
    assert chi2 < 23 + 5 * math.sqrt(2 * 23), chi2


def _brute_nn(locs, bp, pi, ce, m):
    out = []
    for i in range(len(bp) - 1):
        cand = pi[:bp[i]].astype(np.int64)
        if len(cand) == 0:
            out.append(np.zeros(0, np.int64))
            continue
        d2 = _d2(locs[cand], ce[i][None, :])
        order = np.lexsort((cand, d2))
        out.append(cand[order[:min(m, len(cand))]])
    return out


@pytest.mark.parametrize("n,d,bc,m", [(2000, 2, 200, 30), (800, 3, 80, 50), (300, 2, 30, 400)])
def test_neighbors_match_brute_force(n, d, bc, m):
    locs = synth.locs_uniform(n, d, seed=5)
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=3)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
    want = _brute_nn(locs, bp, pi, ce, m)
    assert nnp[0] == 0 and nnp[1] == 0                             # first block: none
    for i, w in enumerate(want):
        np.testing.assert_array_equal(nni[nnp[i]:nnp[i + 1]], w)
        assert nnp[i + 1] - nnp[i] == min(m, bp[i])
        earlier = set(pi[:bp[i]].tolist())
        assert set(nni[nnp[i]:nnp[i + 1]].tolist()) <= earlier


def test_neighbors_nested_in_m_and_per_block_sizes():
    locs = synth.locs_uniform(1200, 2, seed=6)
    bp, pi, ce = oracle.build_blocks(locs, 120, seed=4)
    p10, i10 = oracle.select_neighbors(locs, bp, pi, ce, 10)
    p40, i40 = oracle.select_neighbors(locs, bp, pi, ce, 40)
    for b in range(len(bp) - 1):
        a = i10[p10[b]:p10[b + 1]]
        np.testing.assert_array_equal(a, i40[p40[b]:p40[b]+len(a)])
    mpb = (np.arange(len(bp) - 1) % 7 * 5).astype(np.int32)
    pv, iv = oracle.select_neighbors(locs, bp, pi, ce, -1, m_per_block=mpb)
    for b in range(len(bp) - 1):
        assert pv[b + 1] - pv[b] == min(mpb[b], bp[b])
        np.testing.assert_array_equal(iv[pv[b]:pv[b + 1]], i40[p40[b]:p40[b] + pv[b + 1] - pv[b]])


def test_ties_broken_by_index():
    # a lattice puts many candidates at exactly the same distance from a centroid
    g = np.arange(8) / 8.0
    locs = np.array([(x, y) for x in g for y in g])
    bp, pi, ce = oracle.build_blocks(locs, 16, seed=1)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 9)
    want = _brute_nn(locs, bp, pi, ce, 9)
    for i, w in enumerate(want):
        np.testing.assert_array_equal(nni[nnp[i]:nnp[i + 1]], w)
