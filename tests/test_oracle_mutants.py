"""The pins catch plausible mistakes: each test compiles a copy of the oracle with one
planted mistake (the real source is untouched) and checks that at least one pin fails."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth
from tests import _ref

SRC = os.path.join(os.path.dirname(oracle.__file__), "bv_oracle.c")

MUTANTS = {
    "nugget dropped": ("if (same) c += th->nugget;", "if (same) c += 0.0 * th->nugget;"),
    "Schur complement sign": ("Slk[j * b + k] -= s;", "Slk[j * b + k] += s;"),
    "log-det factor 2 missing": ("dl *= 2.0;", "dl *= 1.0;"),
    "nu = 3/2 closed form": ("return (1.0 + x) * exp(-x);", "return (1.0 + 0.5 * x) * exp(-x);"),
    "conditional mean sign": ("mu[j] = s;", "mu[j] = -s;"),
    "y' from the block instead of the neighbours": ("for (int64_t j = 0; j < m; j++) col[j] = y[nn[j]];",
                                                    "for (int64_t j = 0; j < m; j++) col[j] = y[blk[j % b]];"),
    "2 pi term counts one extra point": ("ell = -0.5 * (u + dl + (double)b * log(2.0 * M_PI));",
                                         "ell = -0.5 * (u + dl + (double)(b + 1) * log(2.0 * M_PI));"),
    "neighbour ties to the highest index": ("return a.d2 < b.d2 || (a.d2 == b.d2 && a.idx < b.idx);",
                                            "return a.d2 < b.d2 || (a.d2 == b.d2 && a.idx > b.idx);"),
    "candidates include the block's first point": ("for (int64_t p = 0; p < block_ptr[i]; p++) {",
                                                   "for (int64_t p = 0; p <= block_ptr[i] && p < n; p++) {"),
    "K-means ties to the highest centre": ("if (t < best) { best = t; bi = (int32_t)c; }",
                                           "if (t <= best) { best = t; bi = (int32_t)c; }"),
    "centroid without the 2^-q scaling": ("cent[c * d + j] = ldexp((double)S[c * d + j] / (double)counts[c], -q);",
                                          "cent[c * d + j] = ldexp((double)S[c * d + j] / (double)counts[c], -q + 1);"),
    "centroid exponent q one bit short": ("*q_out = 61 - ln - (ea + 1);", "*q_out = 60 - ln - (ea + 1);"),
    "prediction cross-covariance with the nugget": (
        "locs_star + (int64_t)blk[k] * d, 0);", "locs_star + (int64_t)blk[k] * d, 1);"),
    "prediction covariance plus the correction": ("cov[r * b + c] -= t;", "cov[r * b + c] += t;"),
    "backward substitution skipped": ("for (int64_t i = n - 1; i >= 0; i--) {\n        double t = x[i];",
                                      "for (int64_t i = n - 1; i >= n; i--) {\n        double t = x[i];"),
    "prediction neighbour keys shifted by one index": (
        "key.idx = (int32_t)j;", "key.idx = (int32_t)(j > 0 ? j - 1 : 0);"),
    "Box-Muller radius without the factor 2": ("sqrt(-2.0 * log(u1))", "sqrt(-1.0 * log(u1))"),
    "Box-Muller pair reuses the cosine": ("rho * sin(2.0 * M_PI * u2)", "rho * cos(2.0 * M_PI * u2)"),
    "conditional-simulation pairs without the location offset": (
        "const uint64_t c = (uint64_t)j * half + (uint64_t)(r / 2);",
        "const uint64_t c = (uint64_t)j + (uint64_t)(r / 2);"),
    "Hilbert without the Gray encoding": ("for (int i = 1; i < d; i++) X[i] ^= X[i - 1];",
                                          "for (int i = 1; i < d; i++) X[i] ^= 0;"),
    "maxmin ties to the highest position": ("if (!used[p] && dmin[p] > far)", "if (!used[p] && dmin[p] >= far)"),
    "KD-tree split at the wrong axis": ("const int ax = depth % d;", "const int ax = (depth + 1) % d;"),
    "Morton with the axes' bits swapped": ("<< (b * d + a);", "<< (b * d + (d - 1 - a));"),
    "block order by Sattolo's shuffle (j < i)": (
        "int64_t j = (int64_t)or_mulhi(or_sm64(zs, (uint64_t)i), (uint64_t)(i + 1));\n        int64_t t = perm[i];",
        "int64_t j = (int64_t)or_mulhi(or_sm64(zs, (uint64_t)i), (uint64_t)i);\n        int64_t t = perm[i];"),
    "block order drawn from the wrong stream position": (
        "int64_t j = (int64_t)or_mulhi(or_sm64(zs, (uint64_t)i), (uint64_t)(i + 1));\n        int64_t t = perm[i];",
        "int64_t j = (int64_t)or_mulhi(or_sm64(zs, (uint64_t)(i - 1)), (uint64_t)(i + 1));\n        int64_t t = perm[i];"),
    "k-means++ drawn proportional to D": [("W += (uint64_t)ldexp(D2[i], s);", "W += (uint64_t)ldexp(sqrt(D2[i]), s);"),
                                          ("pre += (uint64_t)ldexp(D2[i], s);",
                                           "pre += (uint64_t)ldexp(sqrt(D2[i]), s);")],
}
# Not planted: comparing the k-means++ prefix sum with >= instead of > changes a pick only
# when the target equals a prefix sum exactly, which has probability about n / W with the
# total weight W near 2^58 -- no input distinguishes the two rules.


def _build(tmp_path, edits):
    """Compile the oracle with the planted mistake: one (old, new) edit or a list of them."""
    src = open(SRC).read()
    for old, new in ([edits] if isinstance(edits, tuple) else edits):
        assert src.count(old) >= 1, old
        src = src.replace(old, new, 1)
    path = tmp_path / "mut.c"
    path.write_text(src)
    so = str(tmp_path / "libmut.so")
    subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fopenmp", "-shared", "-fPIC",
                    "-o", so, str(path), "-lm"], check=True)
    return so


def _pin_matern():
    x = np.logspace(-3, 1, 50)
    return all(np.allclose(oracle.matern_corr(nu, x), _ref.matern_kv(nu, x), rtol=1e-12)
               for nu in (0.5, 1.5, 2.5))


def _setup():
    n = 240
    locs = synth.locs_uniform(n, 2, 3)
    S = _ref.full_cov(locs, 1.2, 0.1, 1.5, 1e-2)
    y = np.linalg.cholesky(S) @ synth.normal(3, 20, n)
    return n, locs, S, y, oracle.theta(1.2, 0.1, 1.5, 1e-2)


def _pin_one_block():
    n, locs, S, y, th = _setup()
    ll1, _, _ = oracle.loglik(th, locs, y, np.array([0, n]), np.arange(n, dtype=np.int32),
                              np.array([0, 0]), np.zeros(0, np.int32), check=False)
    return abs(ll1 - _ref.exact_loglik(S, y)) < 1e-9 * abs(ll1)


def _pin_dense():
    n, locs, S, y, th = _setup()
    bp, pi, ce = oracle.build_blocks(locs, 24, seed=2)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 12)
    ll, per, st = oracle.loglik(th, locs, y, bp, pi, nnp, nni, check=False)
    P, ldP, _, _ = _ref.bv_dense_precision(S, bp, pi, nnp, nni)
    return st == 0 and abs(ll - _ref.loglik_from_precision(P, ldP, y)) < 1e-9 * abs(ll)


def _lattice():
    g = np.arange(10) / 10.0
    return np.array([(a, b) for a in g for b in g])


def _pin_neighbours():
    lat = _lattice()
    lbp, lpi, lce = oracle.build_blocks(lat, 20, seed=1, iters=5)
    lnp, lni = oracle.select_neighbors(lat, lbp, lpi, lce, 9)
    for i in range(len(lbp) - 1):
        cand = lpi[:lbp[i]].astype(np.int64)
        if len(cand) == 0:
            continue
        diff = lat[cand] - lce[i]
        d2 = diff[:, 0] * diff[:, 0] + diff[:, 1] * diff[:, 1]
        want = cand[np.lexsort((cand, d2))][:min(9, len(cand))]
        if not np.array_equal(lni[lnp[i]:lnp[i + 1]], want):
            return False
    return True


def _pin_centroids():
    lat = _lattice()
    lbp, lpi, lce = oracle.build_blocks(lat, 20, seed=1, iters=5)
    return all(np.allclose(lce[i], lat[lpi[lbp[i]:lbp[i + 1]]].mean(axis=0), atol=1e-12)
               for i in range(len(lbp) - 1))


def _pin_centroid_rule():
    from tests.test_oracle_blocks import integer_mean
    locs = synth.locs_uniform(300, 2, 8) * 2.0 - 1.0
    bp, pi, ce = oracle.build_blocks(locs, 30, seed=4, iters=5)
    amax = float(np.abs(locs).max())
    return all(ce[i, k] == integer_mean(locs[pi[bp[i]:bp[i + 1]], k], 300, amax)
               for i in range(len(bp) - 1) for k in range(2))


def _pin_kmeans_tie():
    # three collinear points; with the two seeded centres at the ends (iters = 0) the
    # middle point is exactly equidistant and must go to the lower centre index
    x = np.array([[0.0], [2.0], [1.0]])
    for seed in range(400):
        lab, cen = oracle.kmeans(x, 2, seed=seed, iters=0)
        if sorted(cen[:, 0].tolist()) == [0.0, 2.0]:
            return lab[2] == 0 and lab[0] == int(np.argmin(np.abs(cen[:, 0] - 0.0)))
    raise AssertionError("no seed puts the centres at both ends")


def _pin_kriging():
    n, locs, S, y, th = _setup()
    lo, ls = locs[:200], locs[200:]
    bp, pi, ce = oracle.build_pred_blocks(ls, 4, seed=5)
    nnp, nni = oracle.select_pred_neighbors(lo, ce, 10**6)
    mean, var, _ = oracle.predict(th, lo, y[:200], ls, bp, pi, nnp, nni)
    Syy, Sxy = S[:200, :200], S[200:, :200]
    kc = S[200:, 200:] - Sxy @ np.linalg.solve(Syy, Sxy.T)
    return (np.allclose(mean, Sxy @ np.linalg.solve(Syy, y[:200]), rtol=1e-8, atol=1e-9)
            and np.allclose(var, np.diag(kc), rtol=1e-8, atol=1e-10))


def _pin_pred_neighbours():
    lat = _lattice()
    ce = np.array([[0.33, 0.71], [0.95, 0.95], [0.0, 0.0]])
    nnp, nni = oracle.select_pred_neighbors(lat, ce, 7)
    for i, c in enumerate(ce):
        d2 = ((lat - c) ** 2).sum(axis=1)
        if not np.array_equal(nni[nnp[i]:nnp[i + 1]], np.lexsort((np.arange(len(lat)), d2))[:7]):
            return False
    return True


def _pin_csim_normal():
    from scipy import stats
    z = np.array([oracle.csim_normal(9, j, 1000, r) for j in range(20) for r in range(1000)])
    a, b = z[0::2], z[1::2]
    return stats.kstest(z, "norm").pvalue > 1e-3 and abs(np.corrcoef(a, b)[0, 1]) < 4 / np.sqrt(len(a))


def _pin_csim_rule():
    from tests.test_oracle_predict import csim_normal_rule
    return all(oracle.csim_normal(9, j, 11, r) == pytest.approx(csim_normal_rule(9, j, 11, r), rel=1e-14, abs=1e-15)
               for j in (0, 1, 5) for r in range(11))


def _pin_hilbert():
    import itertools
    cells = np.array(list(itertools.product(range(16), repeat=2)), np.uint64)
    keys = np.array([oracle.hilbert_index(c << np.uint64(17)) for c in cells], dtype=np.uint64)
    path = cells[np.argsort(keys)].astype(np.int64)
    return bool(np.all(np.abs(np.diff(path, axis=0)).sum(axis=1) == 1))


def _pin_orders():
    # a lattice has many exact distance ties: maxmin must break them to the lowest position
    g = np.arange(6) / 6.0
    ce = np.array([(a, b) for a in g for b in g])
    perm = oracle.order_blocks(ce, "maxmin")
    d2 = ((ce[:, None, :] - ce[None, :, :]) ** 2).sum(-1)
    placed = [perm[0]]
    for q in range(1, len(perm)):
        rest = np.setdiff1d(np.arange(len(ce)), placed)
        dmin = d2[np.ix_(rest, placed)].min(axis=1)
        if perm[q] != rest[dmin == dmin.max()].min():
            return False
        placed.append(perm[q])
    # KD-tree: first half on the low side of axis 0; Morton: first quadrant first
    pts = synth.locs_uniform(64, 2, 9)
    kd = oracle.order_blocks(pts, "kdtree")
    if not max(pts[kd[:32], 0]) < min(pts[kd[32:], 0]):
        return False
    q = (np.arange(8) + 0.5) / 8
    grid = np.array([(a, b) for a in q for b in q])
    mo = oracle.order_blocks(grid, "morton")
    first = np.floor(grid[mo[:16]] * 8).astype(int)
    second = np.floor(grid[mo[16:32]] * 8).astype(int)
    return bool(np.all(first < 4) and np.all(second[:, 0] >= 4) and np.all(second[:, 1] < 4))


def _pin_kmeanspp():
    from tests.test_oracle_blocks import kmeanspp_picks
    locs = synth.locs_uniform(300, 2, 4)
    _, cent = oracle.kmeans(locs, 8, seed=21, iters=0)
    return bool((cent == locs[kmeanspp_picks(locs, 8, 21)]).all())


def _pin_block_order():
    from tests.test_oracle_blocks import fisher_yates
    locs = synth.locs_uniform(400, 2, 6)
    label, _ = oracle.kmeans(locs, 40, 11, iters=5)
    clusters = [c for c in (np.flatnonzero(label == k) for k in range(40)) if len(c)]
    bp, pi, _ = oracle.build_blocks(locs, 40, seed=11, iters=5)
    return len(bp) - 1 == len(clusters) and all(
        np.array_equal(pi[bp[p]:bp[p + 1]], clusters[k]) for p, k in enumerate(fisher_yates(len(clusters), 11)))


PINS = {"hilbert adjacency": _pin_hilbert, "orderings": _pin_orders, "kriging": _pin_kriging, "prediction neighbours": _pin_pred_neighbours,
        "conditional-simulation normals": _pin_csim_normal, "conditional-simulation draw rule": _pin_csim_rule, "matern": _pin_matern, "one block = Eq. 1": _pin_one_block, "dense precision": _pin_dense,
        "neighbours brute force": _pin_neighbours, "centroid = member mean": _pin_centroids,
        "centroid integer-mean rule": _pin_centroid_rule,
        "K-means exact tie": _pin_kmeans_tie, "k-means++ seeding rule": _pin_kmeanspp,
        "block order rule": _pin_block_order}


def _pins():
    """Reduced versions of the pins in test_oracle_*.py; a pin that raises has failed."""
    out = {}
    for name, f in PINS.items():
        try:
            out[name] = bool(f())
        except Exception as e:  # noqa: BLE001 -- a crash is a caught mistake
            out[name] = False
    return out


def test_real_oracle_passes_the_reduced_pins():
    res = _pins()
    assert all(res.values()), res


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    with oracle.use_library(_build(tmp_path, MUTANTS[name])):
        res = _pins()
    assert not all(res.values()), f"mistake '{name}' passed every pin: {res}"
