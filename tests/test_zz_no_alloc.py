"""bv_loglik_noalloc: the log-likelihood entry point for callers that cannot allocate
device memory (a caller running under a memory manager that owns every allocation, or
inside another library's stream-ordered section).  The caller owns every buffer; the
library's per-block partials live in a static device array.  Checked through the C ABI
against bv_loglik on two calls in a row, against the FP64 oracle in 1D, 2D and anisotropic
3D at nu = 1/2, 3/2, 5/2 and a general nu, and on its error returns (a non-positive-
definite block, a malformed structure).

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(bv, n=3000, d=2, bc=300, m=40, seed=0):
    import torch
    locs = synth.locs_uniform(n, d, seed)
    z = synth.normal(seed, 20, n)
    th = bv.theta(1.0, 0.08, 1.5, 1e-3)
    ctx = bv.Context(0)
    ctx.set_data(locs)
    bp, pi = ctx.build_blocks(bc, seed=seed, iters=20)
    ctx.select_neighbors(200)
    y = ctx.simulate(th, z)            # y drawn from the block-Vecchia model
    nnp, nni = ctx.select_neighbors(m)
    dev = dict(locs=torch.from_numpy(np.ascontiguousarray(locs.T)).cuda(),
               y=torch.from_numpy(y).cuda(), bp=torch.from_numpy(bp).cuda(),
               pi=torch.from_numpy(pi).cuda(), nnp=torch.from_numpy(nnp).cuda(),
               nni=torch.from_numpy(nni).cuda())
    return ctx, th, dev, len(bp) - 1, n, d


def test_noalloc_matches_bv_loglik_two_calls():
    import torch
    from paper_2410_04477_gb300 import bv
    ctx, th, dev, bc, n, d = _setup(bv)
    ref, per_ref, st = ctx.loglik(th, bv.BV_FP64, per_block=True)
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    per = torch.zeros(bc, dtype=torch.float64, device="cuda")
    for call in range(2):
        out.fill_(np.nan)
        per.zero_()
        torch.cuda.synchronize()
        st = bv.loglik_noalloc(th, dev["locs"].data_ptr(), dev["y"].data_ptr(), n, d, bc,
                               dev["bp"].data_ptr(), dev["pi"].data_ptr(), dev["nnp"].data_ptr(),
                               dev["nni"].data_ptr(), out.data_ptr(), per.data_ptr(), None)
        assert st == bv.BV_OK
        got = out.item()
        assert abs(got - ref) <= 1e-10 * abs(ref), (call, got, ref)
        np.testing.assert_allclose(per.cpu().numpy(), per_ref, rtol=1e-9, atol=1e-9)
    # a different theta right after: the shared scratch carries nothing over
    th2 = bv.theta(1.4, 0.05, 1.5, 2e-3)
    st = bv.loglik_noalloc(th2, dev["locs"].data_ptr(), dev["y"].data_ptr(), n, d, bc,
                           dev["bp"].data_ptr(), dev["pi"].data_ptr(), dev["nnp"].data_ptr(),
                           dev["nni"].data_ptr(), out.data_ptr(), None, None)
    ref2 = ctx.loglik(th2, bv.BV_FP64)
    assert abs(out.item() - ref2) <= 1e-10 * abs(ref2)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_limits():
    import torch
    from paper_2410_04477_gb300 import bv
    ctx, th, dev, bc, n, d = _setup(bv, n=1200, bc=120, m=400)   # m_i + b_i > 234
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    args = (dev["locs"].data_ptr(), dev["y"].data_ptr(), n, d, bc, dev["bp"].data_ptr(),
            dev["pi"].data_ptr(), dev["nnp"].data_ptr(), dev["nni"].data_ptr(), out.data_ptr(),
            None, None)
    with pytest.raises(bv.BVError) as e:
        bv.loglik_noalloc(th, *args)
    assert e.value.status == bv.BV_EINVAL
    big = list(args)
    big[4] = bv.BV_NOALLOC_MAX_BLOCKS + 1          # more blocks than the scratch holds
    with pytest.raises(bv.BVError) as e:
        bv.loglik_noalloc(th, *big)
    assert e.value.status == bv.BV_EINVAL
    ctx.close()


def _oracle_case(n, d, bc, m, th, seed, ranges=None):
    """Locations, y, the oracle's structure and its ell (Algorithm 1, FP64)."""
    locs = synth.locs_uniform(n, d, seed)
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=seed)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
    oth = oracle.theta(*th, ranges=ranges)
    y = oracle.exact_draw(oth, locs, synth.normal(seed, 20, n))
    ell, per, st = oracle.loglik(oth, locs, y, bp, pi, nnp, nni, check=False)
    return locs, y, bp, pi, nnp, nni, ell, per, st


def _dev(locs, y, bp, pi, nnp, nni):
    import torch
    return dict(locs=torch.from_numpy(np.ascontiguousarray(locs.T)).cuda(), y=torch.from_numpy(y).cuda(),
                bp=torch.from_numpy(bp).cuda(), pi=torch.from_numpy(pi).cuda(),
                nnp=torch.from_numpy(nnp).cuda(), nni=torch.from_numpy(np.ascontiguousarray(nni)).cuda())


def _call(bv, th, dev, n, d, bc, out, per=None):
    return bv.loglik_noalloc(th, dev["locs"].data_ptr(), dev["y"].data_ptr(), n, d, bc, dev["bp"].data_ptr(),
                             dev["pi"].data_ptr(), dev["nnp"].data_ptr(), dev["nni"].data_ptr(), out.data_ptr(),
                             None if per is None else per.data_ptr(), None)


@pytest.mark.parametrize("d,nu,ranges", [(1, 2.5, None), (2, 0.5, None), (2, 2.5, None), (2, 1.2, None),
                                         (3, 0.5, [0.1, 0.1, 0.3]), (3, 1.5, [0.2, 0.15, 0.3])])
def test_noalloc_matches_the_oracle(d, nu, ranges):
    import torch
    from paper_2410_04477_gb300 import bv
    n, bc, m = 2000, 200, 45
    th = (1.3, 0.07, nu, 2e-3)
    locs, y, bp, pi, nnp, nni, ell, per_o, st = _oracle_case(n, d, bc, m, th, 40 + d, ranges)
    assert st == 0
    dev = _dev(locs, y, bp, pi, nnp, nni)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros(len(bp) - 1, dtype=torch.float64, device="cuda")
    for _ in range(2):
        assert _call(bv, bv.theta(*th, ranges=ranges), dev, n, d, len(bp) - 1, out, per) == bv.BV_OK
        got = out.item()
        print(f"d={d} nu={nu}: noalloc {got:.12f} oracle {ell:.12f} |dl| {abs(got - ell):.2e}")
        assert abs(got - ell) <= 1e-10 * abs(ell)
        np.testing.assert_allclose(per.cpu().numpy(), per_o, rtol=1e-9, atol=1e-9)


def test_noalloc_not_positive_definite():
    import torch
    from paper_2410_04477_gb300 import bv
    n, bc, m = 800, 80, 20
    locs = synth.locs_uniform(n, 2, 77)
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=7)
    locs[pi[1]] = locs[pi[0]]      # first block (no conditioning set): a duplicate site
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
    y = synth.normal(77, 20, n)
    th = (1.0, 0.1, 1.5, 0.0)      # sigma^2 = 1 and no nugget: the second pivot is exactly 0
    ell, per_o, st = oracle.loglik(oracle.theta(*th), locs, y, bp, pi, nnp, nni, check=False)
    assert st == 4 and ell == -np.inf
    dev = _dev(locs, y, bp, pi, nnp, nni)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    per = torch.zeros(len(bp) - 1, dtype=torch.float64, device="cuda")
    assert _call(bv, bv.theta(*th), dev, n, 2, len(bp) - 1, out, per) == bv.BV_ENOTPD
    assert out.item() == -np.inf and per[0].item() == -np.inf
    # blocks whose points and conditioning set hold both copies of the site are singular:
    # whether their last pivot rounds to a tiny positive or a non-positive number depends
    # on the order of the operations, so only the other blocks are compared (to 1e-9)
    got = per.cpu().numpy()
    d0, d1 = int(pi[0]), int(pi[1])
    both = np.array([{d0, d1} <= set(np.concatenate([nni[nnp[i]:nnp[i + 1]], pi[bp[i]:bp[i + 1]]]).tolist())
                     for i in range(len(bp) - 1)])
    assert both[0] and both.sum() < len(both) // 2
    assert np.isfinite(got[~both]).all() and np.isfinite(per_o[~both]).all()
    np.testing.assert_allclose(got[~both], per_o[~both], rtol=1e-9, atol=1e-9)
    # the next call with a nugget is fine: the failure word was reset
    th2 = (1.0, 0.1, 1.5, 1e-3)
    assert _call(bv, bv.theta(*th2), dev, n, 2, len(bp) - 1, out) == bv.BV_OK
    ref = oracle.loglik(oracle.theta(*th2), locs, y, bp, pi, nnp, nni)[0]
    assert abs(out.item() - ref) <= 1e-10 * abs(ref)


@pytest.mark.parametrize("flaw", ["block_ptr decreases", "block_ptr[0] != 0", "nn_ptr[0] != 0",
                                  "blocks cover more than n", "point index >= n", "neighbour index < 0"])
def test_noalloc_rejects_a_malformed_structure(flaw):
    import torch
    from paper_2410_04477_gb300 import bv
    n, bc, m = 600, 60, 15
    th = (1.0, 0.1, 0.5, 1e-3)
    locs, y, bp, pi, nnp, nni, ell, _, _ = _oracle_case(n, 2, bc, m, th, 90)
    bp, pi, nnp, nni = bp.copy(), pi.copy(), nnp.copy(), nni.copy()
    if flaw == "block_ptr decreases":
        bp[5] = bp[4] - 1
    elif flaw == "block_ptr[0] != 0":
        bp[0] = 1
    elif flaw == "nn_ptr[0] != 0":
        nnp[0] = 1
    elif flaw == "blocks cover more than n":
        bp[-1] = n + 1
    elif flaw == "point index >= n":
        pi[123] = n
    else:
        nni[len(nni) // 2] = -1
    dev = _dev(locs, y, bp, pi, nnp, nni)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(bv.BVError) as e:
        _call(bv, bv.theta(*th), dev, n, 2, len(bp) - 1, out)
    assert e.value.status == bv.BV_EINVAL
    # a well-formed call right after is exact
    dev = _dev(*_oracle_case(n, 2, bc, m, th, 90)[:6])
    assert _call(bv, bv.theta(*th), dev, n, 2, len(bp) - 1, out) == bv.BV_OK
    assert abs(out.item() - ell) <= 1e-10 * abs(ell)
