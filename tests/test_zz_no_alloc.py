"""bv_loglik_noalloc: the log-likelihood entry point for callers that cannot allocate
device memory (a caller running under a memory manager that owns every allocation, or
inside another library's stream-ordered section).  The caller owns every buffer; the
library's per-block partials live in a static device array.  Checked through the C ABI
against bv_loglik on two calls in a row.

This file is collected last on purpose: if it fails, a run that stops at the first
failure has already run every other test."""
import numpy as np
import pytest

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
