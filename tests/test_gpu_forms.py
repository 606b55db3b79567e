"""GPU: each kernel form the autotuner can choose for a size bin -- one CTA per block, or
one warp per block (FP64 up to N = 64, mixed up to N = 128) -- forced in turn through
BV_KERNEL_FORM and checked against the FP64 oracle on the same structure, so that a form
the timing never picks on these sizes is still tested: K-means blocks (N around 40) and
classic-Vecchia singletons (N = m + 1), closed-form and general smoothness, 2D and 3D."""
import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth

pytestmark = pytest.mark.gpu

REL64 = 1e-10


@pytest.fixture(scope="module")
def bv():
    import torch
    assert torch.cuda.is_available()
    from paper_2410_04477_gb300 import bv as _bv
    return _bv


def _run(bv, locs, y, th, singletons, bc, m, seed):
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        if singletons:
            bp, pi = ctx.build_singletons(seed=seed)
        else:
            bp, pi = ctx.build_blocks(bc, seed=seed, iters=20)
        nnp, nni = ctx.select_neighbors(m)
        ll64, per64, _ = ctx.loglik(bv.theta(*th), bv.BV_FP64, per_block=True)
        llm = ctx.loglik(bv.theta(*th), bv.BV_MIXED)
    return ll64, per64, llm, (bp, pi, nnp, nni)


@pytest.mark.parametrize("form", ["cta", "warp"])
@pytest.mark.parametrize("case", [
    # (n, d, singletons, bc, m, theta = (sigma^2, beta, nu, tau^2))
    (2000, 2, False, 200, 30, (1.0, 0.1, 1.5, 1e-3)),
    (2000, 2, False, 200, 30, (0.8, 0.07, 1.2, 1e-2)),    # general nu
    (1500, 3, False, 150, 40, (1.2, 0.1, 2.5, 1e-2)),
    (1500, 2, True, 0, 30, (1.0, 0.1, 0.5, 1e-3)),       # classic Vecchia, N = 31
])
def test_kernel_form_matches_oracle(bv, form, case, monkeypatch):
    n, d, singletons, bc, m, th = case
    monkeypatch.setenv("BV_KERNEL_FORM", form)
    seed = 90 + n % 7 + d
    locs = synth.locs_uniform(n, d, seed)
    oth = oracle.theta(*th)
    y = oracle.exact_draw(oth, locs, synth.normal(seed, 20, n))
    ll64, per64, llm, gs = _run(bv, locs, y, th, singletons, bc, m, seed)
    ref, per_ref, _ = oracle.loglik(oth, locs, y, *gs)
    assert abs(ll64 - ref) <= REL64 * abs(ref), (form, ll64, ref)
    np.testing.assert_allclose(per64, per_ref, rtol=1e-9, atol=1e-9)
    assert abs(llm - ref) <= 1e-4 * abs(ref), (form, llm, ref)
