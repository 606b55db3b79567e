"""GPU: each kernel form the autotuner can choose for a size bin -- one CTA per block (in
FP64 with one- or two-column factorisation steps), or one warp per block (FP64 up to
N = 64, mixed up to N = 128), or the tensor-core mixed kernel -- forced in turn through
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


@pytest.mark.parametrize("form", ["cta", "cta2", "warp"])
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
    # the oracle builds its own structure; the GPU's must equal it bit for bit
    if singletons:
        obp, opi, oce = oracle.build_singletons(locs, seed=seed)
    else:
        obp, opi, oce = oracle.build_blocks(locs, bc, seed=seed, iters=20)
    onnp, onni = oracle.select_neighbors(locs, obp, opi, oce, m)
    for a, b in zip(gs, (obp, opi, onnp, onni)):
        np.testing.assert_array_equal(a, b)
    ref, per_ref, _ = oracle.loglik(oth, locs, y, obp, opi, onnp, onni)
    assert abs(ll64 - ref) <= REL64 * abs(ref), (form, ll64, ref)
    np.testing.assert_allclose(per64, per_ref, rtol=1e-9, atol=1e-9)
    assert abs(llm - ref) <= 1e-6 * abs(ref), (form, llm, ref, abs(llm - ref))


def test_tensor_core_tile_update_matches_fp64():
    # the mixed kernel's tensor-core tile update C - XI XJ^T (three-part BF16 split, six
    # products, FP32 accumulation) against FP64: within a few FP32 roundings of the terms
    from paper_2410_04477_gb300 import bv
    rng = np.random.default_rng(7)
    for scale in (1.0, 1e-3, 37.0):
        C = rng.standard_normal((16, 16)).astype(np.float32) * np.float32(scale)
        XI = rng.standard_normal((16, 16)).astype(np.float32)
        XJ = rng.standard_normal((16, 16)).astype(np.float32)
        got = bv.tc_update_check(C, XI, XJ).astype(np.float64)
        want = C.astype(np.float64) - XI.astype(np.float64) @ XJ.astype(np.float64).T
        mag = np.abs(C).astype(np.float64) + np.abs(XI).astype(np.float64) @ np.abs(XJ).astype(np.float64).T
        err = np.abs(got - want) / mag
        assert err.max() <= 8 * 2.0 ** -24, (scale, err.max())
    # exact on values that BF16 parts represent exactly
    C = np.arange(256, dtype=np.float32).reshape(16, 16)
    XI = (np.arange(256) % 7 - 3).astype(np.float32).reshape(16, 16)
    XJ = (np.arange(256) % 5 - 2).astype(np.float32).reshape(16, 16)
    np.testing.assert_array_equal(bv.tc_update_check(C, XI, XJ), C - XI @ XJ.T)


@pytest.mark.parametrize("case", [
    # (n, d, singletons, bc, m, theta, ranges): N from 64 to about 215, ragged last tiles
    (3000, 2, False, 300, 120, (1.0, 0.1, 1.5, 1e-3), None),
    (2500, 3, False, 250, 200, (1.0, None, 0.5, 1e-3), [0.1, 0.1, 0.3]),
    (3000, 2, False, 300, 70, (0.8, 0.07, 1.2, 1e-2), None),    # general nu
    (1200, 2, True, 0, 63, (1.0, 0.1, 0.5, 1e-2), None),       # N = 64: the last tile row holds only y
    (1200, 2, True, 0, 78, (1.0, 0.1, 2.5, 1e-2), None),       # N = 79: R = 80 fills the last tile
])
def test_tensor_core_form_matches_oracle(bv, case, monkeypatch):
    n, d, singletons, bc, m, th, ranges = case
    monkeypatch.setenv("BV_KERNEL_FORM", "tc")
    seed = 130 + m
    locs = synth.locs_uniform(n, d, seed)
    oth = oracle.theta(*th, ranges=ranges)
    y = oracle.exact_draw(oth, locs, synth.normal(seed, 20, n))
    gth = bv.theta(*th, ranges=ranges)
    with bv.Context() as ctx:
        ctx.set_data(locs, y)
        if singletons:
            bp, pi = ctx.build_singletons(seed=seed)
        else:
            bp, pi = ctx.build_blocks(bc, seed=seed, iters=20)
        nnp, nni = ctx.select_neighbors(m)
        ctx.set_mixed_tolerance(0.0)          # FP32 throughout: the kernel's own arithmetic
        ll32, per32, _ = ctx.loglik(gth, bv.BV_MIXED, per_block=True)
        nfb = ctx.mixed_fallbacks()
        w = ctx.mixed_block_indicator().astype(np.float64)
        ctx.set_mixed_tolerance(1e-6)
        llm = ctx.loglik(gth, bv.BV_MIXED)
        info = ctx.plan_info(bv.BV_MIXED)
    if singletons:
        obp, opi, oce = oracle.build_singletons(locs, seed=seed)
    else:
        obp, opi, oce = oracle.build_blocks(locs, bc, seed=seed, iters=20)
    onnp, onni = oracle.select_neighbors(locs, obp, opi, oce, m)
    for a, b in zip((bp, pi, nnp, nni), (obp, opi, onnp, onni)):
        np.testing.assert_array_equal(a, b)
    ref, per_ref, _ = oracle.loglik(oth, locs, y, obp, opi, onnp, onni)
    Ns = np.diff(bp) + np.diff(nnp)
    print(f"tc form N {Ns.min()}..{Ns.max()}: unchecked rel {abs(ll32 - ref) / abs(ref):.2e}, "
          f"checked rel {abs(llm - ref) / abs(ref):.2e}, fallbacks {nfb}")
    assert Ns.max() >= 64
    ok = np.isfinite(per32)
    assert ok.all() or nfb > 0
    # every block within the FP32 error its weight predicts (measured |delta_i| / (eps w_i)
    # stays below about 5 on the benchmark workloads)
    err = np.abs(per32 - per_ref)
    assert np.all(err <= 8.0 * 2.0 ** -24 * w + 1e-9), (err / (2.0 ** -24 * np.maximum(w, 1e-30))).max()
    assert abs(ll32 - ref) <= 1e-4 * abs(ref)
    assert abs(llm - ref) <= 1e-6 * abs(ref)
