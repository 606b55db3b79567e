"""Error conventions of the C ABI on the GPU path: parameters outside their domain and
non-finite observations return BV_EINVAL without touching the context; a failed device
allocation returns BV_ENOMEM and leaves the context usable; a non-positive-definite block
returns BV_ENOTPD with ell = -inf and names the block.  The allocation failure is made on
the host (the library's allocation fault switch, BV_FAULT_ALLOC), never on the device."""
import ctypes
import os

import numpy as np
import pytest

import oracle
from paper_2410_04477_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bv():
    import torch
    assert torch.cuda.is_available()
    from paper_2410_04477_gb300 import bv as _bv
    return _bv


@pytest.fixture(scope="module")
def case():
    n, bc, m = 1500, 150, 30
    locs = synth.locs_uniform(n, 2, 301)
    th = (1.1, 0.08, 1.5, 1e-3)
    y = oracle.exact_draw(oracle.theta(*th), locs, synth.normal(301, 20, n))
    bp, pi, ce = oracle.build_blocks(locs, bc, seed=3)
    nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
    ell = oracle.loglik(oracle.theta(*th), locs, y, bp, pi, nnp, nni)[0]
    return dict(locs=locs, y=y, bc=bc, m=m, th=th, ell=ell)


def _ctx(bv, case):
    ctx = bv.Context()
    ctx.set_data(case["locs"], case["y"])
    ctx.build_blocks(case["bc"], seed=3)
    ctx.select_neighbors(case["m"])
    return ctx


def _status(bv, ctx, th, prec=None):
    out = ctypes.c_double(0.0)
    st = bv._lib.bv_loglik(ctx.h, ctypes.byref(th), bv.BV_FP64 if prec is None else prec, ctypes.byref(out), None)
    return st, out.value


@pytest.mark.parametrize("bad", ["sigma2=0", "sigma2<0", "beta=0", "beta<0", "nugget<0", "nu=0", "nu<0",
                                 "nu>20", "sigma2=nan", "beta=inf", "aniso range<0"])
def test_theta_outside_domain_is_einval(bv, case, bad):
    s2, beta, nu, tau2 = case["th"]
    ranges = None
    if bad == "sigma2=0":
        s2 = 0.0
    elif bad == "sigma2<0":
        s2 = -1.0
    elif bad == "beta=0":
        beta = 0.0
    elif bad == "beta<0":
        beta = -0.1
    elif bad == "nugget<0":
        tau2 = -1e-6
    elif bad == "nu=0":
        nu = 0.0
    elif bad == "nu<0":
        nu = -0.5
    elif bad == "nu>20":
        nu = 20.5
    elif bad == "sigma2=nan":
        s2 = float("nan")
    elif bad == "beta=inf":
        beta = float("inf")
    else:
        ranges = [0.1, -0.1]
    with _ctx(bv, case) as ctx:
        for prec in (bv.BV_FP64, bv.BV_MIXED):
            st, _ = _status(bv, ctx, bv.theta(s2, beta, nu, tau2, ranges=ranges), prec)
            assert st == bv.BV_EINVAL, (bad, prec, st)
        # the context is untouched: the next valid call is exact
        ll = ctx.loglik(bv.theta(*case["th"]))
        assert abs(ll - case["ell"]) <= 1e-10 * abs(case["ell"])


def test_non_finite_observations_are_einval(bv, case):
    with _ctx(bv, case) as ctx:
        for v in (float("nan"), float("inf"), -float("inf")):
            y = case["y"].copy()
            y[777] = v
            with pytest.raises(bv.BVError) as e:
                ctx.set_observations(y)
            assert e.value.status == bv.BV_EINVAL
        ll = ctx.loglik(bv.theta(*case["th"]))   # observations unchanged
        assert abs(ll - case["ell"]) <= 1e-10 * abs(case["ell"])
    with bv.Context() as ctx:
        y = case["y"].copy()
        y[0] = float("nan")
        with pytest.raises(bv.BVError) as e:
            ctx.set_data(case["locs"], y)
        assert e.value.status == bv.BV_EINVAL
        locs = case["locs"].copy()
        locs[5, 1] = float("inf")
        with pytest.raises(bv.BVError) as e:
            ctx.set_data(locs, case["y"])
        assert e.value.status == bv.BV_EINVAL


def test_non_finite_device_observation_gives_notpd(bv, case):
    import torch
    with _ctx(bv, case) as ctx:
        y = torch.tensor(case["y"], dtype=torch.float64, device="cuda")
        y[10] = float("nan")
        torch.cuda.synchronize()
        ctx.set_observations(device_ptr=y.data_ptr())
        st, val = _status(bv, ctx, bv.theta(*case["th"]))
        assert st == bv.BV_ENOTPD and val == -np.inf
        ctx.set_observations(case["y"])
        ll = ctx.loglik(bv.theta(*case["th"]))
        assert abs(ll - case["ell"]) <= 1e-10 * abs(case["ell"])


@pytest.mark.parametrize("prec", [0, 1])
def test_injected_allocation_failure_is_enomem_and_recoverable(bv, case, prec):
    with _ctx(bv, case) as ctx:
        os.environ["BV_FAULT_ALLOC"] = "1"
        try:
            st, _ = _status(bv, ctx, bv.theta(*case["th"]), prec)
        finally:
            del os.environ["BV_FAULT_ALLOC"]
        assert st == bv.BV_ENOMEM
        ll = ctx.loglik(bv.theta(*case["th"]), prec)
        tol = 1e-10 if prec == bv.BV_FP64 else 1e-6
        assert abs(ll - case["ell"]) <= tol * abs(case["ell"]), (ll, case["ell"])
        # a second failure after a good plan: the first evaluation of the other
        # precision needs its own plan
        other = 1 - prec
        os.environ["BV_FAULT_ALLOC"] = "1"
        try:
            st, _ = _status(bv, ctx, bv.theta(*case["th"]), other)
        finally:
            del os.environ["BV_FAULT_ALLOC"]
        assert st == bv.BV_ENOMEM
        assert abs(ctx.loglik(bv.theta(*case["th"]), prec) - ll) == 0.0   # the good plan still works
        ll2 = ctx.loglik(bv.theta(*case["th"]), other)
        tol2 = 1e-10 if other == bv.BV_FP64 else 1e-6
        assert abs(ll2 - case["ell"]) <= tol2 * abs(case["ell"])


def test_duplicate_site_without_nugget_is_notpd_in_both_precisions(bv, case):
    # the first two points of block 0 (no conditioning set) made identical, sigma^2 = 1,
    # no nugget: the second pivot is exactly 0 in both precisions (the mixed path's FP64
    # recomputation of the block fails too)
    with bv.Context() as ctx:
        ctx.set_data(case["locs"], case["y"])
        bp, pi = ctx.build_blocks(case["bc"], seed=3)
        locs2 = case["locs"].copy()
        locs2[pi[1]] = locs2[pi[0]]
        ctx.set_data(locs2, case["y"])
        ctx.set_blocks(bp, pi)
        ctx.select_neighbors(case["m"])
        for prec in (bv.BV_FP64, bv.BV_MIXED):
            st, val = _status(bv, ctx, bv.theta(1.0, 0.1, 1.5, 0.0), prec)
            assert st == bv.BV_ENOTPD and val == -np.inf, (prec, st, val)
            assert ctx.last_error_block() == 0
        ll = ctx.loglik(bv.theta(1.0, 0.1, 1.5, 1e-3))   # a nugget restores positive definiteness
        assert ctx.last_error_block() == -1 and np.isfinite(ll)
