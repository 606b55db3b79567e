"""Thin ctypes binding of the C ABI in include/bv.h (same names, argument marshalling only).

Every computation runs in the CUDA library ``_build/libbv.so``; there is no CPU fallback.
Importing this module raises if the library has not been built, and every call raises
``BVError`` on a non-OK status.  ``Context`` wraps one ``bv_ctx``.

Typical use (locations ``locs`` n x d, observations ``y``)::

    with Context() as ctx:
        ctx.set_data(locs, y)
        ctx.build_blocks(bc=n // 10, seed=0)          # K-means blocks, random order
        ctx.select_neighbors(m=60)                    # conditioning sets
        ell = ctx.loglik(theta(1.0, 0.05, 1.5, 1e-4))             # FP64
        ell32 = ctx.loglik(theta(1.0, 0.05, 1.5, 1e-4), BV_MIXED)  # mixed precision
        th, ell_hat, calls = ctx.mle(theta(1.0, 0.1, 1.5, 1e-2),   # start
                                     theta(0.01, 1e-3, 1.5, 1e-6),  # lower box
                                     theta(100, 3.0, 1.5, 10.0))    # upper box
        ctx.set_pred_locations(new_locs)              # prediction (Algorithm 2)
        ctx.build_pred_blocks(bc=len(new_locs) // 10)
        ctx.select_pred_neighbors(m=60)
        mean, var, _ = ctx.predict(th)

Many datasets: ``set_datasets`` + ``build_blocks_multi`` + ``loglik_multi`` / ``mle_multi``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbv.so")

BV_OK, BV_EINVAL, BV_ENOMEM, BV_ECUDA, BV_ENOTPD, BV_ETIMEOUT, BV_ESTATE, BV_EINTERNAL = range(8)
BV_FP64, BV_MIXED = 0, 1
BV_FREE_SIGMA2, BV_FREE_RANGE, BV_FREE_NUGGET, BV_FREE_NU = 1, 2, 4, 8
BV_NFEAT = 40
BV_MLP_NPARAM = 39046
BV_MLP_BLOB = BV_MLP_NPARAM + 2 * BV_NFEAT + 6

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} (run __graft_entry__.build())")
_lib = ctypes.CDLL(LIB_PATH)


class bv_theta(ctypes.Structure):
    _fields_ = [("sigma2", ctypes.c_double), ("range", ctypes.c_double * 3),
                ("nu", ctypes.c_double), ("nugget", ctypes.c_double),
                ("aniso", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class bv_mle_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("max_evals", ctypes.c_int32),
                ("ftol_rel", ctypes.c_double), ("xtol", ctypes.c_double),
                ("init_step", ctypes.c_double), ("init_step_nugget", ctypes.c_double),
                ("newton_first", ctypes.c_int32), ("reserved", ctypes.c_int32)]


def theta(sigma2=1.0, beta=0.1, nu=0.5, nugget=0.0, ranges=None) -> bv_theta:
    t = bv_theta()
    t.sigma2, t.nu, t.nugget = float(sigma2), float(nu), float(nugget)
    if ranges is not None:
        r = list(ranges) + [1.0] * (3 - len(ranges))
        t.aniso = 1
        for k in range(3):
            t.range[k] = float(r[k])
    else:
        t.aniso = 0
        t.range[0] = float(beta)
        t.range[1] = t.range[2] = float(beta)
    return t


def theta_tuple(t: bv_theta):
    return dict(sigma2=t.sigma2, range=list(t.range), nu=t.nu, nugget=t.nugget, aniso=t.aniso)


_P = ctypes.POINTER
_d, _f, _i64, _i32, _u64, _u32, _int, _vp = (ctypes.c_double, ctypes.c_float, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint32,
                                             ctypes.c_int, ctypes.c_void_p)

_SIGS = {
    "bv_create": (_int, [_P(_vp), _int, _vp]),
    "bv_destroy": (None, [_vp]),
    "bv_strerror": (ctypes.c_char_p, [_int]),
    "bv_last_cuda_error": (ctypes.c_char_p, []),
    "bv_set_data": (_int, [_vp, _P(_d), _P(_d), _i64, _i32]),
    "bv_set_datasets": (_int, [_vp, _i32, _P(_i64), _P(_d), _P(_d), _i32]),
    "bv_set_observations": (_int, [_vp, _vp, _i32]),
    "bv_build_blocks": (_int, [_vp, _i64, _u64, _i32, _P(_i64), _P(_i32), _P(_i64)]),
    "bv_order_blocks": (_int, [_vp, _i32, _u64, _P(_i64), _P(_i32)]),
    "bv_build_singletons": (_int, [_vp, _u64, _P(_i64), _P(_i32)]),
    "bv_build_blocks_multi": (_int, [_vp, _P(_i64), _u64, _i32, _P(_i64)]),
    "bv_set_blocks": (_int, [_vp, _i64, _P(_i64), _P(_i32), _P(_d)]),
    "bv_select_neighbors": (_int, [_vp, _i32, _P(_i32), _P(_i64), _P(_i32)]),
    "bv_set_neighbors": (_int, [_vp, _P(_i64), _P(_i32)]),
    "bv_get_sizes": (_int, [_vp, _P(_i64), _P(_i64)]),
    "bv_get_blocks": (_int, [_vp, _P(_i64), _P(_i32), _P(_d)]),
    "bv_get_neighbors": (_int, [_vp, _P(_i64), _P(_i32)]),
    "bv_loglik": (_int, [_vp, _P(bv_theta), _i32, _P(_d), _P(_d)]),
    "bv_loglik_terms": (_int, [_vp, _P(bv_theta), _i32, _P(_d), _P(_d), _P(_d)]),
    "bv_exact_loglik": (_int, [_vp, _P(bv_theta), _i32, _P(_d), _P(_d), _P(_d)]),
    "bv_exact_flops": (_int, [_i64, _P(_d)]),
    "bv_kl_divergence": (_int, [_vp, _P(bv_theta), _i32, _P(_d), _P(_d), _P(_d)]),
    "bv_loglik_terms_multi": (_int, [_vp, _P(bv_theta), _i32, _P(_d), _P(_d)]),
    "bv_mle_multi": (_int, [_vp, _P(bv_theta), _P(bv_theta), _P(bv_theta), _u32, _P(bv_mle_opts),
                            _P(bv_theta), _P(_d), _P(_i32), _P(_i32), _P(_i32)]),
    "bv_warmstart_predict_multi": (_int, [_vp, _P(bv_theta), _P(bv_theta)]),
    "bv_loglik_multi": (_int, [_vp, _P(bv_theta), _i32, _P(_d)]),
    "bv_loglik_async": (_int, [_vp, _P(bv_theta), _i32, _vp]),
    "bv_sync": (_int, [_vp, _P(_i64)]),
    "bv_last_error_block": (_int, [_vp, _P(_i64)]),
    "bv_mixed_fallbacks": (_int, [_vp, _P(_i64)]),
    "bv_mixed_check_info": (_int, [_vp, _P(_i64), _P(_i32), _P(_d)]),
    "bv_set_mixed_tolerance": (_int, [_vp, _d]),
    "bv_mixed_block_indicator": (_int, [_vp, _P(_f)]),
    "bv_loglik_noalloc": (_int, [_P(bv_theta), _vp, _vp, _i64, _i32, _i64, _vp, _vp, _vp, _vp,
                                 _vp, _vp, _vp]),
    "bv_autotune": (_int, [_vp, _i32]),
    "bv_plan_info": (_int, [_vp, _i32, _P(_i32), _P(_i32), _P(_d), _P(_d)]),
    "bv_matern_check": (_int, [_d, _i32, _i64, _P(_d), _P(_d)]),
    "bv_exp_neg_check": (_int, [_i64, _P(_d), _P(_d)]),
    "bv_exp_neg32_check": (_int, [_i64, _P(_f), _P(_f), _P(_f)]),
    "bv_mle_check": (_int, [_P(_d), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32,
                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "bv_tc_update_check": (_int, [_P(_f), _P(_f), _P(_f), _P(_f)]),
    "bv_simulate": (_int, [_vp, _P(bv_theta), _P(_d), _P(_d)]),
    "bv_mle": (_int, [_vp, _P(bv_theta), _P(bv_theta), _P(bv_theta), _u32, _P(bv_mle_opts),
                      _P(bv_theta), _P(_d), _P(_i32)]),
    "bv_set_pred_locations": (_int, [_vp, _P(_d), _P(_d), _i64]),
    "bv_build_pred_blocks": (_int, [_vp, _i64, _u64, _i32, _P(_i64), _P(_i32), _P(_i64)]),
    "bv_select_pred_neighbors": (_int, [_vp, _i32, _P(_i64), _P(_i32)]),
    "bv_get_pred_sizes": (_int, [_vp, _P(_i64), _P(_i64), _P(_i64), _P(_i64)]),
    "bv_predict": (_int, [_vp, _P(bv_theta), _P(_d), _P(_d), _P(_d)]),
    "bv_cond_sim": (_int, [_vp, _i32, _u64, _d, _P(_d), _P(_d), _P(_i64)]),
    "bv_pred_plan_info": (_int, [_vp, _P(_d), _P(_d)]),
    "bv_features": (_int, [_vp, _i32, _u64, _P(_f)]),
    "bv_mlp_train": (_int, [_P(_f), _P(_f), _i64, _i32, _i32, _f, _u64, _P(_f), _P(_f)]),
    "bv_mlp_forward": (_int, [_P(_f), _P(_f), _i64, _P(_f)]),
    "bv_mlp_loss_grad": (_int, [_P(_f), _P(_f), _P(_f), _i64, _P(_f), _P(_f)]),
    "bv_warmstart_load": (_int, [_vp, ctypes.c_char_p]),
    "bv_warmstart_predict": (_int, [_vp, _P(bv_theta), _P(bv_theta)]),
}

for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.restype = _res
    _fn.argtypes = _args

EXPORTED = tuple(_SIGS)


BV_NOALLOC_MAX_BLOCKS = 1048576


def loglik_noalloc(th: bv_theta, d_locs: int, d_y: int, n: int, d: int, bc: int, d_block_ptr: int,
                   d_point_idx: int, d_nn_ptr: int, d_nn_idx: int, d_out: int,
                   d_out_per_block: int | None = None, stream: int | None = None) -> int:
    """bv_loglik_noalloc on caller-owned device buffers (raw device pointers); returns the
    status (BV_OK or BV_ENOTPD), raises on any other."""
    st = _lib.bv_loglik_noalloc(ctypes.byref(th), d_locs, d_y, n, d, bc, d_block_ptr, d_point_idx,
                                d_nn_ptr, d_nn_idx, d_out, d_out_per_block, stream)
    return _check(st, "bv_loglik_noalloc", allow=(BV_ENOTPD,))


def mlp_train(X, T, epochs=100, batch=256, lr=1e-3, seed=0):
    """Train the warm-start MLP on the GPU; returns (blob, per-epoch losses)."""
    Xv, Tv = _arr(X, np.float32), _arr(T, np.float32)
    blob = np.empty(BV_MLP_BLOB, np.float32)
    losses = np.empty(epochs, np.float32)
    _check(_lib.bv_mlp_train(_p(Xv, _f), _p(Tv, _f), len(Xv), epochs, batch, lr, seed,
                             _p(blob, _f), _p(losses, _f)), "bv_mlp_train")
    return blob, losses


def mlp_forward(blob, X):
    b, Xv = _arr(blob, np.float32), _arr(X, np.float32)
    out = np.empty((len(Xv), 6), np.float32)
    _check(_lib.bv_mlp_forward(_p(b, _f), _p(Xv, _f), len(Xv), _p(out, _f)), "bv_mlp_forward")
    return out


def mlp_loss_grad(blob, X, T):
    b, Xv, Tv = _arr(blob, np.float32), _arr(X, np.float32), _arr(T, np.float32)
    loss = ctypes.c_float(0)
    g = np.empty(BV_MLP_NPARAM, np.float32)
    _check(_lib.bv_mlp_loss_grad(_p(b, _f), _p(Xv, _f), _p(Tv, _f), len(Xv), ctypes.byref(loss),
                                 _p(g, _f)), "bv_mlp_loss_grad")
    return loss.value, g


def save_blob(path, blob):
    """Weights file for bv_warmstart_load: 16-byte header then the floats."""
    b = _arr(blob, np.float32)
    with open(path, "wb") as f:
        f.write(b"BVWS" + np.array([1, b.size, 0], np.int32).tobytes() + b.tobytes())


def exact_flops(n):
    f = ctypes.c_double(0)
    _check(_lib.bv_exact_flops(int(n), ctypes.byref(f)), "bv_exact_flops")
    return f.value


def matern_check(nu, x, tabulated=False):
    """Device Matern correlation at scaled distances x (test support)."""
    xv = _arr(x, np.float64)
    out = np.empty_like(xv)
    _check(_lib.bv_matern_check(float(nu), 1 if tabulated else 0, xv.size, _p(xv, _d), _p(out, _d)),
           "bv_matern_check")
    return out


def tc_update_check(C, XI, XJ):
    """C - XI XJ^T (16 x 16 FP32 tiles) by the mixed kernel's tensor-core tile update."""
    a = [_arr(v, np.float32).reshape(16, 16) for v in (C, XI, XJ)]
    out = np.empty((16, 16), np.float32)
    _check(_lib.bv_tc_update_check(_p(a[0], _f), _p(a[1], _f), _p(a[2], _f), _p(out, _f)), "bv_tc_update_check")
    return out


def exp_neg_check(x):
    """The library's device FP64 e^{-x} for an array x >= 0 (diagnostic)."""
    xv = _arr(x, np.float64)
    out = np.empty_like(xv)
    _check(_lib.bv_exp_neg_check(xv.size, _p(xv, _d), _p(out, _d)), "bv_exp_neg_check")
    return out


def mle_check(model, th0, lo, hi, free_mask=None, precision=None, max_evals=2000, ftol_rel=1e-10, xtol=1e-7,
              init_step=0.5, init_step_nugget=0.0, newton_first=True):
    """bv_mle's search on the host-evaluated synthetic likelihood of bv_mle_check:
    (theta_hat, loglik_hat, evaluations, status)."""
    free_mask = BV_FREE_SIGMA2 | BV_FREE_RANGE | BV_FREE_NUGGET if free_mask is None else free_mask
    precision = BV_FP64 if precision is None else precision
    mv = _arr(model, np.float64)
    o = bv_mle_opts(precision, max_evals, ftol_rel, xtol, init_step, init_step_nugget, int(newton_first), 0)
    out = bv_theta()
    ll = ctypes.c_double(0.0)
    ne = ctypes.c_int32(0)
    st = _lib.bv_mle_check(_p(mv, _d), ctypes.byref(th0), ctypes.byref(lo), ctypes.byref(hi), free_mask,
                           ctypes.byref(o), ctypes.byref(out), ctypes.byref(ll), ctypes.byref(ne))
    return out, ll.value, ne.value, st


def exp_neg32_check(x):
    """(own, lib): the mixed kernels' device FP32 e^{-x} and CUDA's expf(-x) for x >= 0."""
    xv = _arr(x, np.float32)
    own, lib = np.empty_like(xv), np.empty_like(xv)
    _check(_lib.bv_exp_neg32_check(xv.size, _p(xv, _f), _p(own, _f), _p(lib, _f)), "bv_exp_neg32_check")
    return own, lib


class BVError(RuntimeError):
    def __init__(self, status, where):
        msg = _lib.bv_strerror(status).decode()
        if status == BV_ECUDA:
            msg += ": " + _lib.bv_last_cuda_error().decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _check(st, where, allow=()):
    if st != BV_OK and st not in allow:
        raise BVError(st, where)
    return st


def _p(a, ct):
    return None if a is None else a.ctypes.data_as(_P(ct))


def _arr(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class Context:
    """One bv_ctx on a CUDA device (its own stream unless `stream` is given)."""

    def __init__(self, device: int = 0, stream: int | None = None):
        h = _vp()
        _check(_lib.bv_create(ctypes.byref(h), device, stream), "bv_create")
        self.h = h
        self.n = 0
        self.d = 0
        self.ndata = 0

    def close(self):
        if self.h:
            _lib.bv_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # data -----------------------------------------------------------------------------
    def set_data(self, locs, y=None):
        locs = _arr(locs, np.float64)
        n, d = locs.shape
        yv = None if y is None else _arr(y, np.float64)
        _check(_lib.bv_set_data(self.h, _p(locs, _d), _p(yv, _d), n, d), "bv_set_data")
        self.n, self.d, self.ndata = n, d, 1

    def set_datasets(self, locs_list, y_list=None):
        n_per = np.array([len(l) for l in locs_list], np.int64)
        locs = _arr(np.concatenate(locs_list), np.float64)
        d = locs.shape[1]
        yv = None if y_list is None else _arr(np.concatenate(y_list), np.float64)
        _check(_lib.bv_set_datasets(self.h, len(locs_list), _p(n_per, _i64), _p(locs, _d),
                                    _p(yv, _d), d), "bv_set_datasets")
        self.n, self.d, self.ndata = int(n_per.sum()), d, len(locs_list)

    def set_observations(self, y=None, device_ptr: int | None = None):
        if device_ptr is not None:
            _check(_lib.bv_set_observations(self.h, device_ptr, 1), "bv_set_observations")
        else:
            yv = _arr(y, np.float64)
            _check(_lib.bv_set_observations(self.h, yv.ctypes.data, 0), "bv_set_observations")

    # preprocessing ------------------------------------------------------------------------
    ORDERS = {"random": 0, "maxmin": 1, "morton": 2, "kdtree": 3, "hilbert": 4}

    def order_blocks(self, order, seed=0):
        """Reorder the blocks by a rule on their centroids: (block_ptr, point_idx)."""
        o = self.ORDERS[order] if isinstance(order, str) else int(order)
        nb, _ = self.sizes()
        bp = np.empty(nb + 1, np.int64)
        pi = np.empty(self.n, np.int32)
        _check(_lib.bv_order_blocks(self.h, o, seed, _p(bp, _i64), _p(pi, _i32)), "bv_order_blocks")
        return bp, pi

    def build_singletons(self, seed=0):
        """Classic Vecchia structure: (block_ptr, point_idx) of n singleton blocks."""
        bp = np.empty(self.n + 1, np.int64)
        pi = np.empty(self.n, np.int32)
        _check(_lib.bv_build_singletons(self.h, seed, _p(bp, _i64), _p(pi, _i32)), "bv_build_singletons")
        return bp, pi

    def build_blocks(self, bc, seed=0, iters=20):
        bp = np.empty(bc + 1, np.int64)
        pi = np.empty(self.n, np.int32)
        nb = ctypes.c_int64(0)
        _check(_lib.bv_build_blocks(self.h, bc, seed, iters, _p(bp, _i64), _p(pi, _i32),
                                    ctypes.byref(nb)), "bv_build_blocks")
        return bp[:nb.value + 1].copy(), pi

    def build_blocks_multi(self, bc_per, seed=0, iters=20):
        bc = _arr(bc_per, np.int64)
        out = np.empty(len(bc), np.int64)
        _check(_lib.bv_build_blocks_multi(self.h, _p(bc, _i64), seed, iters, _p(out, _i64)),
               "bv_build_blocks_multi")
        return out

    def set_blocks(self, block_ptr, point_idx, centroids=None):
        bp = _arr(block_ptr, np.int64)
        pi = _arr(point_idx, np.int32)
        ce = None if centroids is None else _arr(centroids, np.float64)
        _check(_lib.bv_set_blocks(self.h, len(bp) - 1, _p(bp, _i64), _p(pi, _i32), _p(ce, _d)),
               "bv_set_blocks")

    def select_neighbors(self, m, m_per_block=None):
        nb, _ = self.sizes()
        mp = None if m_per_block is None else _arr(m_per_block, np.int32)
        nnp = np.empty(nb + 1, np.int64)
        _check(_lib.bv_select_neighbors(self.h, int(m), _p(mp, _i32), _p(nnp, _i64), None),
               "bv_select_neighbors")
        return self.neighbors()

    def set_neighbors(self, nn_ptr, nn_idx):
        nnp = _arr(nn_ptr, np.int64)
        nni = _arr(nn_idx, np.int32) if len(nn_idx) else np.zeros(1, np.int32)
        _check(_lib.bv_set_neighbors(self.h, _p(nnp, _i64), _p(nni, _i32)), "bv_set_neighbors")

    def sizes(self):
        nb, nn = ctypes.c_int64(0), ctypes.c_int64(0)
        _check(_lib.bv_get_sizes(self.h, ctypes.byref(nb), ctypes.byref(nn)), "bv_get_sizes")
        return nb.value, nn.value

    def blocks(self):
        nb, _ = self.sizes()
        bp = np.empty(nb + 1, np.int64)
        pi = np.empty(self.n, np.int32)
        ce = np.empty((nb, self.d), np.float64)
        _check(_lib.bv_get_blocks(self.h, _p(bp, _i64), _p(pi, _i32), _p(ce, _d)), "bv_get_blocks")
        return bp, pi, ce

    def neighbors(self):
        nb, nn = self.sizes()
        nnp = np.empty(nb + 1, np.int64)
        nni = np.empty(max(nn, 1), np.int32)
        _check(_lib.bv_get_neighbors(self.h, _p(nnp, _i64), _p(nni, _i32)), "bv_get_neighbors")
        return nnp, nni[:nn].copy()

    # evaluation -------------------------------------------------------------------------
    def loglik(self, th: bv_theta, precision=BV_FP64, per_block=False, allow_notpd=False):
        out = ctypes.c_double(0.0)
        nb, _ = self.sizes()
        per = np.empty(nb, np.float64) if per_block else None
        st = _check(_lib.bv_loglik(self.h, ctypes.byref(th), precision, ctypes.byref(out),
                                   _p(per, _d)), "bv_loglik",
                    allow=(BV_ENOTPD,) if allow_notpd else ())
        if per_block:
            return out.value, per, st
        return out.value

    # ---- prediction (Algorithm 2) ----
    def set_pred_locations(self, locs_star, y_true=None):
        ls = _arr(locs_star, np.float64)
        yt = _arr(y_true, np.float64) if y_true is not None else None
        _check(_lib.bv_set_pred_locations(self.h, _p(ls, _d), _p(yt, _d), ls.shape[0]), "bv_set_pred_locations")
        self.n_star = ls.shape[0]

    def build_pred_blocks(self, bc, seed=0, iters=20):
        bp = np.empty(bc + 1, np.int64)
        pi = np.empty(self.n_star, np.int32)
        nb = ctypes.c_int64(0)
        _check(_lib.bv_build_pred_blocks(self.h, bc, seed, iters, _p(bp, _i64), _p(pi, _i32), ctypes.byref(nb)),
               "bv_build_pred_blocks")
        return bp[:nb.value + 1].copy(), pi

    def pred_sizes(self):
        v = [ctypes.c_int64(0) for _ in range(4)]
        _check(_lib.bv_get_pred_sizes(self.h, *[ctypes.byref(x) for x in v]), "bv_get_pred_sizes")
        return tuple(x.value for x in v)

    def select_pred_neighbors(self, m):
        _check(_lib.bv_select_pred_neighbors(self.h, int(m), None, None), "bv_select_pred_neighbors")
        _, nb, nn, _ = self.pred_sizes()
        nnp = np.empty(nb + 1, np.int64)
        nni = np.empty(max(nn, 1), np.int32)
        _check(_lib.bv_select_pred_neighbors(self.h, int(m), _p(nnp, _i64), _p(nni, _i32)),
               "bv_select_pred_neighbors")
        return nnp, nni[:nn].copy()

    def predict(self, th: bv_theta, want=("mean", "var"), packed_cov=False, allow_notpd=False):
        """(mean, var, packed covariance or None); want=() keeps results on the device."""
        ns, _, _, ncov = self.pred_sizes()
        mean = np.empty(ns) if "mean" in want else None
        var = np.empty(ns) if "var" in want else None
        cov = np.empty(max(ncov, 1)) if packed_cov else None
        _check(_lib.bv_predict(self.h, ctypes.byref(th), _p(mean, _d), _p(var, _d), _p(cov, _d)), "bv_predict",
               allow=(BV_ENOTPD,) if allow_notpd else ())
        return mean, var, (cov[:ncov] if cov is not None else None)

    def cond_sim(self, rounds=1000, seed=0, z_crit=1.959963984540054, bounds=True):
        """(lower, upper, covered); covered is -1 without held-out values."""
        ns = self.pred_sizes()[0]
        lo = np.empty(ns) if bounds else None
        up = np.empty(ns) if bounds else None
        cov = ctypes.c_int64(0)
        _check(_lib.bv_cond_sim(self.h, int(rounds), seed, float(z_crit), _p(lo, _d), _p(up, _d),
                                ctypes.byref(cov)), "bv_cond_sim")
        return lo, up, cov.value

    def pred_plan_info(self):
        f, e = ctypes.c_double(0), ctypes.c_double(0)
        _check(_lib.bv_pred_plan_info(self.h, ctypes.byref(f), ctypes.byref(e)), "bv_pred_plan_info")
        return f.value, e.value

    def exact_loglik(self, th: bv_theta, use_y=True):
        """Eq. 1 by a dense device Cholesky: (ell, quad, logdet)."""
        l, q, d = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        _check(_lib.bv_exact_loglik(self.h, ctypes.byref(th), 1 if use_y else 0, ctypes.byref(l),
                                    ctypes.byref(q), ctypes.byref(d)), "bv_exact_loglik")
        return l.value, q.value, d.value

    def kl_divergence(self, th: bv_theta, precision=BV_FP64):
        """(KL, logdet exact, logdet approximate) of the current blocks/neighbours."""
        k, a, b = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        _check(_lib.bv_kl_divergence(self.h, ctypes.byref(th), precision, ctypes.byref(k), ctypes.byref(a),
                                     ctypes.byref(b)), "bv_kl_divergence")
        return k.value, a.value, b.value

    def mixed_check_info(self):
        """(blocks whose terms came from FP64, datasets with blocks recomputed beyond the
        sample, per-dataset bound on the relative error) of the last mixed evaluation."""
        nb = ctypes.c_int64(0)
        nd = ctypes.c_int32(0)
        est = np.zeros(max(self.ndata, 1), np.float64)
        _check(_lib.bv_mixed_check_info(self.h, ctypes.byref(nb), ctypes.byref(nd), _p(est, _d)),
               "bv_mixed_check_info")
        return nb.value, nd.value, est[:self.ndata]

    def set_mixed_tolerance(self, tol: float):
        _check(_lib.bv_set_mixed_tolerance(self.h, float(tol)), "bv_set_mixed_tolerance")

    def mixed_block_indicator(self):
        nb, _ = self.sizes()
        out = np.empty(nb, np.float32)
        _check(_lib.bv_mixed_block_indicator(self.h, _p(out, _f)), "bv_mixed_block_indicator")
        return out

    def mixed_fallbacks(self):
        """Blocks recomputed in FP64 in the last mixed-precision evaluation."""
        b = ctypes.c_int64(0)
        _check(_lib.bv_mixed_fallbacks(self.h, ctypes.byref(b)), "bv_mixed_fallbacks")
        return b.value

    def last_error_block(self):
        """First failing block of the last synchronous evaluation, or -1."""
        b = ctypes.c_int64(0)
        _check(_lib.bv_last_error_block(self.h, ctypes.byref(b)), "bv_last_error_block")
        return b.value

    def loglik_terms(self, th: bv_theta, precision=BV_FP64):
        """(ell, quad, logdet) with ell = -(quad + logdet + n log 2 pi) / 2."""
        l, q, d = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
        _check(_lib.bv_loglik_terms(self.h, ctypes.byref(th), precision, ctypes.byref(l), ctypes.byref(q),
                                    ctypes.byref(d)), "bv_loglik_terms")
        return l.value, q.value, d.value

    def loglik_multi(self, thetas, precision=BV_FP64, allow_notpd=False):
        arr = (bv_theta * len(thetas))(*thetas)
        out = np.empty(len(thetas), np.float64)
        _check(_lib.bv_loglik_multi(self.h, arr, precision, _p(out, _d)), "bv_loglik_multi",
               allow=(BV_ENOTPD,) if allow_notpd else ())
        return out

    def loglik_async(self, thetas, precision, d_out_ptr: int):
        arr = (bv_theta * len(thetas))(*thetas)
        _check(_lib.bv_loglik_async(self.h, arr, precision, d_out_ptr), "bv_loglik_async")

    def sync(self):
        fb = ctypes.c_int64(-1)
        st = _lib.bv_sync(self.h, ctypes.byref(fb))
        return st, fb.value

    def autotune(self, precision=BV_FP64):
        _check(_lib.bv_autotune(self.h, precision), "bv_autotune")

    def plan_info(self, precision=BV_FP64):
        la, nb = ctypes.c_int32(0), ctypes.c_int32(0)
        fl, en = ctypes.c_double(0.0), ctypes.c_double(0.0)
        _check(_lib.bv_plan_info(self.h, precision, ctypes.byref(la), ctypes.byref(nb),
                                 ctypes.byref(fl), ctypes.byref(en)), "bv_plan_info")
        return dict(launches_per_eval=la.value, n_bins=nb.value, flops=fl.value,
                    cov_entries=en.value)

    # sampler / MLE / warm start ----------------------------------------------------------
    def simulate(self, th: bv_theta, z):
        zv = _arr(z, np.float64)
        y = np.empty(self.n, np.float64)
        _check(_lib.bv_simulate(self.h, ctypes.byref(th), _p(zv, _d), _p(y, _d)), "bv_simulate")
        return y

    def mle(self, th0: bv_theta, lo: bv_theta, hi: bv_theta,
            free_mask=BV_FREE_SIGMA2 | BV_FREE_RANGE | BV_FREE_NUGGET, precision=BV_FP64,
            max_evals=2000, ftol_rel=1e-10, xtol=1e-7, init_step=0.5, init_step_nugget=0.0, newton_first=True):
        o = bv_mle_opts(precision, max_evals, ftol_rel, xtol, init_step, init_step_nugget, int(newton_first), 0)
        out = bv_theta()
        ll = ctypes.c_double(0.0)
        ne = ctypes.c_int32(0)
        _check(_lib.bv_mle(self.h, ctypes.byref(th0) if th0 is not None else None, ctypes.byref(lo), ctypes.byref(hi),
                           free_mask, ctypes.byref(o), ctypes.byref(out), ctypes.byref(ll),
                           ctypes.byref(ne)), "bv_mle")
        return out, ll.value, ne.value

    def mle_multi(self, th0, lo: bv_theta, hi: bv_theta,
                  free_mask=BV_FREE_SIGMA2 | BV_FREE_RANGE | BV_FREE_NUGGET, precision=BV_FP64,
                  max_evals=2000, ftol_rel=1e-10, xtol=1e-7, init_step=0.5, init_step_nugget=0.0,
                  newton_first=True):
        """Every dataset's MLE with batched evaluations: (thetas, logliks, evals, statuses, batches).
        th0: a list of starts (one per dataset) or None for the learned warm start."""
        nd = self.ndata
        o = bv_mle_opts(precision, max_evals, ftol_rel, xtol, init_step, init_step_nugget, int(newton_first), 0)
        starts = (bv_theta * nd)(*th0) if th0 is not None else None
        out = (bv_theta * nd)()
        ll = np.empty(nd)
        ne = np.empty(nd, np.int32)
        st = np.empty(nd, np.int32)
        nb = ctypes.c_int32(0)
        _check(_lib.bv_mle_multi(self.h, starts, ctypes.byref(lo), ctypes.byref(hi), free_mask, ctypes.byref(o),
                                 out, _p(ll, _d), _p(ne, _i32), _p(st, _i32), ctypes.byref(nb)), "bv_mle_multi")
        return list(out), ll, ne, st, nb.value

    def loglik_terms_multi(self, thetas, precision=BV_FP64):
        """(ell[ndata], quad[ndata])."""
        arr = (bv_theta * self.ndata)(*thetas)
        ll = np.empty(self.ndata)
        q = np.empty(self.ndata)
        _check(_lib.bv_loglik_terms_multi(self.h, arr, precision, _p(ll, _d), _p(q, _d)), "bv_loglik_terms_multi")
        return ll, q

    def features(self, max_points=10000, seed=0):
        out = np.empty((self.ndata, BV_NFEAT), np.float32)
        _check(_lib.bv_features(self.h, max_points, seed, _p(out, _f)), "bv_features")
        return out

    def warmstart_load(self, path: str):
        _check(_lib.bv_warmstart_load(self.h, path.encode()), "bv_warmstart_load")

    def warmstart_predict(self, th_in: bv_theta):
        out = bv_theta()
        _check(_lib.bv_warmstart_predict(self.h, ctypes.byref(th_in), ctypes.byref(out)),
               "bv_warmstart_predict")
        return out
