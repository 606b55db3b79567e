"""Plain FP64 CPU oracle for the block-Vecchia log-likelihood (arXiv 2410.04477).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package.  It shares no code with the CUDA library in
``paper_2410_04477_gb300``: the arithmetic lives in ``bv_oracle.c`` (compiled here with
``gcc -O2 -ffp-contract=off -fopenmp``) and in the NumPy modules next to it.

What each function follows (details in the C source):
  matern_corr / cov       Eq. 5 (Matern), closed forms at nu = 1/2, 3/2, 5/2
  kmeans / build_blocks   Sec. 2.1 + Algorithm 1 (clustering, block permutation)
  build_singletons        classic Vecchia: blocks of size 1 in a random order (Sec. 1)
  order_blocks            the block orderings of Sec. 2.1 (random, maxmin, Morton, KD-tree,
                          Hilbert)
  select_neighbors        Sec. 2.2 + Algorithm 1 (nearest neighbours of each block)
  block_loglik / loglik   Algorithm 1 (batched steps, literally) and Eq. 4
  exact_loglik            Eq. 1
  exact_draw / bv_draw    input generators: exact GP draw, block-Vecchia draw (Eq. 4)
  build_pred_blocks / select_pred_neighbors / predict
                          Sec. 2.4 + Algorithm 2 (prediction)
  csim_normal / cond_sim  Sec. 2.4 univariate conditional simulation; PICP (Sec. 3.2)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bv_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Theta(ctypes.Structure):
    """Covariance parameters theta = (sigma^2, beta, nu) of Eq. 5, plus a nugget."""
    _fields_ = [("sigma2", ctypes.c_double), ("range", ctypes.c_double * 3),
                ("nu", ctypes.c_double), ("nugget", ctypes.c_double),
                ("aniso", ctypes.c_int32), ("pad", ctypes.c_int32)]


def theta(sigma2=1.0, beta=0.1, nu=0.5, nugget=0.0, ranges=None) -> Theta:
    t = Theta()
    t.sigma2 = float(sigma2)
    t.nu = float(nu)
    t.nugget = float(nugget)
    if ranges is not None:
        r = list(ranges) + [1.0] * (3 - len(ranges))
        t.aniso = 1
        for k in range(3):
            t.range[k] = float(r[k])
    else:
        t.aniso = 0
        t.range[0] = float(beta)
        t.range[1] = t.range[2] = 1.0
    return t


_P = ctypes.POINTER
_d, _i64, _i32, _u64, _int = ctypes.c_double, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64, ctypes.c_int


def _bind(L):
    """Declare the C signatures on a loaded oracle library."""
    if True:
        if True:
            L.or_splitmix64.restype = _u64
            L.or_splitmix64.argtypes = [_u64, _u64]
            L.or_bessel_k.restype = _d
            L.or_bessel_k.argtypes = [_d, _d]
            L.or_matern_corr.restype = _d
            L.or_matern_corr.argtypes = [_d, _d]
            L.or_cov.restype = _d
            L.or_cov.argtypes = [_P(Theta), _int, _P(_d), _P(_d), _int]
            L.or_block_loglik.restype = _d
            L.or_block_loglik.argtypes = [_P(Theta), _P(_d), _P(_d), _int, _P(_i32), _i64,
                                          _P(_i32), _i64, _P(_int)]
            L.or_loglik.restype = _int
            L.or_loglik.argtypes = [_P(Theta), _P(_d), _P(_d), _i64, _int, _i64, _P(_i64),
                                    _P(_i32), _P(_i64), _P(_i32), _P(_d), _P(_d)]
            L.or_exact_loglik.restype = _int
            L.or_exact_loglik.argtypes = [_P(Theta), _P(_d), _P(_d), _i64, _int, _P(_d)]
            L.or_exact_draw.restype = _int
            L.or_exact_draw.argtypes = [_P(Theta), _P(_d), _i64, _int, _P(_d), _P(_d)]
            L.or_bv_draw.restype = _int
            L.or_bv_draw.argtypes = [_P(Theta), _P(_d), _i64, _int, _i64, _P(_i64), _P(_i32),
                                     _P(_i64), _P(_i32), _P(_d), _P(_d)]
            L.or_kmeans.restype = _int
            L.or_kmeans.argtypes = [_P(_d), _i64, _int, _i64, _u64, _int, _P(_i32), _P(_d)]
            L.or_build_blocks.restype = _i64
            L.or_build_blocks.argtypes = [_P(_d), _i64, _int, _i64, _u64, _int, _P(_i64),
                                          _P(_i32), _P(_d)]
            L.or_select_neighbors.restype = _int
            L.or_select_neighbors.argtypes = [_P(_d), _i64, _int, _i64, _P(_i64), _P(_i32),
                                              _P(_d), _i32, _P(_i32), _P(_i64), _P(_i32)]
            L.or_build_singletons.restype = _int
            L.or_build_singletons.argtypes = [_P(_d), _i64, _int, _u64, _P(_i64), _P(_i32), _P(_d)]
            L.or_order_blocks.restype = _int
            L.or_order_blocks.argtypes = [_P(_d), _i64, _int, _int, _u64, _P(_i64)]
            L.or_hilbert_index.restype = _u64
            L.or_hilbert_index.argtypes = [_P(_u64), _int]
            L.or_build_pred_blocks.restype = _i64
            L.or_build_pred_blocks.argtypes = [_P(_d), _i64, _int, _i64, _u64, _int, _P(_i64),
                                               _P(_i32), _P(_d)]
            L.or_select_pred_neighbors.restype = _int
            L.or_select_pred_neighbors.argtypes = [_P(_d), _i64, _int, _i64, _P(_d), _i32,
                                                   _P(_i64), _P(_i32)]
            L.or_predict_block.restype = _int
            L.or_predict_block.argtypes = [_P(Theta), _P(_d), _P(_d), _int, _P(_i32), _i64,
                                           _P(_d), _P(_i32), _i64, _P(_d), _P(_d)]
            L.or_predict.restype = _int
            L.or_predict.argtypes = [_P(Theta), _P(_d), _P(_d), _i64, _int, _P(_d), _i64,
                                     _P(_i64), _P(_i32), _P(_i64), _P(_i32), _P(_d), _P(_d),
                                     _P(_d)]
            L.or_csim_normal.restype = _d
            L.or_csim_normal.argtypes = [_u64, _i64, _i32, _i32]
            L.or_cond_sim.restype = _int
            L.or_cond_sim.argtypes = [_P(_d), _P(_d), _i64, _i32, _u64, _d, _P(_d), _P(_d),
                                      _P(_d), _P(_i64)]
            L.or_num_threads.restype = _int
            L.or_num_threads.argtypes = []
            L.or_set_num_threads.restype = None
            L.or_set_num_threads.argtypes = [_int]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
        return _lib


class use_library:
    """Tests only: route this module's calls to another build of the oracle (a copy with
    a planted mistake), restoring the real one on exit."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self.saved = _lib
        _lib = _bind(ctypes.CDLL(self.path))
        return self

    def __exit__(self, *a):
        global _lib
        _lib = self.saved


def _ptr(a, ct):
    return a.ctypes.data_as(_P(ct)) if a is not None else None


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(k: int) -> None:
    """OpenMP threads for the oracle calls made from this thread from now on."""
    lib().or_set_num_threads(int(k))


def splitmix64(stream: int, counter: int) -> int:
    return int(lib().or_splitmix64(stream, counter))


def bessel_k(nu: float, x: float) -> float:
    return float(lib().or_bessel_k(nu, x))


def matern_corr(nu: float, x) -> np.ndarray:
    x = np.atleast_1d(np.asarray(x, dtype=np.float64))
    f = lib().or_matern_corr
    return np.array([f(nu, float(v)) for v in x.ravel()]).reshape(x.shape)


def cov(th: Theta, si, sj, same: bool) -> float:
    si = _c(si, np.float64)
    sj = _c(sj, np.float64)
    return float(lib().or_cov(ctypes.byref(th), si.size, _ptr(si, _d), _ptr(sj, _d), int(same)))


def kmeans(locs, k, seed, iters=20):
    locs = _c(locs, np.float64)
    n, d = locs.shape
    label = np.empty(n, np.int32)
    cent = np.empty((k, d), np.float64)
    st = lib().or_kmeans(_ptr(locs, _d), n, d, k, seed, iters, _ptr(label, _i32), _ptr(cent, _d))
    if st:
        raise OracleError(st, "kmeans")
    return label, cent


def build_blocks(locs, bc, seed, iters=20):
    """K-means blocks in the random permuted order: (block_ptr, point_idx, centroids)."""
    locs = _c(locs, np.float64)
    n, d = locs.shape
    bp = np.empty(bc + 1, np.int64)
    pi = np.empty(n, np.int32)
    ce = np.empty((bc, d), np.float64)
    nb = lib().or_build_blocks(_ptr(locs, _d), n, d, bc, seed, iters, _ptr(bp, _i64),
                               _ptr(pi, _i32), _ptr(ce, _d))
    if nb < 0:
        raise OracleError(-nb, "build_blocks")
    return bp[:nb + 1].copy(), pi, ce[:nb].copy()


def build_singletons(locs, seed):
    """Classic Vecchia structure: singleton blocks in a random order; centroids are the
    points themselves.  (block_ptr, point_idx, centroids)"""
    locs = _c(locs, np.float64)
    n, d = locs.shape
    bp = np.empty(n + 1, np.int64)
    pi = np.empty(n, np.int32)
    ce = np.empty((n, d), np.float64)
    st = lib().or_build_singletons(_ptr(locs, _d), n, d, seed, _ptr(bp, _i64), _ptr(pi, _i32), _ptr(ce, _d))
    if st:
        raise OracleError(st, "build_singletons")
    return bp, pi, ce


ORDERS = {"random": 0, "maxmin": 1, "morton": 2, "kdtree": 3, "hilbert": 4}


def order_blocks(centroids, order, seed=0):
    """New block order by a rule on the centroids: perm[q] = old position at new q."""
    ce = _c(centroids, np.float64)
    bc, d = ce.shape
    perm = np.empty(bc, np.int64)
    st = lib().or_order_blocks(_ptr(ce, _d), bc, d, ORDERS[order] if isinstance(order, str) else int(order),
                               seed, _ptr(perm, _i64))
    if st:
        raise OracleError(st, "order_blocks")
    return perm


def apply_block_order(block_ptr, point_idx, centroids, perm):
    """The block structure with its blocks placed in the order perm."""
    bp = np.asarray(block_ptr)
    sizes = np.diff(bp)[perm]
    nbp = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    npi = np.concatenate([point_idx[bp[p]:bp[p + 1]] for p in perm]).astype(np.int32)
    return nbp, npi, np.asarray(centroids)[perm].copy()


def hilbert_index(coords):
    """Hilbert index of one point of 21-bit integer coordinates (d = 1..3)."""
    c = _c(np.asarray(coords, np.uint64), np.uint64)
    return int(lib().or_hilbert_index(_ptr(c, _u64), c.size))


def select_neighbors(locs, block_ptr, point_idx, centroids, m, m_per_block=None):
    locs = _c(locs, np.float64)
    n, d = locs.shape
    bp = _c(block_ptr, np.int64)
    pi = _c(point_idx, np.int32)
    ce = _c(centroids, np.float64)
    bc = bp.size - 1
    mp = _c(m_per_block, np.int32) if m_per_block is not None else None
    nnp = np.empty(bc + 1, np.int64)
    L = lib()
    st = L.or_select_neighbors(_ptr(locs, _d), n, d, bc, _ptr(bp, _i64), _ptr(pi, _i32),
                               _ptr(ce, _d), int(m), _ptr(mp, _i32), _ptr(nnp, _i64), None)
    if st:
        raise OracleError(st, "select_neighbors")
    nni = np.empty(max(int(nnp[-1]), 1), np.int32)
    st = L.or_select_neighbors(_ptr(locs, _d), n, d, bc, _ptr(bp, _i64), _ptr(pi, _i32),
                               _ptr(ce, _d), int(m), _ptr(mp, _i32), _ptr(nnp, _i64),
                               _ptr(nni, _i32))
    if st:
        raise OracleError(st, "select_neighbors")
    return nnp, nni[:int(nnp[-1])].copy()


def loglik(th: Theta, locs, y, block_ptr, point_idx, nn_ptr, nn_idx, check=True):
    """Block-Vecchia log-likelihood (Eq. 4 by Algorithm 1): (ell, per_block, status)."""
    locs = _c(locs, np.float64)
    n, d = locs.shape
    y = _c(y, np.float64)
    bp, pi = _c(block_ptr, np.int64), _c(point_idx, np.int32)
    nnp = _c(nn_ptr, np.int64)
    nni = _c(nn_idx, np.int32) if len(nn_idx) else np.zeros(1, np.int32)
    bc = bp.size - 1
    out = np.zeros(1)
    per = np.zeros(bc)
    st = lib().or_loglik(ctypes.byref(th), _ptr(locs, _d), _ptr(y, _d), n, d, bc, _ptr(bp, _i64),
                         _ptr(pi, _i32), _ptr(nnp, _i64), _ptr(nni, _i32), _ptr(out, _d),
                         _ptr(per, _d))
    if check and st:
        raise OracleError(st, "loglik")
    return float(out[0]), per, int(st)


def block_loglik(th: Theta, locs, y, nn, blk):
    locs = _c(locs, np.float64)
    y = _c(y, np.float64)
    m = len(nn)
    nn = _c(nn, np.int32) if m else np.zeros(1, np.int32)
    blk = _c(blk, np.int32)
    st = ctypes.c_int(0)
    v = lib().or_block_loglik(ctypes.byref(th), _ptr(locs, _d), _ptr(y, _d), locs.shape[1],
                              _ptr(nn, _i32), m, _ptr(blk, _i32), blk.size, ctypes.byref(st))
    return float(v), int(st.value)


def exact_loglik(th: Theta, locs, y):
    locs = _c(locs, np.float64)
    y = _c(y, np.float64)
    out = np.zeros(1)
    st = lib().or_exact_loglik(ctypes.byref(th), _ptr(locs, _d), _ptr(y, _d), locs.shape[0],
                               locs.shape[1], _ptr(out, _d))
    if st:
        raise OracleError(st, "exact_loglik")
    return float(out[0])


def exact_draw(th: Theta, locs, z):
    locs = _c(locs, np.float64)
    z = _c(z, np.float64)
    y = np.empty_like(z)
    st = lib().or_exact_draw(ctypes.byref(th), _ptr(locs, _d), locs.shape[0], locs.shape[1],
                             _ptr(z, _d), _ptr(y, _d))
    if st:
        raise OracleError(st, "exact_draw")
    return y


def bv_draw(th: Theta, locs, block_ptr, point_idx, nn_ptr, nn_idx, z):
    locs = _c(locs, np.float64)
    z = _c(z, np.float64)
    bp, pi = _c(block_ptr, np.int64), _c(point_idx, np.int32)
    nnp = _c(nn_ptr, np.int64)
    nni = _c(nn_idx, np.int32) if len(nn_idx) else np.zeros(1, np.int32)
    y = np.zeros_like(z)
    st = lib().or_bv_draw(ctypes.byref(th), _ptr(locs, _d), locs.shape[0], locs.shape[1],
                          bp.size - 1, _ptr(bp, _i64), _ptr(pi, _i32), _ptr(nnp, _i64),
                          _ptr(nni, _i32), _ptr(z, _d), _ptr(y, _d))
    if st:
        raise OracleError(st, "bv_draw")
    return y


def build_pred_blocks(locs_star, bc, seed, iters=20):
    """Algorithm 2 clustering of the new locations: (block_ptr, point_idx, centroids),
    blocks in cluster-index order."""
    ls = _c(locs_star, np.float64)
    n, d = ls.shape
    bp = np.empty(bc + 1, np.int64)
    pi = np.empty(n, np.int32)
    ce = np.empty((bc, d), np.float64)
    nb = lib().or_build_pred_blocks(_ptr(ls, _d), n, d, bc, seed, iters, _ptr(bp, _i64),
                                    _ptr(pi, _i32), _ptr(ce, _d))
    if nb < 0:
        raise OracleError(-nb, "build_pred_blocks")
    return bp[:nb + 1].copy(), pi, ce[:nb].copy()


def select_pred_neighbors(locs, centroids, m):
    """The min(m, n) observations nearest to each prediction block's centroid."""
    locs = _c(locs, np.float64)
    n, d = locs.shape
    ce = _c(centroids, np.float64).reshape(-1, d)
    bc = ce.shape[0]
    nnp = np.empty(bc + 1, np.int64)
    mi = min(int(m), n)
    nni = np.empty(max(bc * mi, 1), np.int32)
    st = lib().or_select_pred_neighbors(_ptr(locs, _d), n, d, bc, _ptr(ce, _d), int(m),
                                        _ptr(nnp, _i64), _ptr(nni, _i32))
    if st:
        raise OracleError(st, "select_pred_neighbors")
    return nnp, nni[:int(nnp[-1])].copy()


def predict_block(th: Theta, locs, y, nn, locs_star, blk):
    """One block of Algorithm 2: (mean[b], Sigma_B[b x b])."""
    locs, y, ls = _c(locs, np.float64), _c(y, np.float64), _c(locs_star, np.float64)
    m = len(nn)
    nn = _c(nn, np.int32) if m else np.zeros(1, np.int32)
    blk = _c(blk, np.int32)
    b = blk.size
    mean = np.empty(b)
    cov = np.empty((b, b))
    st = lib().or_predict_block(ctypes.byref(th), _ptr(locs, _d), _ptr(y, _d), locs.shape[1],
                                _ptr(nn, _i32), m, _ptr(ls, _d), _ptr(blk, _i32), b,
                                _ptr(mean, _d), _ptr(cov, _d))
    if st:
        raise OracleError(st, "predict_block")
    return mean, cov


def predict(th: Theta, locs, y, locs_star, block_ptr, point_idx, nn_ptr, nn_idx, packed_cov=False):
    """Algorithm 2: (mean[n*], var[n*], packed per-block Sigma_B or None)."""
    locs, y, ls = _c(locs, np.float64), _c(y, np.float64), _c(locs_star, np.float64)
    n, d = locs.shape
    bp, pi = _c(block_ptr, np.int64), _c(point_idx, np.int32)
    nnp = _c(nn_ptr, np.int64)
    nni = _c(nn_idx, np.int32) if len(nn_idx) else np.zeros(1, np.int32)
    ns = ls.shape[0]
    mean, var = np.empty(ns), np.empty(ns)
    b = np.diff(bp)
    cov = np.empty(max(int(np.sum(b * (b + 1) // 2)), 1)) if packed_cov else None
    st = lib().or_predict(ctypes.byref(th), _ptr(locs, _d), _ptr(y, _d), n, d, _ptr(ls, _d),
                          bp.size - 1, _ptr(bp, _i64), _ptr(pi, _i32), _ptr(nnp, _i64),
                          _ptr(nni, _i32), _ptr(mean, _d), _ptr(var, _d), _ptr(cov, _d))
    if st:
        raise OracleError(st, "predict")
    return mean, var, cov


def csim_normal(seed: int, j: int, rounds: int, r: int) -> float:
    """Standard normal number r of new location j when each location takes `rounds`."""
    return float(lib().or_csim_normal(seed, j, rounds, r))


def cond_sim(mean, var, rounds, seed, z_crit, y_true=None):
    """Univariate conditional simulation: (lower[n*], upper[n*], covered count)."""
    mean, var = _c(mean, np.float64), _c(var, np.float64)
    yt = _c(y_true, np.float64) if y_true is not None else None
    ns = mean.size
    lo, up = np.empty(ns), np.empty(ns)
    cov = np.zeros(1, np.int64)
    st = lib().or_cond_sim(_ptr(mean, _d), _ptr(var, _d), ns, int(rounds), seed, float(z_crit),
                           _ptr(yt, _d), _ptr(lo, _d), _ptr(up, _d), _ptr(cov, _i64))
    if st:
        raise OracleError(st, "cond_sim")
    return lo, up, int(cov[0])
