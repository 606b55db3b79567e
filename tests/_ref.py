"""Independent NumPy/SciPy constructions used to pin the oracle.

These are not the oracle: they build the same mathematical objects by another route
(Eq. 5 with SciPy's Bessel K_nu instead of the closed forms; dense matrices and library
solves instead of Algorithm 1's batched steps), so that a slip in the oracle shows up as
a mismatch here.
"""
import numpy as np
from scipy.special import gamma, kv


def matern_kv(nu, x):
    """Eq. 5 correlation with SciPy's modified Bessel function of the second kind."""
    x = np.asarray(x, dtype=np.float64)
    out = np.ones_like(x)
    nz = x > 0
    xv = x[nz]
    out[nz] = 2.0 ** (1.0 - nu) / gamma(nu) * xv ** nu * kv(nu, xv)
    return out


def cov_matrix(locs_a, locs_b, sigma2, beta, nu, nugget=0.0, ranges=None, same=None):
    """Dense covariance K(a, b) of Eq. 5 (+ nugget where `same` marks identical points)."""
    a = np.asarray(locs_a, dtype=np.float64)
    b = np.asarray(locs_b, dtype=np.float64)
    diff = a[:, None, :] - b[None, :, :]
    if ranges is not None:
        x = np.sqrt(((diff / np.asarray(ranges)[None, None, : a.shape[1]]) ** 2).sum(-1))
    else:
        x = np.sqrt((diff ** 2).sum(-1)) / beta
    c = sigma2 * matern_kv(nu, x)
    if same is not None:
        c = c + nugget * same
    return c


def full_cov(locs, sigma2, beta, nu, nugget=0.0, ranges=None):
    n = len(locs)
    return cov_matrix(locs, locs, sigma2, beta, nu, nugget, ranges, same=np.eye(n))


def exact_loglik(S, y):
    """Eq. 1 by a library Cholesky."""
    L = np.linalg.cholesky(S)
    z = np.linalg.solve(L, y)
    return -0.5 * len(y) * np.log(2 * np.pi) - np.log(np.diag(L)).sum() - 0.5 * z @ z


def conditional_block_loglik(S, y, nn, blk):
    """log p(y_B | y_NN) for the Gaussian with covariance S, by library solves."""
    nn = np.asarray(nn, dtype=np.int64)
    blk = np.asarray(blk, dtype=np.int64)
    Sbb = S[np.ix_(blk, blk)]
    yb = y[blk]
    if len(nn):
        Snn = S[np.ix_(nn, nn)]
        Snb = S[np.ix_(nn, blk)]
        W = np.linalg.solve(Snn, Snb)
        mu = W.T @ y[nn]
        C = Sbb - Snb.T @ W
    else:
        mu = np.zeros(len(blk))
        C = Sbb
    sign, logdet = np.linalg.slogdet(C)
    assert sign > 0
    r = yb - mu
    return -0.5 * (len(blk) * np.log(2 * np.pi) + logdet + r @ np.linalg.solve(C, r))


def bv_dense_precision(S, block_ptr, point_idx, nn_ptr, nn_idx):
    """Implied block-Vecchia joint: precision A^T D^{-1} A, with A unit block-lower
    triangular (rows B_i: identity on B_i, -(S_NN^{-1} S_NB)^T on NN_i) and D the block
    diagonal of conditional covariances.  Returns (precision, logdet of precision, A, D-blocks)."""
    n = S.shape[0]
    A = np.zeros((n, n))
    Dinv = np.zeros((n, n))
    logdet_D = 0.0
    Dblocks = []
    for i in range(len(block_ptr) - 1):
        blk = point_idx[block_ptr[i]:block_ptr[i + 1]].astype(np.int64)
        nn = nn_idx[nn_ptr[i]:nn_ptr[i + 1]].astype(np.int64)
        A[np.ix_(blk, blk)] = np.eye(len(blk))
        Sbb = S[np.ix_(blk, blk)]
        if len(nn):
            W = np.linalg.solve(S[np.ix_(nn, nn)], S[np.ix_(nn, blk)])
            A[np.ix_(blk, nn)] = -W.T
            C = Sbb - S[np.ix_(nn, blk)].T @ W
        else:
            C = Sbb
        Dinv[np.ix_(blk, blk)] = np.linalg.inv(C)
        logdet_D += np.linalg.slogdet(C)[1]
        Dblocks.append((blk, C))
    P = A.T @ Dinv @ A
    return P, -logdet_D, A, Dblocks


def loglik_from_precision(P, logdet_P, y):
    return -0.5 * (len(y) * np.log(2 * np.pi) - logdet_P + y @ P @ y)
