"""FP64 NumPy oracle for the learned warm start (no counterpart in the paper; the paper's
non-learned heuristic is to start from a cheaper fit, Sec. 2.3).

TEST INFRASTRUCTURE (see oracle/__init__.py).  Plain, slow definitions:
  features()     the 40 summary features of one dataset (semivariogram, structure
                 statistics, nearest-neighbour semivariance and distance)
  mlp_forward()  the MLP 40 -> 128 -> 128 -> 128 -> 6 with exact-erf GELU
  mlp_loss_grad()  the training loss and its gradient by explicit backpropagation
  adam_step()    one step of Adam (Kingma and Ba 2015, Algorithm 1)
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf

import oracle as _o

NFEAT, H, NOUT = 40, 128, 6
LAYERS = [(NFEAT, H), (H, H), (H, H), (H, NOUT)]
NPARAM = sum(i * o + o for i, o in LAYERS)
BLOB = NPARAM + 2 * NFEAT + 6


def features(locs, y, block_ptr, nn_ptr, max_points=10000, seed=0):
    """Semivariogram gamma_k / var(y) in 32 bins of width 1/64 on (0, 0.5] over a seeded
    subsample, then log var(y), the fractions of blocks with 1-4, 5-8, 9-12, 13-16 and 17 or
    more points, the nearest-neighbour semivariance / var(y) and 64 x the mean
    nearest-neighbour distance.  (nn_ptr is accepted for the interface; no feature uses the
    conditioning sizes.)"""
    locs = np.asarray(locs, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    n, d = locs.shape
    keep = []
    for j in range(n):
        r = _o.splitmix64(seed, j)
        if n <= max_points or (r * n) >> 64 < max_points:
            keep.append(j)
    keep = np.array(keep, dtype=np.int64)
    X, V = locs[keep], y[keep]
    P = len(keep)
    sums = np.zeros(32)
    cnts = np.zeros(32, dtype=np.int64)
    for a in range(P - 1):
        diff = X[a + 1:] - X[a]
        d2 = diff[:, 0] * diff[:, 0]
        for k in range(1, d):
            d2 = d2 + diff[:, k] * diff[:, k]
        ok = (d2 > 0) & (d2 <= 0.25)
        kb = np.minimum(np.floor(np.sqrt(d2[ok]) * 64.0).astype(np.int64), 31)
        g = 0.5 * (V[a] - V[a + 1:][ok]) ** 2
        np.add.at(sums, kb, g)
        np.add.at(cnts, kb, 1)
    var = np.mean((y - y.mean()) ** 2)
    f = np.zeros(NFEAT)
    nz = cnts > 0
    f[:32][nz] = sums[nz] / cnts[nz] / var
    # block-size histogram: the fraction of blocks of each size class
    bs = np.diff(np.asarray(block_ptr))
    f[32] = np.log(var)
    for k, (lo, hi) in enumerate(((1, 4), (5, 8), (9, 12), (13, 16), (17, None))):
        inside = (bs >= lo) if hi is None else ((bs >= lo) & (bs <= hi))
        f[33 + k] = np.count_nonzero(inside) / len(bs)
    # nearest other subsample point (squared distance summed left to right, lowest index
    # on ties): semivariance and distance at the smallest lag
    g_nn, d_nn = 0.0, 0.0
    for a in range(P):
        diff = X - X[a]
        d2 = diff[:, 0] * diff[:, 0]
        for k in range(1, d):
            d2 = d2 + diff[:, k] * diff[:, k]
        d2[a] = np.inf
        j = int(np.argmin(d2))
        g_nn += 0.5 * (V[a] - V[j]) ** 2
        d_nn += np.sqrt(d2[j])
    f[38] = g_nn / P / var
    f[39] = 64.0 * d_nn / P
    return f


def unpack(blob):
    blob = np.asarray(blob, dtype=np.float64)
    xm, xs = blob[:NFEAT], blob[NFEAT:2 * NFEAT]
    ym, ys = blob[2 * NFEAT:2 * NFEAT + 3], blob[2 * NFEAT + 3:2 * NFEAT + 6]
    p = blob[2 * NFEAT + 6:]
    Ws, bs = [], []
    off = 0
    for i, o in LAYERS:
        Ws.append(p[off:off + i * o].reshape(i, o))
        off += i * o
        bs.append(p[off:off + o])
        off += o
    return xm, xs, ym, ys, Ws, bs


def _gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def _gelu_d(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def mlp_forward(blob, X):
    """Raw outputs (3 standardised regressions, 3 nu logits) for inputs X[n x 40]."""
    xm, xs, ym, ys, Ws, bs = unpack(blob)
    a = (np.asarray(X, dtype=np.float64) - xm) / xs
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W + b
        a = _gelu(z) if l < len(Ws) - 1 else z
    return a


def nu_class(nu):
    nu = np.asarray(nu)
    return np.where(nu < 1.0, 0, np.where(nu < 2.0, 1, 2))


def mlp_loss_grad(blob, X, T):
    """Mean over rows of  sum_k (out_k - t_k)^2 / 3  +  cross-entropy(softmax(logits), nu
    class), with t the standardised (log sigma^2, log beta, log tau^2); gradient with
    respect to the flat parameter vector, by backpropagation through each layer."""
    xm, xs, ym, ys, Ws, bs = unpack(blob)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    B = X.shape[0]
    t = (T[:, :3] - ym) / ys
    cls = nu_class(T[:, 3])
    acts, pres = [(X - xm) / xs], []
    a = acts[0]
    for l, (W, b) in enumerate(zip(Ws, bs)):
        z = a @ W + b
        pres.append(z)
        a = _gelu(z) if l < len(Ws) - 1 else z
        acts.append(a)
    out = acts[-1]
    e = out[:, :3] - t
    logits = out[:, 3:]
    mx = logits.max(axis=1, keepdims=True)
    ex = np.exp(logits - mx)
    pr = ex / ex.sum(axis=1, keepdims=True)
    loss = np.mean((e ** 2).sum(axis=1) / 3.0 - np.log(pr[np.arange(B), cls]))
    g = np.zeros_like(out)
    g[:, :3] = 2.0 * e / 3.0 / B
    onehot = np.zeros_like(pr)
    onehot[np.arange(B), cls] = 1.0
    g[:, 3:] = (pr - onehot) / B
    grads_W, grads_b = [None] * len(Ws), [None] * len(Ws)
    for l in range(len(Ws) - 1, -1, -1):
        grads_W[l] = acts[l].T @ g
        grads_b[l] = g.sum(axis=0)
        if l > 0:
            g = (g @ Ws[l].T) * _gelu_d(pres[l - 1])
    flat = np.concatenate([np.concatenate([gw.ravel(), gb]) for gw, gb in zip(grads_W, grads_b)])
    return loss, flat


def adam_step(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """Adam step t (t = 1, 2, ...; Kingma and Ba 2015, Algorithm 1): the biased first and
    second moment estimates m <- b1 m + (1 - b1) g and v <- b2 v + (1 - b2) g^2, their
    bias-corrected values m / (1 - b1^t) and v / (1 - b2^t), and the parameter update
    theta <- theta - lr * mhat / (sqrt(vhat) + eps).  Returns (theta, m, v)."""
    theta, g = np.asarray(theta, np.float64), np.asarray(g, np.float64)
    m = b1 * np.asarray(m, np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, np.float64) + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** t)
    vhat = v / (1.0 - b2 ** t)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v
