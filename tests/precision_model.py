"""Precision study (analysis script, not a test): which parts of the augmented block
Cholesky must be FP64 for the mixed-precision log-likelihood to stay accurate.

Run:  python -m tests.precision_model [n] [blocks_per_case]

A NumPy model of one block's factorisation (Algorithm 1 computed as the Cholesky factor of
the augmented matrix [[Sigma^con, Sigma^cross, y_NN], [., Sigma^lk, y_B], [., ., *]]) in
which every matrix entry is either kept in FP64 or rounded to FP32 after each update
(products formed exactly and rounded once, as a fused multiply-add does).  Variants:

  all FP32            every entry FP32 (the FP32 bulk of the mixed path)
  Sigma^new FP64      the trailing (b+1) x (b+1) part -- Sigma^lk, its Schur update, its
                      factor, the block rows of y -- in FP64 (the conditional covariance's
                      factor and log-determinant in FP64)
  + diagonal panels   the same plus the 16 x 16 diagonal panels of Sigma^con in FP64
  rows >= m FP64      everything in the block rows (Sigma^cross, V = L^-1 Sigma^cross, the
                      Schur complement and y) in FP64: only Sigma^con's factor in FP32
  input rounding      FP64 arithmetic on the FP32-rounded covariance entries

Blocks, neighbours and data come from the FP64 oracle (config-5-like datasets: n uniform
points, bc = n/10 K-means blocks, m = 120, y drawn from the block-Vecchia model at m = 30).
The printed relative error of the summed log-likelihood over the sampled blocks shows that
the FP32 rounding of Sigma^con's entries and factor sets the error: FP64 for the
conditional covariance or the diagonal panels does not reduce it.

Second study (python -m tests.precision_model bias [n]): is the per-block FP32 error
zero-mean?  Classic Vecchia (one-point blocks, m = 30) and K-means blocks on config-2-like
data; every block's all-FP32 error delta_i, its error weight w_i (the check's
conditioning indicator) and r_i = delta_i / (2^-24 w_i).  Printed: the sum of delta over
all blocks and over the 29% best-conditioned (lowest w) blocks, the mean of r over both,
and the noise scale sqrt(sum w^2) 2^-24 rms(r); once plainly and once with the FP32
diagonal's residual (sigma^2 + tau^2 - fl32(sigma^2 + tau^2)) added to every pivot.  The
common rounding of the diagonal biases r by w (a mean of -0.011 over the best-conditioned
blocks of the one-point case against +0.007 over the worst quarter), so the blocks a
check leaves in FP32 can carry a sum many times the noise scale; the pivot correction
removes most of it.  A one-sided error of the pivots' reciprocal square roots (modelled as
1/sqrt rounded to FP32 and then 2^-24 low, the size of an approximate hardware 1/sqrt's
error) brings the same pattern back (mean r by w quartile about -0.02, -0.01, 0, +0.005 in
the one-point case, as measured on the GPU with the approximate 1/sqrt), hence the
kernels' correctly rounded 1/sqrt.
"""
import sys

import numpy as np

import oracle
from paper_2410_04477_gb300 import synth
from tests._ref import cov_matrix


def _r32(x):
    return np.asarray(x, np.float64).astype(np.float32).astype(np.float64)


def augmented(locs, y, bp, pi, nnp, nni, i, th):
    s2, beta, nu, tau2 = th
    blk = pi[bp[i]:bp[i + 1]].astype(np.int64)
    nn = nni[nnp[i]:nnp[i + 1]].astype(np.int64)
    idx = np.concatenate([nn, blk])
    C = cov_matrix(locs[idx], locs[idx], s2, beta, nu, tau2, same=np.eye(len(idx)))
    N = len(idx)
    A = np.zeros((N + 1, N + 1))
    A[:N, :N] = C
    A[N, :N] = y[idx]
    return A, len(nn), len(blk)


def block_terms(A, m, keep64):
    """u + log det of the block columns from a right-looking factorisation in which the
    entries marked in keep64 stay FP64 and the others are rounded to FP32 after every
    update; None if a pivot is not positive."""
    A = np.where(keep64, A, _r32(A))
    N = A.shape[0] - 1
    piv = np.zeros(N)
    for k in range(N):
        p = A[k, k]
        piv[k] = p
        if not p > 0:
            return None
        col = A[k + 1:, k] / np.sqrt(p)
        col = np.where(keep64[k + 1:, k], col, _r32(col))
        A[k + 1:, k] = col
        upd = A[k + 1:, k + 1:] - np.outer(col, col)
        A[k + 1:, k + 1:] = np.where(keep64[k + 1:, k + 1:], upd, _r32(upd))
    z = A[N, m:N]
    return (z * z).sum() + np.log(piv[m:N]).sum()


def variants(R, m):
    none = np.zeros((R, R), bool)
    new64 = none.copy()
    new64[m:, m:] = True
    panels = new64.copy()
    for k0 in range(0, m, 16):
        panels[k0:k0 + 16, k0:k0 + 16] = True
    rows = none.copy()
    rows[m:, :] = True
    return {"all FP32": none, "Sigma^new FP64": new64, "+ diagonal panels": panels, "rows >= m FP64": rows}


def study(n=3000, per_case=60):
    cases = [(2.5, 0.3, 1e-4), (2.5, 0.1, 1e-3), (1.5, 0.2, 1e-4), (0.5, 0.3, 1e-4), (1.5, 0.05, 1e-2)]
    for nu, beta, tau2 in cases:
        th = (1.0, beta, nu, tau2)
        locs = synth.locs_uniform(n, 2, 3)
        bp, pi, ce = oracle.build_blocks(locs, n // 10, seed=3)
        gnp, gni = oracle.select_neighbors(locs, bp, pi, ce, 30)
        y = oracle.bv_draw(oracle.theta(*th), locs, bp, pi, gnp, gni, synth.normal(3, 20, n))
        nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, 120)
        bc = len(bp) - 1
        ref, got = 0.0, {}
        for i in range(0, bc, max(1, bc // per_case)):
            A, m, b = augmented(locs, y, bp, pi, nnp, nni, i, th)
            R = A.shape[0]
            c = -0.5 * b * np.log(2 * np.pi)
            ref += c - 0.5 * block_terms(A, m, np.ones((R, R), bool))
            for name, keep in variants(R, m).items():
                t = block_terms(A, m, keep)
                got[name] = got.get(name, 0.0) + (c - 0.5 * t if t is not None else -np.inf)
            t = block_terms(_r32(A), m, np.ones((R, R), bool))
            got["input rounding"] = got.get("input rounding", 0.0) + c - 0.5 * t
        print(f"nu={nu} beta={beta} tau2={tau2}: ell over the sampled blocks {ref:.4f}")
        for name, v in got.items():
            print(f"   {name:20s} relative error {abs(v - ref) / abs(ref):.2e}")


def _terms_lo(A, m, lo, rs_bias=0.0):
    """All-FP32 factorisation of the augmented matrix with lo added to every pivot (None:
    plain), the reciprocal square root of each pivot rounded to FP32 and then scaled by
    (1 + rs_bias) (a one-sided error of an approximate 1/sqrt); u + log det of the block
    columns."""
    A = _r32(A)
    N = A.shape[0] - 1
    piv = np.zeros(N)
    for k in range(N):
        p = A[k, k] if lo is None else float(np.float32(np.float32(A[k, k]) + np.float32(lo)))
        piv[k] = p
        rs = float(np.float32(1.0 / np.sqrt(p))) * (1.0 + rs_bias)
        col = _r32(A[k + 1:, k] * rs)
        A[k + 1:, k] = col
        A[k + 1:, k + 1:] = _r32(A[k + 1:, k + 1:] - np.outer(col, col))
    z = A[N, m:N]
    return (z * z).sum() + np.log(piv[m:N]).sum()


def bias_study(n=20000):
    side = (n / 2e5) ** 0.5   # the config-2 point density
    for singletons, m, th in ((True, 30, (1.0, 0.05, 1.5, 1e-4)), (False, 60, (1.0, 0.05, 1.5, 1e-4)),
                              (False, 30, (1.3, 0.03, 0.5, 3e-3))):
        locs = synth.locs_uniform(n, 2, 1) * side
        if singletons:
            bp, pi, ce = oracle.build_singletons(locs, seed=1)
        else:
            bp, pi, ce = oracle.build_blocks(locs, n // 10, seed=1)
        gnp, gni = oracle.select_neighbors(locs, bp, pi, ce, 100)
        y = oracle.bv_draw(oracle.theta(*th), locs, bp, pi, gnp, gni, synth.normal(1, 20, n))
        nnp, nni = oracle.select_neighbors(locs, bp, pi, ce, m)
        d32 = float(np.float32(np.float32(th[0]) + np.float32(th[3])))
        lo = (th[0] + th[3]) - d32
        dl = {"plain": [], "pivot + diagonal residual": [], "... and 1/sqrt 2^-24 low": []}
        w = []
        step = 2 if singletons else 1
        for i in range(0, len(bp) - 1, step):
            A, mm, b = augmented(locs, y, bp, pi, nnp, nni, i, th)
            N = A.shape[0] - 1
            L = np.linalg.cholesky(A[:N, :N])
            pv = np.diag(L) ** 2
            z = np.linalg.solve(L, A[N, :N])[mm:]
            t64 = np.log(pv[mm:]).sum() + (z * z).sum()
            dl["plain"].append(-0.5 * (_terms_lo(A, mm, None) - t64))
            dl["pivot + diagonal residual"].append(-0.5 * (_terms_lo(A, mm, lo) - t64))
            dl["... and 1/sqrt 2^-24 low"].append(-0.5 * (_terms_lo(A, mm, lo, -2.0 ** -24) - t64))
            w.append(((th[0] + th[3]) / pv).sum() * (1 + (z * z).sum() / b))
        w = np.array(w)
        keep = np.argsort(w)[:int(0.29 * len(w))]
        print(f"{'one-point' if singletons else 'K-means'} blocks, m = {m}, theta = {th}: residual {lo:.3e}")
        q = np.argsort(w)
        for name, d in dl.items():
            d = np.array(d)
            r = d / (2.0 ** -24 * w)
            quart = " ".join(f"{r[q[int(a * len(q)):int((a + .25) * len(q))]].mean():+.4f}" for a in (0, .25, .5, .75))
            print(f"   {name:26s} sum {d.sum():+.3e} (best 29%: {d[keep].sum():+.3e}), mean r {r.mean():+.4f} "
                  f"(by w quartile {quart}), noise scale {np.sqrt((w * w).sum()) * 2.0 ** -24 * np.sqrt((r * r).mean()):.3e}")


if __name__ == "__main__":
    if len(sys.argv) > 1 and sys.argv[1] == "bias":
        bias_study(int(sys.argv[2]) if len(sys.argv) > 2 else 20000)
    else:
        study(int(sys.argv[1]) if len(sys.argv) > 1 else 3000, int(sys.argv[2]) if len(sys.argv) > 2 else 60)
