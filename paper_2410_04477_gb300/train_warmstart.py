"""Train the warm-start MLP on fields simulated by the block-Vecchia model itself.

Training set: datasets of n uniform points in [0,1]^2, theta log-uniform over
sigma^2 in [0.5, 2], beta in [0.02, 0.3], tau^2 in [1e-4, 1e-1], nu uniform over
{0.5, 1.5, 2.5}; each drawn with the library's block-Vecchia sampler (bc = n/10 K-means
blocks, m = 100), featurised with bv_features on the same structure, and the network
trained with bv_mlp_train (the library's own forward, backward and Adam kernels).

    python -m paper_2410_04477_gb300.train_warmstart --n-train 4096 --out weights/warmstart.bvws
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from paper_2410_04477_gb300 import bv, synth

HERE = os.path.dirname(os.path.abspath(__file__))


def make_dataset(ctx, k, n, m=100):
    th = synth.theta_draws(1000 + k, 1)[0]
    s2, beta, tau2, nu = th
    locs = synth.locs_uniform(n, 2, 1000 + k)
    ctx.set_data(locs)
    ctx.build_blocks(n // 10, seed=1000 + k, iters=20)
    ctx.select_neighbors(m)
    ctx.simulate(bv.theta(s2, beta, nu, tau2), synth.normal(1000 + k, 20, n))
    f = ctx.features(max_points=10000, seed=0)[0]
    return f, np.array([np.log(s2), np.log(beta), np.log(tau2), nu])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-train", type=int, default=4096)
    ap.add_argument("--n-val", type=int, default=256)
    ap.add_argument("--n", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--batch", type=int, default=256)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--out", default=os.path.join(HERE, "weights", "warmstart.bvws"))
    args = ap.parse_args()
    os.makedirs(os.path.dirname(args.out), exist_ok=True)
    t0 = time.time()
    X, T = [], []
    with bv.Context(0) as ctx:
        for k in range(args.n_train + args.n_val):
            f, t = make_dataset(ctx, k, args.n)
            X.append(f)
            T.append(t)
            if k % 512 == 0:
                print(f"dataset {k} ({time.time() - t0:.0f}s)", file=sys.stderr, flush=True)
    X, T = np.array(X, np.float32), np.array(T, np.float32)
    t_gen = time.time() - t0
    Xtr, Ttr, Xva, Tva = X[:args.n_train], T[:args.n_train], X[args.n_train:], T[args.n_train:]
    t1 = time.time()
    blob, losses = bv.mlp_train(Xtr, Ttr, epochs=args.epochs, batch=args.batch, lr=args.lr, seed=7)
    t_train = time.time() - t1
    out = bv.mlp_forward(blob, Xva)
    ym, ys = blob[80:83], blob[83:86]
    pred = out[:, :3] * ys + ym
    rmse = np.sqrt(np.mean((pred - Tva[:, :3]) ** 2, axis=0))
    nu_acc = float(np.mean(np.argmax(out[:, 3:], axis=1) == np.round((Tva[:, 3] - 0.5)).astype(int)))
    bv.save_blob(args.out, blob)
    summary = {"n_train": args.n_train, "n_val": args.n_val, "n": args.n, "epochs": args.epochs,
               "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
               "val_rmse_log_sigma2_beta_tau2": rmse.tolist(), "val_nu_accuracy": nu_acc,
               "gen_seconds": round(t_gen, 1), "train_seconds": round(t_train, 1)}
    with open(os.path.splitext(args.out)[0] + ".json", "w") as f:
        json.dump(summary, f, indent=1)
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
