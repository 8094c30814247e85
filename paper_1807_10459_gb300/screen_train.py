"""Train the learned screen on exact greedy runs and calibrate its margin.

Data: exact (batched-mode) greedy parent selection on synthetic networks drawn
by ``synth`` with seeds disjoint from every evaluation network: 10-node sparse
VAR(5) networks (T = 10000), 20-node in-degree-3 VAR(3) networks (T = 5000) and
4-map coupled logistic chains (T = 4000).  Every executed greedy step yields
one sample per candidate: the screen's features (definition in include/idtx.h,
computed by the same kernel as in the screened step, idtx_screen_features)
and the target: by how much the largest of all its surrogate estimates exceeds
the largest of its s0 cheap ones.

The network is trained on the GPU by idtx_screen_train with the pinball loss
of a high quantile (0.99 by default), so it learns how large the excess gets
for a candidate's N, dimensions and cheap-surrogate spread; the margin delta
is the largest under-prediction of the excess (prediction clipped at 0) on
held-out steps (other seeds) times 1.25, so that no held-out candidate's
surrogate maximum exceeds cheap maximum + max(prediction, 0) + delta.  The
summary also reports the network-free rule it improves on: a constant margin
(1.25 x the largest training excess) over the cheap maximum.

Usage (GPU):  python -m paper_1807_10459_gb300.screen_train [--out PATH] [--quick]
Writes PATH (default: screen_weights.npz next to this file), the same screen in
idtx_screen_load's flat layout beside it (.bin), and prints a JSON summary.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))

import paper_1807_10459_gb300 as idtx  # noqa: E402
from paper_1807_10459_gb300 import synth  # noqa: E402

K = 4
N_SURR = 200
S0 = 8


def greedy_samples(series, target, n_past, max_lag, seed, ctx, max_steps=4):
    """Run the exact greedy loop for one target; return (features, targets)."""
    import torch
    s = torch.from_numpy(np.ascontiguousarray(series)).cuda()
    T = series.shape[1]
    n = T - max(max_lag, n_past)
    selected, X, Y = [], [], []
    for step in range(max_steps):
        res, est = idtx.mte_step(s, target, n_past, 1, max_lag, selected, step, k=K,
                                 n_surr=N_SURR, seed=seed, want_estimates=True, ctx=ctx)
        alive = np.flatnonzero(~np.isnan(est[:, 0]))
        dz = n_past + len(selected)
        # the features the screened step computes (idtx_screen_features)
        X += list(idtx.screen_features(est[alive], n, dz, K, N_SURR, S0, ctx=ctx))
        for c in alive:
            Y.append(np.float32(est[c, 1:].max() - est[c, 1:1 + S0].max()))
        if not res[1] or len(alive) <= 1:
            break
        selected.append(res[0])
    return X, Y


def networks(kind_seed_base, quick):
    """(name, series, n_past, max_lag, targets) of the training/holdout networks."""
    out = []
    n_var10 = 2 if quick else 6
    for i in range(n_var10):
        net = synth.var_network(seed=kind_seed_base + 100 + i)
        out.append(("var10", net.series, 3, 5, range(0, 10, 2 if quick else 1)))
    n_var20 = 1 if quick else 3
    for i in range(n_var20):
        net = synth.var_network_indegree(n_nodes=20, order=3, indegree=3, T=5000,
                                         seed=kind_seed_base + 200 + i)
        out.append(("var20", net.series, 3, 3, range(0, 20, 4 if quick else 2)))
    n_log = 1 if quick else 3
    for i in range(n_log):
        maps = synth.logistic_chain(n_maps=4, length=4000, reps=1, seed=kind_seed_base + 300 + i)
        series = np.ascontiguousarray(((maps[0] - maps[0].mean(1, keepdims=True)) /
                                       maps[0].std(1, keepdims=True)).astype(np.float32))
        out.append(("logistic4", series, 2, 3, range(4)))
    return out


def collect(seed_base, quick, ctx):
    X, Y = [], []
    for name, series, n_past, max_lag, targets in networks(seed_base, quick):
        for t in targets:
            x, y = greedy_samples(series, t, n_past, max_lag, seed=seed_base + 7 * t, ctx=ctx)
            X += x
            Y += y
    return np.array(X, np.float32), np.array(Y, np.float32)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(HERE, "screen_weights.npz"))
    ap.add_argument("--quick", action="store_true", help="small data set (for tests)")
    ap.add_argument("--epochs", type=int, default=400)
    ap.add_argument("--dump", default="", help="also save the samples (npz) here")
    ap.add_argument("--quantile", type=float, default=0.99)
    args = ap.parse_args()
    ctx = idtx.Context(0)
    t0 = time.time()
    Xtr, Ytr = collect(5000, args.quick, ctx)
    Xho, Yho = collect(6000, args.quick, ctx)
    t_data = time.time() - t0
    if args.dump:
        np.savez(args.dump, Xtr=Xtr, Ytr=Ytr, Xho=Xho, Yho=Yho)
    mean = Xtr.mean(axis=0)
    sd = Xtr.std(axis=0)
    scale = np.where(sd > 1e-6, 1.0 / np.maximum(sd, 1e-6), 1.0).astype(np.float32)
    sc = idtx.Screen(feat_mean=mean, feat_scale=scale, s0=S0, seed=1)
    t1 = time.time()
    loss = idtx.screen_train(sc, Xtr, Ytr, epochs=args.epochs, batch=256, lr=1e-3, seed=3,
                             quantile=args.quantile, ctx=ctx)
    t_train = time.time() - t1
    pred_ho = np.maximum(idtx.screen_predict(sc, Xho, ctx=ctx), 0.0)
    under = Yho - pred_ho                     # > 0: the prediction was too low
    delta = float(max(under.max(), 0.0) * 1.25)
    sc.delta = delta
    pred_tr = np.maximum(idtx.screen_predict(sc, Xtr, ctx=ctx), 0.0)
    const_margin = float(Ytr.max() * 1.25)     # the network-free rule
    bound = pred_ho + delta
    summary = dict(train_samples=int(len(Ytr)), holdout_samples=int(len(Yho)),
                   quantile=args.quantile, train_loss=float(loss),
                   holdout_max_under=float(under.max()), delta=delta,
                   holdout_mean_bound=float(bound.mean()),
                   holdout_median_bound=float(np.median(bound)),
                   network_free_margin=const_margin,
                   holdout_violations=int(np.count_nonzero(Yho > bound)),
                   network_free_violations=int(np.count_nonzero(Yho > const_margin)),
                   holdout_max_excess=float(Yho.max()),
                   train_violations=int(np.count_nonzero(Ytr > pred_tr + delta)),
                   data_seconds=round(t_data, 1), train_seconds=round(t_train, 1),
                   epochs=args.epochs, s0=S0, n_surr=N_SURR, k=K)
    sc.save(args.out, **summary)
    sc.save_bin(os.path.splitext(args.out)[0] + ".bin")  # for idtx_screen_load
    print(json.dumps(summary))


if __name__ == "__main__":
    main()
