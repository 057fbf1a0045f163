"""Learned schedule: an MLP cost model that picks the amalgamation setting of each pattern.

Relaxed amalgamation trades explicit zeros (wasted flops) for wider supernodes (fewer, larger
tiles and launches); the best trade depends on the pattern. For a new pattern the inspector is
run once per candidate setting in host-only mode (cheap: no device work), the network predicts
the log factorization time from the resulting plan statistics, and the setting with the
smallest prediction is used. The fixed rule (PRESETS[DEFAULT]) is the fallback when no model is
given. The network is trained on factorization times the executor measures on the GPU (CUDA
events around sym_factor) across generated patterns, by the library's own MLP kernels.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

from . import MLP, SYM_PREC_FP64, Solver, sym_options_default

# (name, amalgamate, nrelax[3], zrelax_permille[3])
PRESETS = [
    ("fundamental", 0, (4, 16, 48), (800, 100, 50)),
    ("light", 1, (2, 8, 24), (500, 50, 20)),
    ("default", 1, (4, 16, 48), (800, 100, 50)),
    ("wide", 1, (8, 32, 96), (900, 200, 100)),
    ("widest", 1, (16, 64, 192), (950, 300, 150)),
]
DEFAULT = 2
HIDDEN = 32


def options(preset, host_only=False):
    name, am, nr, zr = PRESETS[preset]
    opt = sym_options_default()
    opt.amalgamate = am
    opt.nrelax[:] = nr
    opt.zrelax_permille[:] = zr
    opt.precision = SYM_PREC_FP64
    return opt


def features(n, nnz_a, info, preset):
    """Plan statistics of one (pattern, setting), log-scaled, plus the setting itself."""
    _, am, nr, zr = PRESETS[preset]
    lg = lambda v: math.log1p(max(float(v), 0.0))
    f = [lg(n), lg(nnz_a / max(n, 1)), lg(info.nnz_l), lg(info.storage_l / max(info.nnz_l, 1)),
         lg(info.exec_flops), lg(info.exec_flops / max(info.flops, 1.0)), lg(info.nsuper), lg(info.nlevels),
         lg(info.max_ncols), lg(info.nlaunch_factor), lg(info.upd_tasks), lg(info.upd_entries),
         lg(info.dense_tasks), lg(info.npairs), float(am)]
    f += [lg(v) for v in nr] + [v / 1000.0 for v in zr]
    return np.asarray(f, dtype=np.float64)


NFEAT = 21


def plan_features(M):
    """Features of every preset for matrix M (host-only inspections)."""
    rows = []
    for p in range(len(PRESETS)):
        s = Solver(M.n, M.Ap, M.Ai, M.perm, opt=options(p), host_only=True)
        rows.append(features(M.n, M.nnz, s.info(), p))
        s.close()
    return np.stack(rows)


def time_factor(M, preset, torch, reps=3, warm=2):
    """Median CUDA-event time (ms) of sym_factor for one setting (graph replay, FP64)."""
    s = Solver(M.n, M.Ap, M.Ai, M.perm, opt=options(preset))
    stream = torch.cuda.current_stream()
    s.set_stream(stream)
    Ax = torch.from_numpy(M.Ax).cuda()
    for _ in range(warm):
        s.factor(Ax)
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s.factor(Ax)
        e1.record(stream)
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
    s.close()
    return float(np.median(ts))


def collect(mats, torch, flop_budget=4e10, log=None):
    """Features and measured times of every (pattern, preset); patterns whose default plan
    exceeds flop_budget are skipped (and counted)."""
    X, Y, G, skipped = [], [], [], 0
    for gi, M in enumerate(mats):
        F = plan_features(M)
        if math.expm1(F[DEFAULT][4]) > flop_budget:
            skipped += 1
            continue
        for p in range(len(PRESETS)):
            X.append(F[p])
            Y.append(math.log(time_factor(M, p, torch)))
            G.append(gi)
        if log:
            log(f"{gi + 1}/{len(mats)} {M.name}: " + " ".join(f"{math.exp(y):.2f}" for y in Y[-len(PRESETS):]))
    return np.asarray(X), np.asarray(Y), np.asarray(G), skipped


class CostModel:
    """Trained network plus its input normalization."""

    def __init__(self, theta, mean, std, hidden=HIDDEN):
        self.theta = np.asarray(theta, dtype=np.float32)
        self.mean = np.asarray(mean, dtype=np.float64)
        self.std = np.asarray(std, dtype=np.float64)
        self.hidden = hidden
        self._net = None

    @staticmethod
    def fit(X, Y, torch, steps=3000, lr=3e-3, seed=0, hidden=HIDDEN):
        mean = X.mean(axis=0)
        std = X.std(axis=0) + 1e-6
        net = MLP(X.shape[1], hidden, seed=seed)
        Xt = torch.from_numpy(((X - mean) / std).astype(np.float32)).cuda()
        Yt = torch.from_numpy(Y.astype(np.float32)).cuda()
        loss0 = net.gradient(Xt, Yt)[1]
        loss = net.train(Xt, Yt, steps, lr)
        cm = CostModel(net.get_params(), mean, std, hidden)
        cm._net = net
        return cm, loss0, loss

    def predict(self, X, torch):
        if self._net is None:
            self._net = MLP(X.shape[1], self.hidden)
            self._net.set_params(self.theta)
        Xt = torch.from_numpy(((np.asarray(X) - self.mean) / self.std).astype(np.float32)).cuda()
        return self._net.predict(Xt).cpu().numpy().astype(np.float64)

    def choose(self, M, torch):
        """Preset index with the smallest predicted factorization time for matrix M."""
        return int(np.argmin(self.predict(plan_features(M), torch)))

    def save(self, path):
        with open(path, "w") as f:
            json.dump({"hidden": self.hidden, "theta": self.theta.tolist(), "mean": self.mean.tolist(),
                       "std": self.std.tolist(), "presets": [p[0] for p in PRESETS]}, f)

    @staticmethod
    def load(path):
        with open(path) as f:
            d = json.load(f)
        return CostModel(d["theta"], d["mean"], d["std"], d["hidden"])


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_weights.json")


def pretrained():
    """The network trained on 1600 generated patterns (400 more held out) of the pattern suite;
    its training run is `python -m paper_1705_06575_gb300.costmodel --patterns 2000 --holdout 0.2
    --seed 20000`."""
    return CostModel.load(WEIGHTS)


def choose_preset(M, torch, model=None):
    """The learned choice, or the fixed rule when no model is available."""
    return DEFAULT if model is None else model.choose(M, torch)


def evaluate(model, X, Y, G, torch):
    """Per held-out pattern: measured time of the model's choice, of the fixed rule and of the best
    setting. Returns summary statistics."""
    groups = np.unique(G)
    pred = model.predict(X, torch)
    r_chosen, r_best, wins, losses = [], [], 0, 0
    for g in groups:
        idx = np.nonzero(G == g)[0]
        t = np.exp(Y[idx])
        c = idx[int(np.argmin(pred[idx]))] - idx[0]
        r_chosen.append(t[DEFAULT] / t[c])
        r_best.append(t[DEFAULT] / t.min())
        wins += t[c] < 0.98 * t[DEFAULT]
        losses += t[c] > 1.02 * t[DEFAULT]
    gm = lambda r: float(np.exp(np.mean(np.log(r))))
    return {"patterns": int(groups.size), "geomean_speedup_vs_fixed_rule": gm(r_chosen),
            "geomean_speedup_of_best_setting": gm(r_best), "wins": int(wins), "losses": int(losses),
            "total_time_ratio": float(sum(np.exp(Y[np.nonzero(G == g)[0]])[DEFAULT] for g in groups) /
                                      sum(np.exp(Y[np.nonzero(G == g)[0]])[int(np.argmin(pred[np.nonzero(G == g)[0]]))]
                                          for g in groups))}


def main(argv=None):
    """Collect, train and evaluate: python -m paper_1705_06575_gb300.costmodel --patterns N --out DIR"""
    import argparse
    import sys

    import torch

    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, here)
    import workloads as w

    ap = argparse.ArgumentParser()
    ap.add_argument("--patterns", type=int, default=240)
    ap.add_argument("--holdout", type=float, default=0.2)
    ap.add_argument("--seed", type=int, default=5000)
    ap.add_argument("--out", default="costmodel_out")
    args = ap.parse_args(argv)
    os.makedirs(args.out, exist_ok=True)
    t0 = time.time()
    mats = w.pattern_suite(args.patterns, args.seed)
    X, Y, G, skipped = collect(mats, torch, log=lambda s: print(s, flush=True))
    np.savez(os.path.join(args.out, "data.npz"), X=X, Y=Y, G=G)
    groups = np.unique(G)
    ntest = max(1, int(round(args.holdout * groups.size)))
    test_g = groups[-ntest:]
    tr = ~np.isin(G, test_g)
    model, l0, l1 = CostModel.fit(X[tr], Y[tr], torch)
    model.save(os.path.join(args.out, "model.json"))
    ev = evaluate(model, X[~tr], Y[~tr], G[~tr], torch)
    ev_train = evaluate(model, X[tr], Y[tr], G[tr], torch)
    res = {"patterns": args.patterns, "skipped_over_budget": skipped, "train_patterns": int(groups.size - ntest),
           "heldout": ev, "train": ev_train, "loss_initial": l0, "loss_final": l1,
           "seconds": time.time() - t0}
    with open(os.path.join(args.out, "eval.json"), "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
