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

from . import (MLP, SYM_PREC_FP64, SYM_PROFILE_OFF, SYM_PROFILE_ON, SYM_PROFILE_RESET, Solver,
               sym_options_default, sym_profile_launches)

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


# ---------------------------------------------------------------------------------------------
# Per-supernode rules: the network predicts, for every fundamental supernode and every preset
# rule, the time that supernode's share of the factorization takes when that rule decides its
# merge with the next supernode; each supernode then gets the rule with the smallest prediction
# (sym_analyze_rules). The training targets are the launch times the executor measures
# (sym_profile_launches, one profiled factorization per pattern and preset), spread over the
# supernodes of each launch by their tasks' flops and from a final supernode to its fundamental
# ones by their share of sum c_j^2.

RULES = np.array([[am, *nr, *zr] for (_, am, nr, zr) in PRESETS], dtype=np.int32)
NFEAT_SN = 21


def fund_table(M):
    """Per fundamental supernode of M (in SYM_EXPORT_FSUPER order): its structure and that of the
    next supernode, with which the amalgamation rule may merge it."""
    s = Solver(M.n, M.Ap, M.Ai, M.perm, opt=options(0), host_only=True)
    sup = s.export("super").astype(np.int64)
    rowptr = s.export("rowptr")
    parent = s.export("parent")
    level = s.export("level")
    sparent = s.export("sparent")
    cc = s.export("colcount").astype(np.float64)
    s.close()
    nf = sup.size - 1
    ncols = np.diff(sup).astype(np.float64)
    nrows = np.diff(rowptr).astype(np.float64)
    csq = np.add.reduceat(cc * cc, sup[:-1]) if nf else np.zeros(0)
    nnz = ncols * nrows - ncols * (ncols - 1) / 2
    last = sup[1:] - 1
    elig = np.zeros(nf, dtype=bool)
    if nf > 1:
        elig[:-1] = parent[last[:-1]] == last[:-1] + 1
    nxt_c = np.zeros(nf)
    nxt_r = np.zeros(nf)
    nxt_c[:-1], nxt_r[:-1] = ncols[1:], nrows[1:]
    # the merged trapezoid: the next supernode's rows plus this one's own columns
    mc = ncols + nxt_c
    mrows = ncols + nxt_r
    total = mc * mrows - mc * (mc - 1) / 2
    nnz_next = np.zeros(nf)
    nnz_next[:-1] = nnz[1:]
    zfrac = np.where(elig, (total - nnz - nnz_next) / np.maximum(total, 1), 0.0)
    nchild = np.bincount(sparent[sparent >= 0], minlength=nf).astype(np.float64)
    sub = ncols.copy()  # columns in the subtree (children precede parents)
    for f in range(nf):
        if sparent[f] >= 0:
            sub[sparent[f]] += sub[f]
    nlev = max(1, int(level.max()) + 1) if nf else 1
    return {"nf": nf, "ncols": ncols, "nrows": nrows, "nxt_c": nxt_c, "nxt_r": nxt_r, "elig": elig,
            "zfrac": zfrac, "nnz": nnz, "csq": csq, "level": level / nlev, "nchild": nchild, "sub": sub,
            "n": float(M.n), "deg": float(M.nnz) / max(M.n, 1), "sup": sup}


def sn_features(tab, rule):
    """Feature rows of every fundamental supernode under one preset rule."""
    lg = np.log1p
    nf = tab["nf"]
    am, nr, zr = PRESETS[rule][1], PRESETS[rule][2], PRESETS[rule][3]
    cols = [lg(tab["ncols"]), lg(tab["nrows"]), lg(tab["nrows"] - tab["ncols"]), lg(tab["nxt_c"]),
            lg(tab["nxt_r"]), tab["elig"].astype(np.float64), tab["zfrac"], lg(tab["nnz"]), lg(tab["csq"]),
            tab["level"].astype(np.float64), lg(tab["nchild"]), lg(tab["sub"]),
            np.full(nf, math.log1p(tab["n"])), np.full(nf, math.log1p(tab["deg"])), np.full(nf, float(am))]
    cols += [np.full(nf, math.log1p(v)) for v in nr] + [np.full(nf, v / 1000.0) for v in zr]
    return np.stack(cols, axis=1)


def supernode_times(s, ms):
    """Milliseconds of every final supernode of handle s: launch i of the factor schedule
    (ms[i + 1]; ms[0] is the zeroing and scatter of A) spread over the supernodes of its tasks in
    proportion to their flops (update tiles: 2 m n ncols(K) per entry; dense tiles: equal)."""
    sup = s.export("super")
    ncols = np.diff(sup).astype(np.float64)
    L = s.export("factor_launches").reshape(-1, 5)
    kinds = L[:, 0] & 0xffffffff
    T = s.export("tasks").reshape(-1, 4)
    U = s.export("upd_tasks").reshape(-1, 4)
    E = s.export("upd_entries").reshape(-1, 5)
    ew = 2.0 * (E[:, 1] >> 32).astype(np.float64) * (E[:, 2] & 0xffffffff).astype(np.float64) * \
        ncols[(E[:, 0] & 0xffffffff)]
    ecum = np.concatenate([[0.0], np.cumsum(ew)])
    t = np.zeros(ncols.size)
    for i in range(L.shape[0]):
        off, cnt = int(L[i, 1]), int(L[i, 2])
        if kinds[i] == 1:
            u = U[off:off + cnt]
            J = u[:, 0] & 0xffffffff
            w = ecum[u[:, 3]] - ecum[u[:, 2]]
        else:
            J = T[off:off + cnt, 0].astype(np.int64)
            w = np.ones(cnt)
        tot = w.sum()
        if tot > 0:
            np.add.at(t, J, ms[i + 1] * w / tot)
    return t


def fund_times(tab, s, ms):
    """Per fundamental supernode: its final supernode's time times its share of that supernode's
    sum c_j^2."""
    t = supernode_times(s, ms)
    sup = s.export("super")
    J = np.searchsorted(sup, tab["sup"][:-1], side="right") - 1
    csqJ = np.bincount(J, weights=tab["csq"], minlength=sup.size - 1)
    return t[J] * tab["csq"] / np.maximum(csqJ[J], 1e-30)


def profiled_factor(M, torch, precision=SYM_PREC_FP64, opt=None, rules=None):
    """(handle, per-launch milliseconds) of one profiled factorization after one warm-up."""
    if opt is None:
        opt = options(DEFAULT)
    opt.precision = precision
    s = Solver(M.n, M.Ap, M.Ai, M.perm, opt=opt, rules=rules)
    s.set_stream(torch.cuda.current_stream())
    Ax = torch.from_numpy(M.Ax).cuda()
    s.factor(Ax)
    s.profile(SYM_PROFILE_RESET)
    s.profile(SYM_PROFILE_ON)
    s.factor(Ax)
    s.profile(SYM_PROFILE_OFF)
    return s, np.asarray(sym_profile_launches(s.h, 0))


def collect_sn(mats, torch, precision=SYM_PREC_FP64, flop_budget=4e10, log=None, max_rows=None, seed=0):
    """Rows (features, log per-supernode milliseconds) over every (pattern, preset); patterns whose
    default plan exceeds flop_budget are skipped (and counted)."""
    X, Y, skipped = [], [], 0
    for gi, M in enumerate(mats):
        if _default_flops(M) > flop_budget:
            skipped += 1
            continue
        tab = fund_table(M)
        for p in range(len(PRESETS)):
            s, ms = profiled_factor(M, torch, precision, opt=options(p))
            tf = fund_times(tab, s, ms)
            s.close()
            X.append(sn_features(tab, p))
            Y.append(np.log(tf + 1e-4))
        if log:
            log(f"{gi + 1}/{len(mats)} {M.name}: {tab['nf']} fundamental supernodes")
    X = np.concatenate(X) if X else np.zeros((0, NFEAT_SN))
    Y = np.concatenate(Y) if Y else np.zeros(0)
    if max_rows and X.shape[0] > max_rows:
        idx = np.random.default_rng(seed).choice(X.shape[0], max_rows, replace=False)
        X, Y = X[idx], Y[idx]
    return X, Y, skipped


def _default_flops(M):
    s = Solver(M.n, M.Ap, M.Ai, M.perm, opt=options(DEFAULT), host_only=True)
    f = s.info().flops
    s.close()
    return f


MARGIN = 0.25  # a supernode leaves the pattern's rule only for a predicted gain above this


def choose_rules(model, M, torch, margin=MARGIN):
    """Rule per fundamental supernode, in two steps from the per-supernode predictions t(F, p):
    the preset p* with the smallest predicted total sum_F t(F, p) for the whole pattern, then,
    for each F, the preset with the smallest t(F, p) where that beats t(F, p*) by more than the
    margin (the predictions are additive only approximately; small predicted gains stay with
    p*). Returns (rules per F, p*)."""
    tab = fund_table(M)
    pred = np.exp(np.stack([model.predict(sn_features(tab, p), torch) for p in range(len(PRESETS))], axis=1))
    pstar = int(np.argmin(pred.sum(axis=0)))
    best = np.argmin(pred, axis=1)
    gain = pred[np.arange(pred.shape[0]), best] < (1.0 - margin) * pred[:, pstar]
    return np.where(gain, best, pstar).astype(np.int32), pstar


def time_graph(M, torch, precision=SYM_PREC_FP64, opt=None, rules=None, reps=3, warm=2):
    """Median CUDA-event time (ms) of sym_factor (graph replay)."""
    if opt is None:
        opt = options(DEFAULT)
    opt.precision = precision
    s = Solver(M.n, M.Ap, M.Ai, M.perm, opt=opt, rules=rules)
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


def evaluate_sn(model, mats, torch, precision=SYM_PREC_FP64, flop_budget=4e10, pattern_model=None, log=None):
    """Measured factorization time per held-out pattern: fixed rule, best single preset, the
    per-pattern choice (pattern_model, optional) and the per-supernode choice."""
    rows, skipped = [], 0
    for gi, M in enumerate(mats):
        if _default_flops(M) > flop_budget:
            skipped += 1
            continue
        t = [time_graph(M, torch, precision, opt=options(p)) for p in range(len(PRESETS))]
        fr, pstar = choose_rules(model, M, torch)
        t_sn = time_graph(M, torch, precision, rules=(RULES, fr)) if np.any(fr != pstar) else t[pstar]
        row = {"name": M.name, "fixed": t[DEFAULT], "best_preset": min(t), "per_supernode": t_sn,
               "pattern_rule_from_sn": t[pstar], "pstar": pstar,
               "rules_used": np.bincount(fr, minlength=len(PRESETS)).tolist()}
        if pattern_model is not None:
            row["per_pattern"] = t[pattern_model.choose(M, torch)]
        rows.append(row)
        if log:
            log(f"{gi + 1}/{len(mats)} {M.name}: fixed {t[DEFAULT]:.3f} best {min(t):.3f} per-supernode {t_sn:.3f}")
    gm = lambda a: float(np.exp(np.mean(np.log(a)))) if len(a) else None
    fixed = np.array([r["fixed"] for r in rows])
    out = {"patterns": len(rows), "skipped_over_budget": skipped,
           "geomean_speedup_per_supernode": gm(fixed / np.array([r["per_supernode"] for r in rows])),
           "geomean_speedup_best_preset": gm(fixed / np.array([r["best_preset"] for r in rows])),
           "geomean_speedup_pattern_rule_from_sn": gm(fixed / np.array([r["pattern_rule_from_sn"] for r in rows])),
           "supernodes_off_pattern_rule": float(np.mean([1.0 - r["rules_used"][r["pstar"]] / max(1, sum(r["rules_used"]))
                                                         for r in rows])) if rows else None,
           "total_time_ratio_per_supernode": float(fixed.sum() / sum(r["per_supernode"] for r in rows)) if rows else None}
    if pattern_model is not None and rows:
        out["geomean_speedup_per_pattern"] = gm(fixed / np.array([r["per_pattern"] for r in rows]))
    return out, rows


WEIGHTS_SN = {"fp64": os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_sn_fp64.json"),
              "fp32": os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_sn_fp32.json")}


def pretrained_sn(arm="fp64"):
    """The per-supernode network of one arm (fp64: FP64 factor; fp32: the mixed-precision FP32
    factor), trained by `python -m paper_1705_06575_gb300.costmodel sn` (its evaluation is saved
    beside the weights)."""
    return CostModel.load(WEIGHTS_SN[arm])


def suite5(count, seed, flop_budget, log=None):
    """The first `count` patterns of the suite from `seed` on within the flop budget: a spec is
    dropped when its estimate exceeds three budgets, a built pattern when its analyzed plan
    exceeds one. Returns (patterns, dropped by estimate, dropped after analysis)."""
    import workloads as w
    out, est_skip, exact_skip, i = [], 0, 0, 0
    while len(out) < count:
        spec = w.suite5_spec(i, seed)
        i += 1
        if w.suite5_estimate_flops(spec) > 3 * flop_budget:
            est_skip += 1
            continue
        M = w.suite5_build(spec)
        if _default_flops(M) > flop_budget:
            exact_skip += 1
            continue
        out.append(M)
    if log:
        log(f"suite from seed {seed}: {len(out)} patterns, {est_skip} over budget by estimate, {exact_skip} after analysis")
    return out, est_skip, exact_skip


def main_sn(argv=None):
    """Per-supernode rules: collect per-supernode times on training patterns of the suite, train
    one network per arm, evaluate on held-out patterns (disjoint seeds) by measured time.

    python -m paper_1705_06575_gb300.costmodel sn --train N --holdout H [--arms fp64,fp32] --out DIR
    python -m paper_1705_06575_gb300.costmodel sn --eval-only --holdout H --out DIR

    --eval-only evaluates the packaged networks (pretrained_sn) on the held-out patterns instead
    of training new ones (the training suite is not built)."""
    import argparse
    import sys

    import torch

    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, here)
    from . import SYM_PREC_MIXED

    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=300)
    ap.add_argument("--holdout", type=int, default=400)
    ap.add_argument("--holdout-fp32", type=int, default=None)
    ap.add_argument("--arms", default="fp64,fp32")
    ap.add_argument("--seed", type=int, default=50000)
    ap.add_argument("--budget", type=float, default=4e10)
    ap.add_argument("--max-rows", type=int, default=200000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default="costmodel_out")
    ap.add_argument("--eval-only", action="store_true")
    args = ap.parse_args(argv)
    os.makedirs(args.out, exist_ok=True)
    log = lambda m: print(m, flush=True)
    t0 = time.time()
    train, tr_est, tr_exact = suite5(0 if args.eval_only else args.train, args.seed, args.budget, log)
    hold, ho_est, ho_exact = suite5(args.holdout, args.seed + 1_000_000, args.budget, log)
    result = {"suite": "2D 5/9-point and 3D 7/27-point grids of sides 32..128, Erdos-Renyi n 50k..200k, degree 4..16",
              "flop_budget": args.budget,
              "train_patterns": len(train), "train_skipped_estimate": tr_est, "train_skipped_analysis": tr_exact,
              "holdout_patterns_requested": len(hold), "holdout_skipped_estimate": ho_est,
              "holdout_skipped_analysis": ho_exact, "arms": {}}
    for arm in args.arms.split(","):
        prec = SYM_PREC_FP64 if arm == "fp64" else SYM_PREC_MIXED
        if args.eval_only:
            model = pretrained_sn(arm)
            extra = {"weights": os.path.basename(WEIGHTS_SN[arm])}
        else:
            X, Y, _ = collect_sn(train, torch, prec, flop_budget=args.budget, max_rows=args.max_rows,
                                 log=lambda m: None)
            model, l0, l1 = CostModel.fit(X, Y, torch, steps=args.steps)
            model.save(os.path.join(args.out, f"costmodel_sn_{arm}.json"))
            extra = {"rows": int(X.shape[0]), "loss_initial": l0, "loss_final": l1}
        nh = len(hold) if arm == "fp64" or args.holdout_fp32 is None else min(len(hold), args.holdout_fp32)
        ev, rows = evaluate_sn(model, hold[:nh], torch, prec, flop_budget=args.budget, log=log)
        ev.update(extra)
        result["arms"][arm] = ev
        with open(os.path.join(args.out, f"eval_sn_{arm}_rows.json"), "w") as f:
            json.dump(rows, f)
        log(json.dumps({arm: ev}))
    result["seconds"] = time.time() - t0
    with open(os.path.join(args.out, "eval_sn.json"), "w") as f:
        json.dump(result, f, indent=1)
    print(json.dumps(result), flush=True)


WEIGHTS_PATTERN = {"fp32": os.path.join(os.path.dirname(os.path.abspath(__file__)), "costmodel_pattern_fp32.json")}


def pretrained_pattern(arm="fp32"):
    """The per-pattern network of one arm trained by `python -m paper_1705_06575_gb300.costmodel
    pattern --arm fp32 --train 400 --holdout 400` (its evaluation is saved beside the weights)."""
    return CostModel.load(WEIGHTS_PATTERN[arm])


def main_pattern(argv=None):
    """Per-pattern preset choice for one arm, on the suite at its stated sizes: the network of
    `features` (one row per preset) trained on measured graph times of every preset of the
    training patterns, then judged on held-out patterns (disjoint seeds) by measured time.

    python -m paper_1705_06575_gb300.costmodel pattern --arm fp32 --train N --holdout H --out DIR"""
    import argparse
    import sys

    import torch

    here = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, here)
    from . import SYM_PREC_MIXED

    ap = argparse.ArgumentParser()
    ap.add_argument("--arm", default="fp32", choices=["fp64", "fp32"])
    ap.add_argument("--train", type=int, default=400)
    ap.add_argument("--holdout", type=int, default=400)
    ap.add_argument("--seed", type=int, default=50000)
    ap.add_argument("--budget", type=float, default=4e10)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--out", default="costmodel_out")
    args = ap.parse_args(argv)
    os.makedirs(args.out, exist_ok=True)
    log = lambda m: print(m, flush=True)
    prec = SYM_PREC_FP64 if args.arm == "fp64" else SYM_PREC_MIXED
    t0 = time.time()

    def measure(mats):
        X, Y, G = [], [], []
        for gi, M in enumerate(mats):
            F = plan_features(M)
            t = [time_graph(M, torch, prec, opt=options(p)) for p in range(len(PRESETS))]
            X.append(F)
            Y.append(np.log(t))
            G += [gi] * len(PRESETS)
            log(f"{gi + 1}/{len(mats)} {M.name}: " + " ".join(f"{v:.3f}" for v in t))
        return np.concatenate(X), np.concatenate(Y), np.asarray(G)

    train, tr_est, tr_exact = suite5(args.train, args.seed, args.budget, log)
    hold, ho_est, ho_exact = suite5(args.holdout, args.seed + 1_000_000, args.budget, log)
    X, Y, _ = measure(train)
    model, l0, l1 = CostModel.fit(X, Y, torch, steps=args.steps)
    model.save(os.path.join(args.out, f"costmodel_pattern_{args.arm}.json"))
    Xh, Yh, Gh = measure(hold)
    ev = evaluate(model, Xh, Yh, Gh, torch)
    gm = lambda a: float(np.exp(np.mean(np.log(a))))
    T = np.exp(Yh).reshape(-1, len(PRESETS))
    ev.update({"geomean_speedup_best_preset": gm(T[:, DEFAULT] / T.min(axis=1)),
               "arm": args.arm, "train_patterns": len(train), "holdout_patterns": len(hold),
               "train_skipped_estimate": tr_est, "train_skipped_analysis": tr_exact,
               "holdout_skipped_estimate": ho_est, "holdout_skipped_analysis": ho_exact,
               "flop_budget": args.budget, "loss_initial": l0, "loss_final": l1, "seconds": time.time() - t0})
    with open(os.path.join(args.out, f"eval_pattern_{args.arm}.json"), "w") as f:
        json.dump(ev, f, indent=1)
    print(json.dumps(ev), flush=True)


def main(argv=None):
    """Collect, train and evaluate: python -m paper_1705_06575_gb300.costmodel --patterns N --out DIR
    (`sn` as the first argument: the per-supernode rules, see main_sn)."""
    import sys
    argv = sys.argv[1:] if argv is None else argv
    if argv and argv[0] == "sn":
        return main_sn(argv[1:])
    if argv and argv[0] == "pattern":
        return main_pattern(argv[1:])
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
