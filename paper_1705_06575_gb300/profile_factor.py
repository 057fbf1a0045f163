"""Profiling driver: factor one named workload and report where the time goes.

    python -m paper_1705_06575_gb300.profile_factor --workload conduct3d7_48 [--one-stream]
        [--no-graphs] [--mixed [--no-tensor-cores]] [--levels] [--repeat N] [--batch B [--autotune]]
        [--solve NRHS]

Without --levels it factors the matrix once per repeat (after one warm-up factorization) and
exits: a fixed, short command to run under a profiler. With --one-stream --no-graphs every launch
of the schedule executes in list order, so a profiler's launch index equals the index in
sym_export(FACTOR_LAUNCHES) among launches of the same kernel. With --levels it runs one
profiled factorization (CUDA events around every launch, one stream) and prints a JSON summary:
per level of the supernodal tree and per kernel kind the milliseconds, launches and tasks, the
serialised total and the time a two-stream schedule would take if both streams' launches kept
their serialised durations (an upper bound on what the lookahead can overlap). With --batch B the
same runs on B value sets of the pattern at once (sym_factor_batch, and sym_solve_batch with
--solve), --levels adding the solve's milliseconds per kernel kind.
"""
from __future__ import annotations

import argparse
import json
import os
import sys

import numpy as np

from . import (SYM_FLAG_NO_GRAPHS, SYM_FLAG_NO_TENSOR_CORES, SYM_FLAG_ONE_STREAM, SYM_PROFILE_OFF,
               SYM_PROFILE_ON, SYM_PROFILE_RESET, Solver, sym_autotune, sym_factor_batch, sym_profile,
               sym_profile_launches, sym_profile_read, sym_solve_batch, sym_solve_multi)

KIND_NAMES = {1: "update", 2: "potrf", 3: "trsm", 4: "gemm", 5: "trtri"}
SOLVE_KIND_NAMES = {11: "fgather", 12: "fstep", 13: "fpush", 14: "bgather", 15: "bstep", 16: "fsum", 17: "perm"}


def level_summary(s, ms):
    """Per-level breakdown of one profiled factorization (ms: sym_profile_launches(h, 0))."""
    raw = s.export("factor_launches").reshape(-1, 5)
    kind = raw[:, 0] & 0xffffffff
    level = raw[:, 0] >> 32
    count = raw[:, 2]
    stream = raw[:, 3] >> 32
    wait = (raw[:, 4] & 0xffffffff).astype(np.uint32).astype(np.int32)
    if len(ms) != len(raw) + 1:
        raise RuntimeError(f"{len(ms)} timed launches for a schedule of {len(raw)} (+1 scatter)")
    t = np.asarray(ms[1:])
    end = np.zeros(len(raw))
    tail = {0: 0.0, 1: 0.0}
    for i in range(len(raw)):
        st = int(stream[i])
        start = tail[st] if wait[i] < 0 else max(tail[st], end[wait[i]])
        end[i] = start + t[i]
        tail[st] = end[i]
    levels = []
    for lv in range(int(level.max()) + 1 if len(raw) else 0):
        row = {"level": lv}
        for k, name in KIND_NAMES.items():
            sel = (level == lv) & (kind == k)
            if sel.any():
                row[name] = {"ms": round(float(t[sel].sum()), 3), "launches": int(sel.sum()),
                             "tasks": int(count[sel].sum())}
        row["aux_stream_ms"] = round(float(t[(level == lv) & (stream == 1)].sum()), 3)
        levels.append(row)
    return {"scatter_ms": float(ms[0]), "serialised_ms": float(t.sum()),
            "two_stream_bound_ms": float(max(tail.values())), "levels": levels}


def solve_level_summary(s, ms):
    """Per level and kernel kind, the milliseconds of one profiled solve of up to 8 right-hand
    sides (ms: sym_profile_launches(h, 1): the permutation in, the forward and backward launch
    lists, the permutation out)."""
    rows = {}
    lists = [s.export("fwd_launches").reshape(-1, 5), s.export("bwd_launches").reshape(-1, 5)]
    if len(ms) != 2 + sum(len(x) for x in lists):
        return {"error": f"{len(ms)} timed launches"}
    i = 1
    for raw in lists:
        for rec in raw:
            kind, level = int(rec[0] & 0xffffffff), int(rec[0] >> 32)
            key = f"{level}:{SOLVE_KIND_NAMES.get(kind, kind)}"
            rows[key] = round(rows.get(key, 0.0) + float(ms[i]), 3)
            i += 1
    return rows


def main(argv=None):
    import torch

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import workloads as w

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="conduct3d7_48")
    ap.add_argument("--one-stream", action="store_true")
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--mixed", action="store_true", help="FP32 factor (SYM_PREC_MIXED)")
    ap.add_argument("--no-tensor-cores", action="store_true", help="FP32 updates on the SIMT pipes")
    ap.add_argument("--levels", action="store_true")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--batch", type=int, default=0,
                    help="factor this many value sets of the workload's pattern together (sym_factor_batch)")
    ap.add_argument("--solve", type=int, default=0,
                    help="after the factorizations, solve with this many right-hand sides (repeat + 1 times)")
    ap.add_argument("--autotune", action="store_true", help="batches: run sym_autotune first")
    args = ap.parse_args(argv)
    M = w.cfg(args.workload)
    flags = ((SYM_FLAG_ONE_STREAM if args.one_stream else 0) | (SYM_FLAG_NO_GRAPHS if args.no_graphs else 0) |
             (SYM_FLAG_NO_TENSOR_CORES if args.no_tensor_cores else 0))
    s = Solver(M.n, M.Ap, M.Ai, M.perm, flags=flags, precision="mixed" if args.mixed else None)
    if args.batch > 1:  # value sets drawn like the workload's (same pattern, seeds 0..batch-1)
        nb = args.batch
        vals = np.stack([w.cfg(args.workload, b).Ax for b in range(nb)])
        V = torch.from_numpy(vals).cuda()
        out = {"workload": args.workload, "batch": nb}
        if args.autotune:
            out["autotune"] = sym_autotune(s.h, nb, V, M.nnz, 2)
        B = X = None
        if args.solve > 0:
            B = torch.from_numpy(np.random.default_rng(5).standard_normal((nb, args.solve, M.n))).cuda()
            X = torch.empty_like(B)

        def step():
            sym_factor_batch(s.h, nb, V, M.nnz)
            if B is not None:
                sym_solve_batch(s.h, nb, args.solve, B, M.n, args.solve * M.n, X, M.n, args.solve * M.n)

        for _ in range(args.repeat + 1):
            step()
        torch.cuda.synchronize()
        if args.levels:
            sym_profile(s.h, SYM_PROFILE_RESET)
            sym_profile(s.h, SYM_PROFILE_ON)
            step()
            torch.cuda.synchronize()
            sym_profile(s.h, SYM_PROFILE_OFF)
            out.update(level_summary(s, sym_profile_launches(s.h, 0)))
            if B is not None:
                out["solve_kinds_ms"] = {name: round(sym_profile_read(s.h, k)[0], 3)
                                         for k, name in SOLVE_KIND_NAMES.items() if sym_profile_read(s.h, k)[1]}
                out["solve_levels"] = solve_level_summary(s, sym_profile_launches(s.h, 1))
        out.update({"steps": args.repeat + 1 + (1 if args.levels else 0), "status": "ok"})
        print(json.dumps(out))
        s.close()
        return 0
    Ax = torch.from_numpy(M.Ax).cuda()
    s.factor(Ax)  # warm-up (and graph capture unless --no-graphs)
    torch.cuda.synchronize()
    if args.levels:
        sym_profile(s.h, SYM_PROFILE_RESET)
        sym_profile(s.h, SYM_PROFILE_ON)
        s.factor(Ax)
        torch.cuda.synchronize()
        sym_profile(s.h, SYM_PROFILE_OFF)
        out = level_summary(s, sym_profile_launches(s.h, 0))
        out["workload"] = args.workload
        if args.solve > 0:  # one profiled solve: milliseconds per level and kernel kind
            B = torch.from_numpy(np.ascontiguousarray(w.rhs(M.n, args.solve, np.random.default_rng(7)).T)).cuda()
            X = torch.empty_like(B)
            sym_solve_multi(s.h, args.solve, B, M.n, X, M.n)
            torch.cuda.synchronize()
            sym_profile(s.h, SYM_PROFILE_RESET)
            sym_profile(s.h, SYM_PROFILE_ON)
            sym_solve_multi(s.h, args.solve, B, M.n, X, M.n)
            torch.cuda.synchronize()
            sym_profile(s.h, SYM_PROFILE_OFF)
            out["solve_levels"] = solve_level_summary(s, sym_profile_launches(s.h, 1))
        print(json.dumps(out))
    else:
        for _ in range(args.repeat):
            s.factor(Ax)
        out = {"workload": args.workload, "factorizations": args.repeat + 1, "status": "ok"}
        if args.solve > 0:
            B = torch.from_numpy(np.ascontiguousarray(w.rhs(M.n, args.solve, np.random.default_rng(7)).T)).cuda()
            X = torch.empty_like(B)
            for _ in range(args.repeat + 1):
                sym_solve_multi(s.h, args.solve, B, M.n, X, M.n)
            out["solves"] = args.repeat + 1
        torch.cuda.synchronize()
        print(json.dumps(out))
    s.close()
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
