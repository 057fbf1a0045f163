#!/usr/bin/env python
"""Benchmark of the numeric refactorization + solve (one JSON line on stdout).

Workload: the 64^3 7-point conductivity matrix (n = 262,144; per-edge w ~ U(0.5, 2.0), diagonal
sum of w + 1e-3; geometric nested dissection), 4 right-hand sides b ~ N(0,1), FP64. One step is
the whole hot path on one set of values: scatter of A into the supernodal panels, the level-
scheduled supernodal left-looking factorization, and the forward + backward solve of the 4
right-hand sides. The pattern is analyzed once, outside the timed region (the paper times the
numeric phase on a fixed pattern).

value  = factor flops (sum of squared column counts of L) per step / step time, summed over ranks
e2e    = the same metric through the host-pointer C ABI (H2D of A's values and B, D2H of X)
roofline: the kernel kind with the largest share of the step, against the measured FP64 FMA peak
cpu_baseline / --impl reference: the CPU FP64 oracle (up-looking factor), single thread, timed on
the leading block of the same matrix (a bounded sample; see --cpu-flops).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "conduct3d7_64"
WORKLOADS = {
    "conduct3d7_64": "64^3 7-point conductivity (n=262144, w~U(0.5,2), diag=sum w+1e-3), geometric "
                     "nested dissection, 4 RHS b~N(0,1), FP64",
    # smaller cases of the same family, for profiler captures and quick checks
    "conduct3d7_48": "48^3 7-point conductivity (n=110592), same recipe",
    "conduct3d27_40": "40^3 27-point conductivity (n=64000), same recipe",
    "laplace2d5_64": "64^2 5-point (n=4096), diag 4+U(0,0.1), off -U(0.9,1.1)",
}
WORKLOAD_DESC = WORKLOADS[WORKLOAD]
NRHS = 4
METRIC = "refactor GFLOP/s and ms/(factor+solve) vs plain FP64 GPU path at bwd err<=1e-12"
# DRAM traffic of the dominant kernel (the FP64 update, k_update_flat) per launch of the 64^3
# step, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum averaged over the 19
# update launches of one step). It holds only for the kernel source it was taken on: the
# sha256 (first 16 hex digits) of the kernel's definition text in csrc/kernels.cu. When that
# text changes, the line reports null until the traffic is captured again.
UPDATE_TRAFFIC = {"bytes_per_launch": 5.4518e8, "kernel_sha16": "6f9b0de4cc0dd30c"}

CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def kernel_source_sha16(name="k_update_flat"):
    """sha256 (16 hex digits) of the definition of a kernel template in csrc/kernels.cu: from the
    template line before the kernel's name to the first closing brace at column 0."""
    import hashlib
    import re
    src = open(os.path.join(ROOT, "paper_1705_06575_gb300", "csrc", "kernels.cu")).read()
    m = re.search(r"\ntemplate <[^\n]*>\n[^\n]*\n\s*" + re.escape(name) + r"\(", src)
    if not m:
        return None
    end = src.index("\n}\n", m.start())
    return hashlib.sha256(src[m.start():end + 3].encode()).hexdigest()[:16]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_aggregate(ms, units, world):
    """Whole-job figures of one timed region: the slowest rank's time and the units of work all
    ranks processed (each rank runs its own replica or its own shard; no data exchange)."""
    if world <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def shard(count, rank, world):
    """Contiguous share [lo, hi) of count independent matrices for one rank."""
    per, extra = divmod(count, world)
    lo = rank * per + min(rank, extra)
    return lo, lo + per + (1 if rank < extra else 0)


def start_clock_sampler(path):
    try:
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={CLOCK_QUERY}", "--format=csv", "-lms", "200"],
                                stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except (FileNotFoundError, OSError):
        return None


def read_clocks(path, gpu_index):
    try:
        lines = [l.strip() for l in open(path) if l.strip()]
    except OSError:
        return None
    if len(lines) < 2:
        return None
    head = [h.strip() for h in lines[0].split(",")]
    sm, smax, reasons = [], [], set()
    names = {"clocks_event_reasons.hw_slowdown": "hw_slowdown",
             "clocks_event_reasons.hw_thermal_slowdown": "hw_thermal_slowdown",
             "clocks_event_reasons.sw_thermal_slowdown": "sw_thermal_slowdown",
             "clocks_event_reasons.sw_power_cap": "sw_power_cap"}
    for l in lines[1:]:
        f = [x.strip() for x in l.split(",")]
        if len(f) != len(head):
            continue
        row = dict(zip(head, f))
        if row.get("index") not in (str(gpu_index), None):
            continue
        try:
            sm.append(float(row["clocks.current.sm [MHz]"].split()[0]))
            smax.append(float(row["clocks.max.sm [MHz]"].split()[0]))
        except (KeyError, ValueError):
            continue
        for k, v in row.items():
            for key, nm in names.items():
                if k.startswith(key) and v.lower() == "active":
                    reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "samples": len(sm),
            "reasons": sorted(reasons)}


def backward_error(M, B, X):
    """Normwise backward error max_c ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    import scipy.sparse as sp
    L = sp.csc_matrix((M.Ax, M.Ai, M.Ap), shape=(M.n, M.n))
    A = L + sp.tril(L, -1).T
    anorm = abs(A).sum(axis=1).max()
    R = B - A @ X
    return float(max(np.abs(R[:, c]).max() / (anorm * np.abs(X[:, c]).max() + np.abs(B[:, c]).max())
                     for c in range(B.shape[1])))


def leading_block(o, target_flops):
    """Smallest k whose leading k x k factor has at least target_flops flops, and those flops.

    flops(k) = sum_j |L_j ∩ [0, k)|^2; an entry at position t of column j (t = 0 for the
    diagonal) raises that sum by 2t + 1 once k passes its row, so flops(k) is a prefix sum."""
    t = np.arange(o.Li.size, dtype=np.float64) - np.repeat(o.Lp[:-1], np.diff(o.Lp)).astype(np.float64)
    per_row = np.bincount(o.Li, weights=2.0 * t + 1.0, minlength=o.n)
    cum = np.cumsum(per_row)  # cum[k-1] = flops(k)
    k = int(np.searchsorted(cum, target_flops)) + 1
    k = min(k, o.n)
    return k, float(cum[k - 1])


def oracle_sample(M, target_flops, repeats=1):
    """Time the CPU oracle (single thread) on the leading block of the matrix whose factor has
    about target_flops flops. Returns (GFLOP/s, seconds per run, kmax, sample flops, oracle)."""
    import oracle
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    kmax, fl = leading_block(o, target_flops)
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        rc = o.factor(M.Ax, kmax)
        times.append(time.perf_counter() - t0)
        assert rc == 0
    t = float(np.median(times))
    return fl / t / 1e9, t, kmax, fl, o


def block_entry_error(o, kmax, sx, Lx):
    """max |L_gpu - L_oracle| / max |L_oracle| over the entries of the leading kmax x kmax block,
    which the oracle's up-looking factorization computed exactly. sx: the library's exports
    (super, rowptr, rows, lxptr); Lx: its panels (widened to float64)."""
    sup, rowptr, rows, lxptr = sx["super"], sx["rowptr"], sx["rows"], sx["lxptr"]
    err = ref_max = 0.0
    for J in range(sup.size - 1):
        f, l = int(sup[J]), int(sup[J + 1])
        if f >= kmax:
            break
        l2 = min(l, kmax)
        R = rows[rowptr[J]:rowptr[J + 1]]
        panel = Lx[lxptr[J]:lxptr[J + 1]].reshape(l - f, R.size)
        lo, hi = int(o.Lp[f]), int(o.Lp[l2])
        rr = o.Li[lo:hi]
        cc = np.repeat(np.arange(l2 - f), np.diff(o.Lp[f:l2 + 1]))
        keep = rr < kmax
        got = panel[cc[keep], np.searchsorted(R, rr[keep])]
        ref = o.Lx[lo:hi][keep]
        if ref.size:
            err = max(err, float(np.abs(got - ref).max()))
            ref_max = max(ref_max, float(np.abs(ref).max()))
    return err / ref_max if ref_max > 0 else 0.0


def solver_exports(s):
    return {k: s.export(k) for k in ("super", "rowptr", "rows", "lxptr")}


def sig4(x):
    """Floats of a nested result rounded to 4 significant digits (keeps the line short)."""
    if isinstance(x, float):
        return float(f"{x:.4g}")
    if isinstance(x, dict):
        return {k: sig4(v) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig4(v) for v in x]
    return x


def make_workload(name):
    import workloads as w
    return w.cfg(name)


def line_config(M, workload, world):
    """The config object of the line, identical for both arms."""
    return {"workload": workload, "description": WORKLOADS[workload], "n": int(M.n), "nnz_a_lower": int(M.nnz),
            "nrhs": NRHS, "parallelism": f"replicas x{world}",
            "l2": "no flush: the factor's 1.57 GB working set exceeds the 129 MB L2"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    M = make_workload(args.workload)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    kmax, fl = leading_block(o, args.ref_flops)
    for _ in range(args.warmup):
        o.factor(M.Ax, kmax)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        rc = o.factor(M.Ax, kmax)
        ts.append(time.perf_counter() - t0)
        assert rc == 0
    t = float(np.mean(ts))
    val = fl / t / 1e9
    sample = (f"up-looking FP64 oracle factor of the leading {kmax} x {kmax} block of the workload "
              f"matrix ({fl:.3g} flops), single thread, per step")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": line_config(M, args.workload, world),
            "cpu_baseline": {"value": val, "unit": "GFLOP/s", "cores": 1, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_kinds(S, s, fn, steps, names=None):
    """Per-kind CUDA-event milliseconds of steps calls of fn, launched kernel by kernel."""
    s.profile(S.SYM_PROFILE_RESET)
    s.profile(S.SYM_PROFILE_ON)
    for _ in range(steps):
        fn()
    import torch
    torch.cuda.synchronize()
    s.profile(S.SYM_PROFILE_OFF)
    kinds = {}
    for name, kid in S.KINDS.items():
        if names and name not in names:
            continue
        kms, knl, kfl = s.profile_read(kid)
        if knl:
            kinds[name] = {"ms_per_step": kms / steps, "launches_per_step": knl / steps,
                           "gflops_alg": kfl / kms / 1e6 if kms > 0 else None}
    return kinds


def bench_mixed(S, torch, M, B, flops, args, stream, barrier, world, ref=None):
    """The mixed-precision form on the same matrix and right-hand sides: FP32 factor + FP64
    conjugate gradients preconditioned by it, to backward error <= 1e-12 on every right-hand
    side. Timed like the main step (scatter + factor + solve). ref = (oracle, kmax) gives the FP32
    factor's entry-wise error against the oracle on the leading block it factored."""
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.set_stream(stream)
    s.set_refinement(1e-12, 100)
    Ax = torch.from_numpy(M.Ax).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xt = torch.empty_like(Bt)

    def step():
        s.factor(Ax)
        S.sym_solve_multi(s.h, NRHS, Bt, M.n, Xt, M.n)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1) / args.steps
    ms, _ = dist_aggregate(ms, 0.0, world)
    it, _ = s.refinement_info()
    X = Xt.cpu().numpy().T
    berr = backward_error(M, B, X)
    ms_f = _event_ms(torch, stream, lambda: s.factor(Ax), args.steps)
    kinds = profile_kinds(S, s, lambda: s.factor(Ax), args.steps,
                          ("scatter", "update", "potrf", "trsm", "gemm", "trtri"))
    out = {"ms": ms, "ms_factor": ms_f, "ms_solve": ms - ms_f, "it": it, "berr": berr}
    if ref is not None:
        out["factor_err_vs_oracle"] = block_entry_error(ref[0], ref[1], solver_exports(s), s.factor_panels())
    s.close()
    return out, kinds


def bench_batched(S, torch, args, stream, barrier, world):
    """Batched refactorization: 512 value sets on one 128 x 128 9-point pattern (w ~ U(0.5, 2),
    diagonal 1.05 sum |w|), one right-hand side each, factor + solve of the whole batch per step,
    against the same work done by one-matrix calls in sequence (timed on 16 and scaled to 512)."""
    import workloads as w
    nb = args.batch
    M, vals = w.same_pattern_batch(lambda r: w.dd2d9(128, r), nb, 2000)
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.set_stream(stream)
    info = s.info()
    V = torch.from_numpy(vals).cuda()
    B = torch.from_numpy(np.random.default_rng(5).standard_normal((nb, M.n))).cuda()
    X = torch.empty_like(B)

    def step():
        S.sym_factor_batch(s.h, nb, V, M.nnz)
        S.sym_solve_batch(s.h, nb, 1, B, M.n, M.n, X, M.n, M.n)

    tuned, changed = S.sym_autotune(s.h, nb, V, M.nnz, 2)  # kernel forms of the small-tile launches
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ms, _ = dist_aggregate(ms, 0.0, world)  # every rank factors its own batch: the slowest rank
    kinds = profile_kinds(S, s, step, args.steps)
    Xh = X.cpu().numpy()
    worst = 0.0
    for b in (0, nb // 2, nb - 1):
        Mb = w.Matrix(M.n, M.Ap, M.Ai, vals[b])
        worst = max(worst, backward_error(Mb, B[b].cpu().numpy()[:, None], Xh[b][:, None]))
    # the same work, one matrix per call
    one = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    one.set_stream(stream)
    xs = torch.empty(M.n, dtype=torch.float64, device="cuda")
    nseq = min(16, nb)
    for b in range(2):
        one.factor(V[b])
        S.sym_solve(one.h, B[b], xs)
    torch.cuda.synchronize()
    e0.record(stream)
    for b in range(nseq):
        one.factor(V[b])
        S.sym_solve(one.h, B[b], xs)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_seq = e0.elapsed_time(e1) / nseq * nb
    s.close()
    one.close()
    return {"ms": ms, "gflops": info.flops * nb * world / (ms * 1e-3) / 1e9, "x_seq": ms_seq / ms,
            "berr": worst, "autotuned": f"{changed}/{tuned}"}, kinds


def _event_ms(torch, stream, fn, reps):
    """Milliseconds per call of fn over reps calls, CUDA events on stream (after 3 warm-ups)."""
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def bench_small_latency(S, torch, stream):
    """The small 2D case (64^2 5-point, n = 4096, one right-hand side): launch- and
    latency-bound, reported in microseconds per factor + solve with its level count."""
    import workloads as w
    M = w.cfg("laplace2d5_64")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.set_stream(stream)
    info = s.info()
    Ax = torch.from_numpy(M.Ax).cuda()
    b = torch.from_numpy(w.rhs(M.n, 1, np.random.default_rng(7))[:, 0].copy()).cuda()
    x = torch.empty_like(b)
    us_f = 1e3 * _event_ms(torch, stream, lambda: s.factor(Ax), 50)
    us_s = 1e3 * _event_ms(torch, stream, lambda: S.sym_solve(s.h, b, x), 50)
    us = 1e3 * _event_ms(torch, stream, lambda: (s.factor(Ax), S.sym_solve(s.h, b, x)), 50)
    berr = backward_error(M, b.cpu().numpy()[:, None], x.cpu().numpy()[:, None])
    s.close()
    return {"us": us, "us_factor": us_f, "us_solve": us_s, "levels": info.nlevels,
            "launches": int(info.nlaunch_factor + info.nlaunch_solve), "berr": berr}


def bench_uneven_batch(S, torch, stream, precision="fp64"):
    """An uneven batch: 256 independent 5-point grids with sides uniform in 32..256, factored and
    solved (one right-hand side) as one block-diagonal matrix with one plan, in FP64 or as the
    mixed-precision form (FP32 factor, FP64 refinement to backward error <= 1e-12)."""
    import workloads as w
    mats, sides = w.uneven_grid_batch(256, np.random.default_rng(3000))
    U = w.block_diagonal(mats)
    s = S.Solver(U.n, U.Ap, U.Ai, U.perm, precision=precision)
    s.set_stream(stream)
    if precision == "mixed":
        s.set_refinement(1e-12, 100)
    info = s.info()
    Ax = torch.from_numpy(U.Ax).cuda()
    b = torch.from_numpy(w.rhs(U.n, 1, np.random.default_rng(8))[:, 0].copy()).cuda()
    x = torch.empty_like(b)
    ms = _event_ms(torch, stream, lambda: (s.factor(Ax), S.sym_solve(s.h, b, x)), 5)
    berr = backward_error(U, b.cpu().numpy()[:, None], x.cpu().numpy()[:, None])
    s.close()
    return {"ms": ms, "gflops": info.flops / (ms * 1e-3) / 1e9, "berr": berr}


def bench_mixed_vector(S, torch, stream):
    """The 3-dof vector problem (48^3 nodes x 3, 27-point coupling, coefficients 1 / 1e2 / 1e4 by
    subdomain): FP32 factor + FP64 conjugate-gradient refinement to backward error <= 1e-12 for
    one right-hand side, with the refinement's iteration count, against one FP64 factorization."""
    import workloads as w
    M = w.cfg("vector3d27_48")
    b = torch.from_numpy(w.rhs(M.n, 1, np.random.default_rng(9))[:, 0].copy()).cuda()
    x = torch.empty_like(b)
    Ax = torch.from_numpy(M.Ax).cuda()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.set_stream(stream)
    s.set_refinement(1e-12, 200)
    ms_f = _event_ms(torch, stream, lambda: s.factor(Ax), 3)
    ms = _event_ms(torch, stream, lambda: (s.factor(Ax), S.sym_solve(s.h, b, x)), 3)
    it, _ = s.refinement_info()
    berr = backward_error(M, b.cpu().numpy()[:, None], x.cpu().numpy()[:, None])
    s.close()
    d = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    d.set_stream(stream)
    ms_f64 = _event_ms(torch, stream, lambda: d.factor(Ax), 1)
    d.close()
    return {"ms": ms, "ms_f32": ms_f, "ms_f64_factor": ms_f64, "it": it, "berr": berr}


def bench_conduct27(S, torch, stream):
    """The 27-point 40^3 conductivity matrix (n = 64,000; dense separators of up to ~2400
    columns): FP64 factor + 4-RHS solve per step."""
    import workloads as w
    M = w.cfg("conduct3d27_40")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.set_stream(stream)
    info = s.info()
    Ax = torch.from_numpy(M.Ax).cuda()
    B = w.rhs(M.n, NRHS, np.random.default_rng(11))
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xt = torch.empty_like(Bt)
    ms = _event_ms(torch, stream, lambda: (s.factor(Ax), S.sym_solve_multi(s.h, NRHS, Bt, M.n, Xt, M.n)), 10)
    berr = backward_error(M, B, Xt.cpu().numpy().T)
    s.close()
    return {"ms": ms, "gflops": info.flops / (ms * 1e-3) / 1e9, "berr": berr}


def bench_auto_order(S, torch, M, B, stream):
    """The benchmark matrix under the inspector's own ordering (SYM_ORDER_AUTO) instead of the
    geometric nested dissection: analysis time, factor flops, and FP64 factor + 4-RHS solve."""
    t0 = time.perf_counter()
    s = S.Solver(M.n, M.Ap, M.Ai, ordering="auto")
    analyze_s = time.perf_counter() - t0
    s.set_stream(stream)
    info = s.info()
    Ax = torch.from_numpy(M.Ax).cuda()
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xt = torch.empty_like(Bt)
    ms = _event_ms(torch, stream, lambda: (s.factor(Ax), S.sym_solve_multi(s.h, NRHS, Bt, M.n, Xt, M.n)), 5)
    berr = backward_error(M, B, Xt.cpu().numpy().T)
    s.close()
    return {"ms": ms, "flops": info.flops, "gflops": info.flops / (ms * 1e-3) / 1e9, "analyze_s": analyze_s,
            "method": "nd" if info.ordering_method == S.SYM_ORDER_METHOD_ND else "md", "berr": berr}


def bench_sparse_rhs(S, torch, s, M, args, stream):
    """Forward solve L y = P b for sparse b over the reach set (VI-Prune + VS-Block) on the
    benchmark matrix: b = one column of A (a local source) and b with 1% random nonzeros, each
    against the same solve for a full b (every supernode visited, i.e. no pruning)."""
    rng = np.random.default_rng(77)
    j = M.n // 3
    cases = {"colA": M.Ai[M.Ap[j]:M.Ap[j + 1]].astype(np.int32),
             "rand1pct": rng.choice(M.n, size=M.n // 100, replace=False).astype(np.int32),
             "full": np.arange(M.n, dtype=np.int32)}
    out = {}
    for name, bidx in cases.items():
        r = S.Reach(s.h, bidx)
        bv = torch.from_numpy(rng.standard_normal(bidx.size)).cuda()
        xv = torch.empty(r.size(), dtype=torch.float64, device="cuda")
        out[name + "_ms"] = _event_ms(torch, stream, lambda: r.solve(bv, xv), args.steps)
        out[name + "_reach"] = r.size()
        r.close()
    return out


def run_ours(args):
    import torch

    import paper_1705_06575_gb300 as S
    import workloads as w

    rank, world, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    M = make_workload(args.workload)  # every rank factors its own replica (independent problems)
    t0 = time.perf_counter()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    analyze_s = time.perf_counter() - t0
    info = s.info()
    # kernels per step: the factor's and the FP64 solve's (sym_info; the fused narrow levels of an
    # FP64 solve skip the same launches for any number of right-hand sides)
    launches_step = int(info.nlaunch_factor + info.nlaunch_solve)
    stream = torch.cuda.current_stream()
    s.set_stream(stream)
    Ax = torch.from_numpy(M.Ax).cuda()
    B = w.rhs(M.n, NRHS, np.random.default_rng(1000 * 1 + 7))
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()  # row q = right-hand side q
    Xt = torch.empty_like(Bt)
    peak64 = S.sym_fma_peak(64)

    def step():
        s.factor(Ax)
        S.sym_solve_multi(s.h, NRHS, Bt, M.n, Xt, M.n)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # raw nvidia-smi samples of the timed region (summarised in the line's "clocks"); the
    # directory can be chosen with SYM_BENCH_CLOCKS_DIR
    clock_dir = os.environ.get("SYM_BENCH_CLOCKS_DIR", tempfile.gettempdir())
    clock_path = os.path.join(clock_dir, f"bench_clocks_r{rank}.csv")
    os.makedirs(clock_dir, exist_ok=True)
    sampler = start_clock_sampler(clock_path) if rank == 0 else None
    time.sleep(0.3 if sampler else 0)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    if sampler:
        sampler.terminate()
        sampler.wait()
    ms_step = ev0.elapsed_time(ev1) / args.steps
    # Per-kernel breakdown: the same K steps again, launched kernel by kernel with a CUDA event
    # after every launch on the launching stream (the timed steps above replay CUDA graphs).
    kinds = profile_kinds(S, s, step, args.steps)
    ms_step, total_flops = dist_aggregate(ms_step, info.flops, world)
    X = Xt.cpu().numpy().T
    berr = backward_error(M, B, X)

    factor_kinds = ("scatter", "update", "potrf", "trsm", "gemm", "trtri")
    ms_factor_kernels = sum(kinds[k]["ms_per_step"] for k in factor_kinds if k in kinds)
    ms_solve_kernels = sum(v["ms_per_step"] for k, v in kinds.items() if k not in factor_kinds)
    # the factor alone as the timed step runs it (graph replay), so the solve's share of the step
    ms_factor = _event_ms(torch, stream, lambda: s.factor(Ax), args.steps)
    dom = max(kinds, key=lambda k: kinds[k]["ms_per_step"])
    dms, dnl, dfl = s.profile_read(S.KINDS[dom])
    peak_tf = peak64 / 1e3
    exec_tf = dfl / dms / 1e9  # executed flops (explicit zeros of amalgamated panels included) / ms
    # The method's useful work: for the update kernel the exact-pattern share of sum c_j^2
    # (sym_stats.update_flops); other kernels have no such split and report executed flops.
    useful = info.update_flops * args.steps if dom == "update" else dfl
    achieved_tf = useful / dms / 1e9
    kname = {"update": "k_update_flat"}.get(dom, f"k_{dom}")  # the FP64 update kernel
    traffic = None
    if (dom == "update" and args.workload == WORKLOAD and UPDATE_TRAFFIC["bytes_per_launch"] is not None
            and UPDATE_TRAFFIC["kernel_sha16"] == kernel_source_sha16("k_update_flat")):
        traffic = UPDATE_TRAFFIC["bytes_per_launch"]
    roofline = {"bound": "alu", "kernel": kname, "achieved": achieved_tf, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved_tf / peak_tf, "frac_executed": exec_tf / peak_tf,
                "flops": "useful (exact pattern, no amalgamation zeros); frac_executed counts executed flops",
                "traffic": traffic, "launches_per_step": dnl / args.steps,
                "peak_source": "FP64 FMA peak measured live by sym_fma_peak (152 SMs x 2 DFMA/clk)",
                "share_of_step": dms / args.steps / ms_step,
                "timing": "kernel time from CUDA events in a profiled pass of the same K steps"}

    # End to end through the host-pointer C ABI: pinned host buffers, copies inside the timing.
    Ax_h = torch.from_numpy(M.Ax).pin_memory()
    B_h = torch.from_numpy(np.asfortranarray(B).T.copy()).pin_memory()
    X_h = torch.empty_like(B_h).pin_memory()

    def e2e_step():
        S.sym_factor_host(s.h, Ax_h.data_ptr())
        S.sym_solve_host_ptr(s.h, NRHS, B_h.data_ptr(), M.n, X_h.data_ptr(), M.n)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2)
    for _ in range(e2e_steps):
        e2e_step()
    torch.cuda.synchronize()
    t_e2e = (time.perf_counter() - t0) / e2e_steps
    t_e2e, _ = dist_aggregate(t_e2e, 0.0, world)
    berr_e2e = backward_error(M, B, X_h.numpy().T)

    cpu = None
    ref = None
    factor_vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        g, t, kmax, fl, o = oracle_sample(M, args.cpu_flops)
        cpu = {"value": g, "unit": "GFLOP/s", "cores": 1, "host_cores": os.cpu_count(), "kind": "oracle",
               "sample": (f"up-looking FP64 oracle factor of the leading {kmax} x {kmax} block of the "
                          f"workload matrix ({fl:.3g} flops, {t:.1f} s), single thread")}
        ref = (o, kmax)
        s.factor(Ax)
        torch.cuda.synchronize()
        factor_vs_oracle = {"block": kmax,
                            "fp64": block_entry_error(o, kmax, solver_exports(s), s.factor_panels())}

    variants, detail = {}, {"kernels": kinds}
    if not args.no_variants:
        variants["mixed_64"], detail["mixed_64_factor_kernels"] = bench_mixed(
            S, torch, M, B, info.flops, args, stream, barrier, world, ref)
        variants["mixed_64"]["x_vs_fp64"] = ms_step / variants["mixed_64"]["ms"]
        if factor_vs_oracle is not None and "factor_err_vs_oracle" in variants["mixed_64"]:
            factor_vs_oracle["fp32_mixed"] = variants["mixed_64"].pop("factor_err_vs_oracle")
        if args.batch > 0:
            variants["batch_512x128sq"], detail["batch_kernels"] = bench_batched(S, torch, args, stream, barrier,
                                                                                 world)
        variants["sparse_rhs"] = bench_sparse_rhs(S, torch, s, M, args, stream)
        variants["auto_order_64"] = bench_auto_order(S, torch, M, B, stream)
        for key, fn in (("lat_64sq", bench_small_latency), ("uneven_256", bench_uneven_batch),
                        ("uneven_256_mixed", lambda S_, t_, st_: bench_uneven_batch(S_, t_, st_, "mixed")),
                        ("c27_40", bench_conduct27), ("vec48_mixed", bench_mixed_vector)):
            try:
                variants[key] = fn(S, torch, stream)
            except S.SymError as e:  # a library error is reported, not fatal to the main line
                variants[key] = {"error": str(e)}
    clocks = read_clocks(clock_path, local) if rank == 0 else None
    value = total_flops / (ms_step * 1e-3) / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": line_config(M, args.workload, world),
        "gpu_launches": int(args.steps * launches_step),
        "clocks": clocks,
        "e2e": {"value": total_flops / t_e2e / 1e9, "unit": "GFLOP/s", "ms_per_step": t_e2e * 1e3,
                "h2d_bytes_per_step": 8 * (M.nnz + M.n * NRHS), "d2h_bytes_per_step": 8 * M.n * NRHS},
        "roofline": roofline,
    }
    if cpu is not None:
        line["cpu_baseline"] = cpu
    line.update({
        "ms_factor": ms_factor, "ms_solve": ms_step - ms_factor, "ms_factor_kernels": ms_factor_kernels,
        "ms_solve_kernels": ms_solve_kernels, "analyze_s": analyze_s,
        "backward_error": berr, "backward_error_e2e": berr_e2e, "factor_vs_oracle": factor_vs_oracle,
        "workload_stats": {"nnz_l": info.nnz_l, "factor_flops": info.flops, "update_flops": info.update_flops,
                           "exec_flops": info.exec_flops, "supernodes": info.nsuper, "levels": info.nlevels},
        "value_definition": "factor flops (sum c_j^2) / (factor + solve) time per step",
        "variants_note": "ms per step of each variant (definitions in bench.py); per-kernel times on stderr",
        "variants": sig4(variants),
    })
    if rank == 0:
        detail_dir = os.environ.get("SYM_BENCH_DETAIL_DIR", tempfile.gettempdir())
        os.makedirs(detail_dir, exist_ok=True)
        with open(os.path.join(detail_dir, "bench_detail.json"), "w") as f:
            json.dump(detail, f, indent=1)
        print(json.dumps({"per_kernel_ms": {k: round(v["ms_per_step"], 3) for k, v in kinds.items()}}),
              file=sys.stderr, flush=True)
        print(json.dumps(line), flush=True)
    s.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=WORKLOAD,
                    help="the benchmark workload is the default; the others are smaller cases")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="skip the mixed-precision and batched variants")
    ap.add_argument("--batch", type=int, default=512, help="matrices of the batched variant (0: skip)")
    ap.add_argument("--cpu-flops", type=float, default=1.0e10,
                    help="flops of the leading block the oracle baseline factors")
    ap.add_argument("--ref-flops", type=float, default=2.0e9,
                    help="flops of the leading block per step of --impl reference")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
