"""CPU check of the host scheduler: the exported launch schedule is executed by a numpy emulator
of the kernels with the semantics of one GPU launch (every task of a launch sees the state from
before the launch; writes land afterwards) and with a conflict check (within one launch no two
tasks write the same element and no task reads an element another task writes). The emulated
factor and solve must reproduce the oracle. A schedule with a missing dependency or a race
fails here without a GPU."""
import numpy as np
import pytest

import oracle
import paper_1705_06575_gb300 as S
import workloads as w

NB = 64
BG = 16
CW = 512  # columns per forward push chunk
K_UPDATE, K_POTRF, K_TRSM, K_GEMM, K_TRTRI = 1, 2, 3, 4, 5
PANEL_NONE, PANEL_FUSED, PANEL_COVERED = 0, 1, 2
S_FGATHER, S_FSTEP, S_FPUSH, S_BGATHER, S_BSTEP, S_FSUM = 11, 12, 13, 14, 15, 16


class Sched:
    def __init__(self, s):
        self.sup = s.export("super")
        self.rowptr = s.export("rowptr")
        self.rows = s.export("rows")
        self.rel = s.export("rel")
        self.tasks = s.export("tasks").reshape(-1, 4)
        ut = s.export("upd_tasks").reshape(-1, 4)
        self.ut = np.stack([ut[:, 0] & 0xffffffff, ut[:, 0] >> 32, ut[:, 1], ut[:, 2], ut[:, 3]], 1)
        ue = s.export("upd_entries").reshape(-1, 5)
        self.ue = np.stack([ue[:, 0] & 0xffffffff, ue[:, 0] >> 32, ue[:, 1] & 0xffffffff, ue[:, 1] >> 32,
                            ue[:, 2], ue[:, 3], ue[:, 4]], 1)
        self.panel = s.export("batch_panel").reshape(-1, 4)  # {role, pmax, ncmax, head} per factor launch
        self.spanel = {"fwd_launches": s.export("fwd_panel").reshape(-1, 4),
                       "bwd_launches": s.export("bwd_panel").reshape(-1, 4)}
        self.cptr = s.export("contrib_ptr")
        self.contrib = s.export("contrib")
        # offset of each supernode's pushed products: its rows below the diagonal block, once per
        # column chunk, in supernode order
        nc = np.diff(self.sup).astype(np.int64)
        off = np.diff(self.rowptr).astype(np.int64) - nc
        self.tx = np.concatenate([[0], np.cumsum(off * ((nc + CW - 1) // CW))])
        self.launches = {}
        self.tb = {}
        for k in ("factor_launches", "fwd_launches", "bwd_launches"):
            raw = s.export(k).reshape(-1, 5)
            self.launches[k] = np.stack([raw[:, 0] & 0xffffffff, raw[:, 1], raw[:, 2], raw[:, 3] >> 32,
                                         (raw[:, 4] & 0xffffffff).astype(np.uint32).astype(np.int32)], 1)
            self.tb[k] = raw[:, 4] >> 32  # 32: small-tile kernel variant
            self.cluster = getattr(self, "cluster", {})
            self.cluster[k] = raw[:, 3] & 0xffffffff  # 4 on the solve: cluster-form step tasks

    def J(self, j):
        f, l = int(self.sup[j]), int(self.sup[j + 1])
        nr = int(self.rowptr[j + 1] - self.rowptr[j])
        return f, l - f, nr, (l - f + NB - 1) // NB

    def row_base(self, j, i):
        _, nc, nr, ncb = self.J(j)
        return i * NB if i < ncb else nc + (i - ncb) * NB

    def row_len(self, j, i):
        _, nc, nr, ncb = self.J(j)
        end = nc if i < ncb else nr
        return min(NB, end - self.row_base(j, i))

    def tile(self, j, i, c):
        """(row slice, col slice) of tile (i, c) of supernode j's panel."""
        rb = self.row_base(j, i)
        _, nc, _, _ = self.J(j)
        return slice(rb, rb + self.row_len(j, i)), slice(c * NB, min(nc, (c + 1) * NB))


def concurrent_pairs(L):
    """Pairs (i, j), i < j, of launches that may overlap: j is not ordered after i by stream
    order (launches of one stream run in list order) or by a chain of waits."""
    n = len(L)
    after = [set() for _ in range(n)]  # launches that finish before launch j starts
    last = {}
    for j in range(n):
        stream, wait = int(L[j][3]), int(L[j][4])
        preds = []
        if stream in last:
            preds.append(last[stream])
        if wait >= 0:
            preds.append(wait)
        for p in preds:
            after[j] |= after[p] | {p}
        last[stream] = j
    return [(i, j) for j in range(n) for i in range(j) if i not in after[j]]


def half_rows(tile, half):
    """Rows of a tile restricted to its first (half 1) or second (half 2) 32 rows."""
    rs, cs = tile
    if half:
        lo = rs.start + (half - 1) * (NB // 2)
        rs = slice(lo, max(lo, min(rs.stop, lo + NB // 2)))
    return rs, cs


class Launch:
    """Collects the effects of the tasks of one launch, then applies them; conflict checks."""

    def __init__(self):
        self.writes = {}  # key -> (task id, value)
        self.reads = []   # (task id, key)

    def read(self, t, key):
        self.reads.append((t, key))

    def write(self, t, key, value):
        assert key not in self.writes or self.writes[key][0] == t, ("two tasks write", key)
        self.writes[key] = (t, value)

    def commit(self, store):
        for t, key in self.reads:
            if key in self.writes:
                assert self.writes[key][0] == t, ("read of an element another task writes", key)
        for key, (_, v) in self.writes.items():
            store[key] = v


def emulate_factor(sc, panels, store, batch=False):
    """store maps ('L', j, r, c) and ('I', j, s, r, c) to values. batch: the launches as a batch
    runs them (a fused narrow level's POTRF launch factors, solves and inverts whole panels; its
    TRSM and TRTRI launches do nothing)."""
    def get(j, r, c):
        return store[("L", j, r, c)]

    record = []
    for li, ((kind, off, count, _, _), tb) in enumerate(zip(sc.launches["factor_launches"], sc.tb["factor_launches"])):
        kind = int(kind)
        L = Launch()
        record.append(L)
        role = int(sc.panel[li, 0]) if batch else 0
        if role == PANEL_COVERED:
            L.commit(store)
            continue
        for t in range(int(off), int(off + count)):
            if role == PANEL_FUSED:
                j = int(sc.tasks[t][0])
                f, nc, nr, ncb = sc.J(j)
                assert ncb == 1 and nc <= 32 and nr * nc <= sc.panel[li, 1] and nc <= sc.panel[li, 2]
                Pn = np.array([[get(j, r, c) for c in range(nc)] for r in range(nr)])
                for r in range(nr):
                    for c in range(nc):
                        L.read(t, ("L", j, r, c))
                Lc = np.linalg.cholesky(np.tril(Pn[:nc]) + np.tril(Pn[:nc], -1).T)
                X = np.linalg.solve(Lc, Pn[nc:].T).T
                full = np.vstack([Lc, X])
                for r in range(nr):
                    for c in range(nc):
                        L.write(t, ("L", j, r, c), full[r, c])
                Inv = np.linalg.inv(Lc)
                for a in range(nc):
                    for b in range(nc):
                        L.write(t, ("I", j, 0, a, b), Inv[a, b])
            elif kind == K_UPDATE:
                j, bi, bj, e0, e1 = (int(v) for v in sc.ut[t])
                rs, cs = sc.tile(j, bi, bj)
                rb, cb = rs.start, cs.start
                acc = {}
                for r in range(rs.start, rs.stop):
                    for c in range(cs.start, cs.stop):
                        acc[(r, c)] = get(j, r, c)
                        L.read(t, ("L", j, r, c))
                for e in range(e0, e1):
                    K, r_lo, c_lo, m, n, relr, relc = (int(v) for v in sc.ue[e])
                    _, kc, _, _ = sc.J(K)
                    A = np.array([[get(K, r_lo + a, k) for k in range(kc)] for a in range(m)])
                    B = np.array([[get(K, c_lo + b, k) for k in range(kc)] for b in range(n)])
                    for a in range(m):
                        for k in range(kc):
                            L.read(t, ("L", K, r_lo + a, k))
                    for b in range(n):
                        for k in range(kc):
                            L.read(t, ("L", K, c_lo + b, k))
                    P = A @ B.T if A.size else np.zeros((0, B.shape[0]))
                    for a in range(m):
                        for b in range(n):
                            key = (rb + int(sc.rel[relr + a]) - rb, cb + int(sc.rel[relc + b]) - cb)
                            acc[key] -= P[a, b]
                for (r, c), v in acc.items():
                    L.write(t, ("L", j, r, c), v)
            elif kind in (K_POTRF, K_TRSM, K_GEMM, K_TRTRI):
                j, ti, tj, ts_ = (int(v) for v in sc.tasks[t])
                f, nc, nr, ncb = sc.J(j)
                if kind == K_POTRF:
                    rs, cs = sc.tile(j, ti, ti)
                    D = np.array([[get(j, r, c) if r - rs.start >= c - cs.start else 0.0 for c in range(cs.start, cs.stop)]
                                  for r in range(rs.start, rs.stop)])
                    for r in range(rs.start, rs.stop):
                        for c in range(cs.start, cs.stop):
                            L.read(t, ("L", j, r, c))
                    Lc = np.linalg.cholesky(D)
                    for a, r in enumerate(range(rs.start, rs.stop)):
                        for b, c in enumerate(range(cs.start, cs.stop)):
                            L.write(t, ("L", j, r, c), Lc[a, b] if a >= b else 0.0)
                elif kind == K_TRSM:
                    i, s = ti, tj
                    drs, dcs = sc.tile(j, s, s)
                    rs, cs = half_rows(sc.tile(j, i, s), ts_ >> 16)
                    D = np.array([[get(j, r, c) for c in range(dcs.start, dcs.stop)] for r in range(drs.start, drs.stop)])
                    X = np.array([[get(j, r, c) for c in range(cs.start, cs.stop)] for r in range(rs.start, rs.stop)])
                    for r in range(drs.start, drs.stop):
                        for c in range(dcs.start, dcs.stop):
                            if r - drs.start >= c - dcs.start:
                                L.read(t, ("L", j, r, c))
                    if X.size:
                        X = np.linalg.solve(np.tril(D), X.T).T
                    for a, r in enumerate(range(rs.start, rs.stop)):
                        for b, c in enumerate(range(cs.start, cs.stop)):
                            L.write(t, ("L", j, r, c), X[a, b])
                elif kind == K_GEMM:
                    i, jj, s = ti, tj, ts_ & 0xffff
                    rs, cs = half_rows(sc.tile(j, i, jj), ts_ >> 16)
                    ars, acs = half_rows(sc.tile(j, i, s), ts_ >> 16)
                    brs, _ = sc.tile(j, jj, s)
                    A = np.array([[get(j, r, c) for c in range(acs.start, acs.stop)] for r in range(ars.start, ars.stop)])
                    B = np.array([[get(j, r, c) for c in range(acs.start, acs.stop)] for r in range(brs.start, brs.stop)])
                    for r in list(range(ars.start, ars.stop)) + list(range(brs.start, brs.stop)):
                        for c in range(acs.start, acs.stop):
                            L.read(t, ("L", j, r, c))
                    P = A @ B.T if A.size else np.zeros((0, B.shape[0]))
                    for a, r in enumerate(range(rs.start, rs.stop)):
                        for b, c in enumerate(range(cs.start, cs.stop)):
                            L.write(t, ("L", j, r, c), get(j, r, c) - P[a, b])
                else:  # K_TRTRI
                    s = ti
                    rs, cs = sc.tile(j, s, s)
                    D = np.array([[get(j, r, c) for c in range(cs.start, cs.stop)] for r in range(rs.start, rs.stop)])
                    Inv = np.linalg.inv(np.tril(D))
                    for a in range(Inv.shape[0]):
                        for b in range(Inv.shape[1]):
                            L.write(t, ("I", j, s, a, b), Inv[a, b])
            else:
                raise AssertionError(f"unknown kind {kind}")
        L.commit(store)
    # launches that may run at the same time (two streams) must not touch each other's elements
    for i, j in concurrent_pairs(sc.launches["factor_launches"]):
        wi, wj = set(record[i].writes), set(record[j].writes)
        ri = {k for _, k in record[i].reads}
        rj = {k for _, k in record[j].reads}
        assert not (wi & (wj | rj)) and not (ri & wj), ("concurrent launches conflict", i, j)


def emulate_solve(sc, store, y, batch=False):
    """y: dict index -> value (permuted numbering), updated in place. batch: the launches as a
    batch runs them (a fused narrow level's step launch does the level's sums, steps and pushes
    or gathers and steps; its other launches do nothing)."""
    def Lv(j, r, c):
        return store[("L", j, r, c)]

    def Iv(j, s, a, b):
        return store[("I", j, s, a, b)]

    for name in ("fwd_launches", "bwd_launches"):
        for li, (kind, off, count, _, _) in enumerate(sc.launches[name]):
            kind = int(kind)
            cluster_form = int(sc.cluster[name][li]) == 4
            role = int(sc.spanel[name][li, 0]) if batch else PANEL_NONE
            L = Launch()
            if role == PANEL_COVERED:
                L.commit(y)
                continue
            for t in range(int(off), int(off + count)):
                j, ti, tc, _ = (int(v) for v in sc.tasks[t])
                f, nc, nr, ncb = sc.J(j)
                R = sc.rows[sc.rowptr[j]:sc.rowptr[j + 1]]
                tsz = lambda s: min(NB, nc - s * NB)
                if role == PANEL_FUSED:
                    assert ncb == 1 and nc <= 32 and nr * nc <= sc.spanel[name][li, 1]
                    Inv = np.array([[Iv(j, 0, a, b) for b in range(nc)] for a in range(nc)])
                    if kind == S_FSTEP:
                        v = []
                        for c in range(nc):
                            keys = [("t", int(e)) for e in sc.contrib[sc.cptr[f + c]:sc.cptr[f + c + 1]]]
                            for k in keys + [f + c]:
                                L.read(t, k)
                            v.append(y[f + c] - sum(y[k] for k in keys))
                        z = Inv @ np.array(v)
                        for c in range(nc):
                            L.write(t, f + c, z[c])
                        for r in range(nc, nr):
                            L.write(t, ("t", int(sc.tx[j]) + (r - nc)), sum(Lv(j, r, c) * z[c] for c in range(nc)))
                    else:
                        assert kind == S_BSTEP
                        v = []
                        for c in range(nc):
                            for r in range(nc, nr):
                                L.read(t, int(R[r]))
                            L.read(t, f + c)
                            v.append(y[f + c] - sum(Lv(j, r, c) * y[int(R[r])] for r in range(nc, nr)))
                        z = Inv.T @ np.array(v)
                        for c in range(nc):
                            L.write(t, f + c, z[c])
                elif kind == S_FGATHER:
                    bj, ut = ti, tc
                    cb = bj * NB
                    acc = {f + cb + r: y[f + cb + r] for r in range(min(NB, nc - cb))}
                    for key in acc:
                        L.read(t, key)
                    _, _, _, e0, e1 = (int(v) for v in sc.ut[ut])
                    for e in range(e0, e1):
                        K, r_lo, c_lo, m, n, relr, relc = (int(v) for v in sc.ue[e])
                        fk, kc, _, _ = sc.J(K)
                        for b in range(n):
                            v = sum(Lv(K, c_lo + b, k) * y[fk + k] for k in range(kc))
                            for k in range(kc):
                                L.read(t, fk + k)
                            acc[f + int(sc.rel[relc + b])] -= v
                    for key, v in acc.items():
                        L.write(t, key, v)
                elif kind == S_FPUSH:
                    i, ch = ti, tc
                    rs, _ = sc.tile(j, i, 0)
                    cols = range(ch * CW, min(nc, (ch + 1) * CW))
                    for c in cols:
                        L.read(t, f + c)
                    for r in range(rs.start, rs.stop):
                        v = sum(Lv(j, r, c) * y[f + c] for c in cols)
                        L.write(t, ("t", int(sc.tx[j]) + ch * (nr - nc) + (r - nc)), v)
                elif kind == S_FSUM:
                    cb = ti
                    for c in range(cb * 256, min(nc, (cb + 1) * 256)):
                        g = f + c
                        keys = [("t", int(e)) for e in sc.contrib[sc.cptr[g]:sc.cptr[g + 1]]]
                        for k in keys:
                            L.read(t, k)
                        L.read(t, g)
                        L.write(t, g, y[g] - sum(y[k] for k in keys))
                elif kind == S_BGATHER:
                    c0 = ti * BG
                    for c in range(c0, min(nc, c0 + BG)):
                        v = sum(Lv(j, r, c) * y[int(R[r])] for r in range(nc, nr))
                        for r in range(nc, nr):
                            L.read(t, int(R[r]))
                        L.read(t, f + c)
                        L.write(t, f + c, y[f + c] - v)
                elif kind in (S_FSTEP, S_BSTEP) and cluster_form:
                    # cluster task {J, i, s}: apply the solved tile s (if any) to tile i; the task
                    # next to s (i = s + 1 forward, s - 1 backward) then solves tile i in place
                    i, s = ti, tc
                    fwd = kind == S_FSTEP
                    has_s = s >= 0 if fwd else s < ncb
                    gi = [f + i * NB + a for a in range(tsz(i))]
                    v = np.array([y[k] for k in gi])
                    for k in gi:
                        L.read(t, k)
                    if has_s:
                        gs = [f + s * NB + b for b in range(tsz(s))]
                        zs = np.array([y[k] for k in gs])
                        for k in gs:
                            L.read(t, k)
                        for a in range(tsz(i)):
                            if fwd:
                                v[a] -= sum(Lv(j, i * NB + a, s * NB + b) * zs[b] for b in range(tsz(s)))
                            else:
                                v[a] -= sum(Lv(j, s * NB + b, i * NB + a) * zs[b] for b in range(tsz(s)))
                    if i == (s + 1 if fwd else s - 1):
                        Inv = np.array([[Iv(j, i, a, b) for b in range(tsz(i))] for a in range(tsz(i))])
                        v = Inv @ v if fwd else Inv.T @ v
                    for k, val in zip(gi, v):
                        L.write(t, k, val)
                elif kind in (S_FSTEP, S_BSTEP):
                    i, s = ti, tc
                    fwd = kind == S_FSTEP

                    def solved(u):
                        g = [f + u * NB + a for a in range(tsz(u))]
                        v = np.array([y[k] for k in g])
                        Inv = np.array([[Iv(j, u, a, b) for b in range(tsz(u))] for a in range(tsz(u))])
                        return g, (Inv @ v if fwd else Inv.T @ v)

                    if i == s:
                        targets = ([s - 1] if s >= 1 else []) + ([s] if s == ncb - 1 else []) if fwd else \
                                  ([s + 1] if s + 1 < ncb else []) + ([0] if s == 0 else [])
                        for u in targets:
                            g, v = solved(u)
                            for k, val in zip(g, v):
                                L.read(t, k)
                                L.write(t, k, val)
                    else:
                        g, zs = solved(s)
                        for k in g:
                            L.read(t, k)
                        for a in range(tsz(i)):
                            k = f + i * NB + a
                            if fwd:
                                v = sum(Lv(j, i * NB + a, s * NB + b) * zs[b] for b in range(tsz(s)))
                            else:
                                v = sum(Lv(j, s * NB + b, i * NB + a) * zs[b] for b in range(tsz(s)))
                            L.read(t, k)
                            L.write(t, k, y[k] - v)
                else:
                    raise AssertionError(f"unknown kind {kind}")
            L.commit(y)


@pytest.mark.parametrize("maker", [
    lambda: w.laplace2d5(14, np.random.default_rng(1)),
    lambda: w.conduct3d(6, np.random.default_rng(2), "box"),
    lambda: w.random_spd_pattern(150, 1.0, np.random.default_rng(3)),      # one wide supernode: 3 tiles
    lambda: w.random_spd_pattern(220, 0.03, np.random.default_rng(4)),
    lambda: w.wide_block(520, 40, np.random.default_rng(5)),                # two push chunks
])
@pytest.mark.parametrize("batch", [False, True])
def test_schedule_emulation_reproduces_oracle(maker, batch):
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sc = Sched(s)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax) == 0
    # H1: the panels hold the lower part of C = P A P^T, zeros elsewhere
    store = {}
    Cval = {}
    for jcol in range(M.n):
        for p in range(o.Cp[jcol], o.Cp[jcol + 1]):
            Cval[(int(o.Ci[p]), jcol)] = M.Ax[o.Cmap[p]]
    for j in range(len(sc.sup) - 1):
        f, nc, nr, _ = sc.J(j)
        R = sc.rows[sc.rowptr[j]:sc.rowptr[j + 1]]
        for r in range(nr):
            for c in range(nc):
                store[("L", j, r, c)] = Cval.get((int(R[r]), f + c), 0.0) if R[r] >= f + c else 0.0
    emulate_factor(sc, None, store, batch)
    # compare with the oracle on its pattern
    for j in range(len(sc.sup) - 1):
        f, nc, nr, _ = sc.J(j)
        R = list(sc.rows[sc.rowptr[j]:sc.rowptr[j + 1]])
        for c in range(nc):
            col = f + c
            for p in range(o.Lp[col], o.Lp[col + 1]):
                r = R.index(int(o.Li[p]))
                assert abs(store[("L", j, r, c)] - o.Lx[p]) <= 1e-12 * np.abs(o.Lx).max()
    # solve with one right-hand side in the permuted space
    b = np.random.default_rng(9).standard_normal(M.n)
    y = {k: b[o.perm[k]] for k in range(M.n)}
    emulate_solve(sc, store, y, batch)
    x = np.zeros(M.n)
    for k in range(M.n):
        x[o.perm[k]] = y[k]
    ref = o.solve(b)[:, 0]
    assert np.abs(x - ref).max() <= 1e-10 * np.abs(ref).max()


def test_emulator_detects_a_missing_launch():
    """Planted mistake: dropping one trailing-update launch from the schedule is detected."""
    M = w.random_spd_pattern(150, 1.0, np.random.default_rng(3))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sc = Sched(s)
    kinds = [int(x) for x in sc.launches["factor_launches"][:, 0]]
    sc.launches["factor_launches"] = np.delete(sc.launches["factor_launches"], kinds.index(K_GEMM), axis=0)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    o.factor(M.Ax)
    store = {}
    Cval = {(int(o.Ci[p]), jc): M.Ax[o.Cmap[p]] for jc in range(M.n) for p in range(o.Cp[jc], o.Cp[jc + 1])}
    f, nc, nr, _ = sc.J(0)
    R = sc.rows[sc.rowptr[0]:sc.rowptr[1]]
    for r in range(nr):
        for c in range(nc):
            store[("L", 0, r, c)] = Cval.get((int(R[r]), f + c), 0.0) if R[r] >= f + c else 0.0
    try:
        emulate_factor(sc, None, store)
        err = max(abs(store[("L", 0, int(np.nonzero(R == o.Li[p])[0][0]), c)] - o.Lx[p])
                  for c in range(nc) for p in range(o.Lp[c], o.Lp[c + 1]))
    except np.linalg.LinAlgError:
        err = np.inf
    assert err > 1e-3


def test_conflict_checker():
    L = Launch()
    L.write(0, ("L", 0, 1, 1), 1.0)
    with pytest.raises(AssertionError):
        L.write(1, ("L", 0, 1, 1), 2.0)  # two tasks write one element
    L2 = Launch()
    L2.read(0, 5)
    L2.write(1, 5, 3.0)
    with pytest.raises(AssertionError):
        L2.commit({})  # a task reads what another task of the launch writes



def test_lookahead_streams_are_used_and_ordered():
    """Wide supernodes get a second stream: some trailing updates run concurrently with the
    next panel's factorization, and every auxiliary launch waits for the panel it reads."""
    M = w.random_spd_pattern(300, 1.0, np.random.default_rng(8))  # one supernode, 5 column tiles
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    L = Sched(s).launches["factor_launches"]
    aux = [i for i in range(len(L)) if L[i][3] == 1]
    assert aux, "no lookahead launch"
    assert all(L[i][4] >= 0 for i in aux)
    pairs = concurrent_pairs(L)
    assert any(int(L[i][0]) == K_POTRF or int(L[j][0]) == K_POTRF for i, j in pairs)


def test_level_summary_of_the_profiling_driver():
    """The profiling driver's two-stream bound follows the schedule's streams and waits: with
    every launch taking 1 ms it equals the longest chain of dependent launches, at most the
    serialised total, and each level's kinds add up to the schedule."""
    from paper_1705_06575_gb300.profile_factor import level_summary
    M = w.conduct3d(16, np.random.default_rng(5), "star")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    raw = s.export("factor_launches").reshape(-1, 5)
    out = level_summary(s, np.ones(len(raw) + 1))
    assert out["serialised_ms"] == len(raw)
    assert out["two_stream_bound_ms"] <= out["serialised_ms"]
    assert sum(v["launches"] for r in out["levels"] for k, v in r.items() if isinstance(v, dict)) == len(raw)
    stream = raw[:, 3] >> 32
    if (stream == 1).any():
        assert out["two_stream_bound_ms"] < out["serialised_ms"]


@pytest.mark.parametrize("maker", [
    lambda: w.dd2d9(128, np.random.default_rng(2000)),                       # the batched pattern
    lambda: w.laplace2d5(64, np.random.default_rng(0)),                      # the latency case
    lambda: w.conduct3d(16, np.random.default_rng(6), "star"),
    lambda: w.random_spd_pattern(300, 0.02, np.random.default_rng(7)),
])
def test_small_tile_launches_fit_their_kernels(maker):
    """Launches marked for the small-tile kernels (tb = 32) hold only what those kernels handle:
    diagonal tiles of order <= 32 for POTRF and TRTRI (one-warp forms keep a packed triangle of
    order 32), TRSM tiles of <= 32 columns and <= 64 rows, update tiles of <= 32 rows and columns;
    no trailing-GEMM launch is marked. Unmarked update tiles and TRSM row tiles stay within one
    64 x 64 tile, and every update entry within the rows and columns of its tile (the tensor-core
    update expands entries to tile positions 0..63)."""
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sc = Sched(s)
    small_seen = 0
    for (kind, off, count, _, _), tb in zip(sc.launches["factor_launches"], sc.tb["factor_launches"]):
        kind, off, count, tb = int(kind), int(off), int(count), int(tb)
        assert tb in (0, 32)
        if tb == 32:
            small_seen += 1
            assert kind != K_GEMM
        for t in range(off, off + count):
            if kind == K_UPDATE:
                j, bi, bj, e0, e1 = (int(v) for v in sc.ut[t])
                rs, cs = sc.tile(j, bi, bj)
                tm, tn = rs.stop - rs.start, cs.stop - cs.start
                assert 0 < tm <= NB and 0 < tn <= NB
                if tb == 32:
                    assert tm <= 32 and tn <= 32
                for e in range(e0, e1):
                    K, r_lo, c_lo, m, n, relr, relc = (int(v) for v in sc.ue[e])
                    assert 0 < m <= tm and 0 < n <= tn
                    pr = sc.rel[relr:relr + m] - sc.row_base(j, bi)
                    pc = sc.rel[relc:relc + n] - bj * NB
                    assert pr.min() >= 0 and pr.max() < tm and len(set(pr.tolist())) == m
                    assert pc.min() >= 0 and pc.max() < tn and len(set(pc.tolist())) == n
            elif kind in (K_POTRF, K_TRTRI, K_TRSM):
                j, ti, tj, d = (int(v) for v in sc.tasks[t])
                _, nc, _, _ = sc.J(j)
                s_ = tj if kind == K_TRSM else ti
                ts = min(NB, nc - s_ * NB)
                assert 0 < ts <= NB
                if kind == K_TRSM:
                    tm = sc.row_len(j, ti)
                    assert 0 < tm <= NB and (d >> 16) in (0, 1, 2)
                if tb == 32:
                    assert ts <= 32
    if M.n >= 4096:
        assert small_seen > 0  # the grids exercise the small-tile forms


@pytest.mark.parametrize("maker", [
    lambda: w.dd2d9(128, np.random.default_rng(2000)),                       # the batched pattern
    lambda: w.conduct3d(16, np.random.default_rng(6), "star"),
    lambda: w.random_spd_pattern(300, 0.02, np.random.default_rng(7)),
])
def test_small_solve_launches_fit_the_warp_forms(maker):
    """Solve launches marked tb = 32 (run one warp per task and matrix in batches) hold only
    supernodes of at most 32 columns: a sum task covers all of its supernode's columns with one
    lane per column, a push task one row tile (<= 64 rows) and one column chunk, a gather task
    one slice, and a step task is the whole one-tile diagonal block, {J, 0, 0, 0}. A level with a
    wider supernode marks none of its sum, push and gather launches."""
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sc = Sched(s)
    level = s.export("level")
    seen = 0
    for key in ("fwd_launches", "bwd_launches"):
        for (kind, off, count, _, _), tb in zip(sc.launches[key], sc.tb[key]):
            kind, off, count, tb = int(kind), int(off), int(count), int(tb)
            js = [int(sc.tasks[t][0]) for t in range(off, off + count)]
            if kind in (S_FSUM, S_FPUSH, S_BGATHER):
                lv = {int(level[j]) for j in js}
                assert len(lv) == 1
                wide = [j for j in np.where(level == lv.pop())[0] if sc.J(j)[1] > 32]
                assert tb == (0 if wide else 32)
            if tb != 32:
                continue
            seen += 1
            for t in range(off, off + count):
                j, a, b, c = (int(v) for v in sc.tasks[t])
                _, nc, nr, ncb = sc.J(j)
                assert nc <= 32 and ncb == 1
                if kind in (S_FSTEP, S_BSTEP):
                    assert (a, b, c) == (0, 0, 0)
                elif kind == S_FSUM:
                    assert a == 0
                elif kind == S_FPUSH:
                    assert a >= ncb and b == 0 and 0 < sc.row_len(j, a) <= NB
                elif kind == S_BGATHER:
                    assert a * BG < nc and nr > nc
    assert seen > 0


@pytest.mark.parametrize("maker", [
    lambda: w.conduct3d(16, np.random.default_rng(6), "star"),
    lambda: w.random_spd_pattern(300, 0.02, np.random.default_rng(7)),
    lambda: w.dd2d9(128, np.random.default_rng(2000)),
])
def test_step_launches_have_a_kernel_form(maker):
    """Every column-tile step of the plan's solve is either a cluster step (supernodes wider than
    32 columns) or a one-tile step of the small form: the executor launches no other step form."""
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sc = Sched(s)
    for key in ("fwd_launches", "bwd_launches"):
        for (kind, off, count, _, _), tb, cl in zip(sc.launches[key], sc.tb[key], sc.cluster[key]):
            if int(kind) in (S_FSTEP, S_BSTEP):
                assert int(cl) == 4 or int(tb) == 32


@pytest.mark.parametrize("maker", [
    lambda: w.dd2d9(128, np.random.default_rng(2000)),                       # the batched pattern
    lambda: w.laplace2d5(30, np.random.default_rng(1)),
    lambda: w.conduct3d(10, np.random.default_rng(3), "star"),
])
def test_batch_panel_marks(maker):
    """Every level whose supernodes all have at most 32 columns has its POTRF launch marked fused
    (with the level's largest panel and widest supernode) and its TRSM and TRTRI launches marked
    covered; nothing else is marked."""
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sc = Sched(s)
    level = s.export("level")
    nc = np.diff(sc.sup)
    nr = np.diff(sc.rowptr)
    raw = s.export("factor_launches").reshape(-1, 5)
    lkind, llev = raw[:, 0] & 0xffffffff, raw[:, 0] >> 32
    fused_levels = set()
    for lv in range(int(level.max()) + 1):
        sel = level == lv
        pmax, ncmax = int((nc * nr)[sel].max()), int(nc[sel].max())
        eligible = ncmax <= 32 and int(((llev == lv) & (lkind == K_POTRF)).sum()) == 1
        head = [li for li in np.nonzero(llev == lv)[0] if lkind[li] == K_POTRF]
        for li in np.nonzero(llev == lv)[0]:
            role, pm, nm, hd = (int(v) for v in sc.panel[li])
            if not eligible:
                assert role == PANEL_NONE
            elif lkind[li] == K_POTRF:
                assert (role, pm, nm, hd) == (PANEL_FUSED, pmax, ncmax, li)
            elif lkind[li] in (K_TRSM, K_TRTRI):
                assert (role, hd) == (PANEL_COVERED, head[0])
            else:
                assert role == PANEL_NONE
        if eligible:
            fused_levels.add(lv)
    assert fused_levels  # every pattern here has narrow levels at its leaves


@pytest.mark.parametrize("maker", [
    lambda: w.dd2d9(128, np.random.default_rng(2000)),                       # the batched pattern
    lambda: w.laplace2d5(30, np.random.default_rng(1)),
    lambda: w.conduct3d(10, np.random.default_rng(3), "star"),
])
def test_solve_panel_marks(maker):
    """In both solve lists, every level whose supernodes all have at most 32 columns has its step
    launch marked fused (with the level's largest panel and widest supernode) and its other
    launches marked covered."""
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sc = Sched(s)
    level = s.export("level")
    nc = np.diff(sc.sup)
    nr = np.diff(sc.rowptr)

    nfused = 0
    for name, step in (("fwd_launches", S_FSTEP), ("bwd_launches", S_BSTEP)):
        raw = s.export(name).reshape(-1, 5)
        kind, lev = raw[:, 0] & 0xffffffff, raw[:, 0] >> 32
        for lv in range(int(level.max()) + 1):
            sel = level == lv
            pmax, ncmax = int((nc * nr)[sel].max()), int(nc[sel].max())
            steps = [li for li in np.nonzero(lev == lv)[0] if kind[li] == step]
            eligible = ncmax <= 32 and len(steps) == 1
            for li in np.nonzero(lev == lv)[0]:
                role, pm, nm, hd = (int(v) for v in sc.spanel[name][li])
                if not eligible:
                    assert role == PANEL_NONE
                elif li == steps[0]:
                    assert (role, pm, nm, hd) == (PANEL_FUSED, pmax, ncmax, li)
                    nfused += 1
                else:
                    assert (role, hd) == (PANEL_COVERED, steps[0])
    assert nfused >= 2


def test_launch_counts_skip_fused_levels():
    """sym_info's kernel counts leave out the launches that a fused narrow level covers: every
    covered solve launch for one right-hand side (the panels of this grid fit the one-warp form),
    and none of the factor's on levels of fewer than 1216 supernodes; with the fused levels off,
    the whole schedule (+ zeroing and scatter, + the two permutations)."""
    M = w.laplace2d5(30, np.random.default_rng(1))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    off = S.Solver(M.n, M.Ap, M.Ai, M.perm, flags=S.SYM_FLAG_HOST_ONLY | S.SYM_FLAG_NO_FUSED_LEVELS)
    nf = len(s.export("factor_launches")) // 5
    nfwd, nbwd = len(s.export("fwd_launches")) // 5, len(s.export("bwd_launches")) // 5
    covered = int((s.export("fwd_panel").reshape(-1, 4)[:, 0] == 2).sum() +
                  (s.export("bwd_panel").reshape(-1, 4)[:, 0] == 2).sum())
    assert covered > 0
    assert (off.info().nlaunch_factor, off.info().nlaunch_solve) == (nf + 2, nfwd + nbwd + 2)
    assert s.info().nlaunch_factor == nf + 2  # (no level of this grid has 1216 supernodes)
    assert s.info().nlaunch_solve == nfwd + nbwd + 2 - covered
