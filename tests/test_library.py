"""CPU tests of the C-ABI library: it builds, loads, exports every declared entry point, and its
host symbolic inspector is bit-exact against the independent oracle. No GPU compute here: the
handles are analyzed with SYM_FLAG_HOST_ONLY."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_1705_06575_gb300 as S
import workloads as w

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [("perm", "perm"), ("parent", "parent"), ("colcount", "colcount"), ("fsuper", "fsn"),
         ("super", "sn"), ("rowptr", "srp"), ("rows", "sri"), ("sparent", "sparent"),
         ("descptr", "dp"), ("desc", "dk"), ("descr0", "dr0"), ("descnin", "dnin"),
         ("relptr", "relp"), ("rel", "rel"), ("level", "level"), ("levelptr", "lvp"),
         ("levellist", "lvl")]


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(sym_[a-z_0-9]+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    lib = S.load()
    names = declared_functions()
    assert {"sym_analyze", "sym_factor", "sym_solve"} <= names
    for name in names:
        assert hasattr(lib, name), name


def compare(M, perm=None, relax=oracle.DEFAULT_RELAX):
    opt = S.sym_options_default()
    if relax is None:
        opt.amalgamate = 0
    else:
        opt.nrelax[:] = relax[:3]
        opt.zrelax_permille[:] = relax[3:]
    s = S.Solver(M.n, M.Ap, M.Ai, perm, opt=opt, host_only=True)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, perm, relax=relax, want_rel=True)
    for a, b in PAIRS:
        got = s.export(a)
        ref = getattr(o, b)
        if ref is None:  # no descendant pairs: the oracle keeps no map
            assert got.size <= 1 and not got[1:].any()
            continue
        assert np.array_equal(got, ref), a
    info = s.info()
    assert info.nnz_l == o.nnzL
    assert info.flops == float(o.flops_exact)
    s.close()


@pytest.mark.parametrize("n,density,seed", [(1, 1.0, 0), (2, 1.0, 1), (50, 0.1, 2), (300, 0.02, 3),
                                            (800, 0.005, 4), (200, 1.0, 5), (400, 0.003, 6)])
def test_symbolic_bit_exact_random(n, density, seed):
    rng = np.random.default_rng(seed)
    M = w.random_spd_pattern(n, density, rng)
    compare(M)
    compare(M, perm=rng.permutation(n).astype(np.int32))
    compare(M, relax=None)
    compare(M, relax=(2, 8, 24, 500, 50, 10))


@pytest.mark.parametrize("maker", [
    lambda: w.cfg("laplace2d5_64"),
    lambda: w.dd2d9(40, np.random.default_rng(1)),
    lambda: w.conduct3d(14, np.random.default_rng(2), "star"),
    lambda: w.conduct3d(10, np.random.default_rng(3), "box"),
    lambda: w.vector3d27(6, np.random.default_rng(4), sub=3),
    lambda: w.erdos_renyi(600, 4, np.random.default_rng(5)),
])
def test_symbolic_bit_exact_workloads(maker):
    M = maker()
    compare(M, perm=M.perm)


def test_special_structures():
    n = 40
    Ap = np.arange(n + 1, dtype=np.int64)
    Ai = np.arange(n, dtype=np.int32)
    compare(w.Matrix(n, Ap, Ai, np.ones(n)))  # diagonal
    u = np.arange(n - 1)
    Ap, Ai, Ax = w.lower_csc(n, u, u + 1, -np.ones(n - 1), np.full(n, 3.0))
    compare(w.Matrix(n, Ap, Ai, Ax))  # tridiagonal
    Ap, Ai, Ax = w.lower_csc(n, u, np.full(n - 1, n - 1), -np.ones(n - 1), np.full(n, float(n)))
    compare(w.Matrix(n, Ap, Ai, Ax))  # arrowhead
    Ap, Ai, Ax = w.lower_csc(n, np.zeros(n - 1, int), u + 1, -np.ones(n - 1), np.full(n, float(n)))
    compare(w.Matrix(n, Ap, Ai, Ax))  # arrow pointing the other way: dense fill
    # two disconnected blocks
    Ap, Ai, Ax = w.lower_csc(n, np.r_[u[:10], u[20:30]], np.r_[u[:10] + 1, u[20:30] + 1],
                             -np.ones(20), np.full(n, 3.0))
    compare(w.Matrix(n, Ap, Ai, Ax))


def test_empty_matrix_host_only():
    s = S.Solver(0, np.zeros(1, np.int64), np.zeros(0, np.int32), host_only=True)
    assert s.info().nsuper == 0 and s.info().nnz_l == 0


def test_invalid_inputs_are_rejected():
    n = 3
    Ap = np.array([0, 2, 3, 4])
    with pytest.raises(S.SymError) as e:
        S.Solver(n, Ap, np.array([2, 0, 1, 2]), host_only=True)  # diagonal not first
    assert e.value.code == S.SYM_ERR_INVALID
    with pytest.raises(S.SymError):
        S.Solver(n, np.array([0, 2, 2, 3]), np.array([0, 2, 2]), host_only=True)  # missing diagonal
    with pytest.raises(S.SymError):
        S.Solver(n, Ap, np.array([0, 5, 1, 2]), host_only=True)  # row out of range
    with pytest.raises(S.SymError):
        S.Solver(n, Ap, np.array([0, 2, 1, 2]), perm=np.array([0, 0, 2]), host_only=True)
    opt = S.sym_options_default()
    opt.zrelax_permille[0] = 2000
    with pytest.raises(S.SymError):
        S.Solver(n, Ap, np.array([0, 2, 1, 2]), opt=opt, host_only=True)


def test_host_only_handle_refuses_numeric_calls():
    M = w.laplace2d5(8, np.random.default_rng(0))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    with pytest.raises(S.SymError) as e:
        s.factor_host(M.Ax)
    assert e.value.code == S.SYM_ERR_STATE
    with pytest.raises(S.SymError):
        s.solve_host(np.zeros(M.n))


def test_plan_sizes_cfg2_scale():
    """The 64^3 7-point workload: sizes of the plan (sizing check, not a parity target)."""
    M = w.cfg("conduct3d7_64")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    i = s.info()
    assert i.nnz_l == 156727345
    assert abs(i.flops - 4.15e11) / 4.15e11 < 0.01
    assert i.max_ncols == 6080 and i.nlevels == 20


@pytest.mark.parametrize("maker,nb", [
    (lambda: w.cfg("laplace2d5_64"), 5),
    (lambda: w.conduct3d(12, np.random.default_rng(3), "star"), 20),
    (lambda: w.random_spd_pattern(700, 0.005, np.random.default_rng(4)), 1),
    (lambda: w.random_spd_pattern(300, 0.02, np.random.default_rng(5)), 40),
])
def test_reach_set_bit_exact(maker, nb):
    """The library's reach of a sparse right-hand side (etree paths) equals the oracle's
    depth-first search of the dependence graph of L, as sets of permuted columns."""
    M = maker()
    rng = np.random.default_rng(nb)
    bidx = rng.choice(M.n, size=nb, replace=False).astype(np.int32)
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    r = S.Reach(s.h, bidx)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    iperm = np.empty(M.n, dtype=np.int64)
    iperm[o.perm] = np.arange(M.n)
    ref = np.sort(o.reach(iperm[bidx].astype(np.int32)))
    cols = r.export(0)
    assert np.array_equal(cols, ref)
    assert np.array_equal(r.indices(), o.perm[ref])
    sup = s.export("super")
    held = np.unique(np.searchsorted(sup, cols, side="right") - 1)
    assert np.array_equal(r.export(1), held)
    r.close()


def test_reach_rejects_bad_patterns():
    M = w.laplace2d5(10, np.random.default_rng(0))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    for bad in ([M.n], [-1], [3, 3]):
        with pytest.raises(S.SymError):
            S.Reach(s.h, np.array(bad))


@pytest.mark.parametrize("maker", [
    lambda: w.cfg("laplace2d5_64"),
    lambda: w.conduct3d(16, np.random.default_rng(3), "star"),
    lambda: w.vector3d27(6, np.random.default_rng(4), sub=3),
    lambda: w.random_spd_pattern(300, 0.05, np.random.default_rng(2)),
])
def test_update_entries_against_their_definition(maker):
    """Every update entry of tile (bi, bj) of J lists a contiguous run of descendant K's rows whose
    relative positions fall in the tile's rows (r_lo, m) and columns (c_lo, n), checked against
    the rows and relative maps; on a diagonal tile the two runs coincide (m = n, r_lo = c_lo),
    which the FP64 update kernel relies on to compute the lower triangle only."""
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, host_only=True)
    sup = s.export("super"); rp = s.export("rowptr"); rows = s.export("rows")
    ut = s.export("upd_tasks").reshape(-1, 4)
    ue = s.export("upd_entries").reshape(-1, 5)
    NB = 64
    for J, bi, bj, e0, e1 in zip(ut[:, 0] & 0xffffffff, ut[:, 0] >> 32, ut[:, 1], ut[:, 2], ut[:, 3]):
        f, nc = int(sup[J]), int(sup[J + 1] - sup[J])
        RJ = rows[rp[J]:rp[J + 1]]
        ncb = (nc + NB - 1) // NB
        rb = bi * NB if bi < ncb else nc + (bi - ncb) * NB
        rend = min(rb + NB, nc if bi < ncb else len(RJ))
        tile_rows = set(RJ[rb:rend].tolist())
        tile_cols = set(range(f + bj * NB, f + min(nc, (bj + 1) * NB)))
        for K, r_lo, c_lo, m, n in zip(ue[e0:e1, 0] & 0xffffffff, ue[e0:e1, 0] >> 32, ue[e0:e1, 1] & 0xffffffff,
                                       ue[e0:e1, 1] >> 32, ue[e0:e1, 2]):
            RK = rows[rp[K]:rp[K + 1]]
            assert set(RK[r_lo:r_lo + m].tolist()) == tile_rows & set(RK.tolist())
            assert set(RK[c_lo:c_lo + n].tolist()) == tile_cols & set(RK.tolist())
            if bi == bj:
                assert m == n and r_lo == c_lo


@pytest.mark.parametrize("maker", [lambda r: w.laplace2d5(20, r), lambda r: w.conduct3d(8, r, "box"),
                                   lambda r: w.random_spd_pattern(300, 0.02, r)])
def test_update_flops_split_of_sum_c_squared(maker):
    """sym_stats.update_flops is the share of sum c_j^2 that descendant updates carry: counted
    here entry by entry on the oracle's exact column patterns (column k adds 2 (c_k - t) flops to
    the column of its t-th row when that column lies in another supernode)."""
    M = maker(np.random.default_rng(23))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, flags=S.SYM_FLAG_HOST_ONLY)
    info = s.info()
    sup = s.export("super")
    o = oracle.Oracle(M.n, M.Ap, M.Ai, s.export("perm"))
    col2s = np.repeat(np.arange(sup.size - 1), np.diff(sup))
    total = 0
    for k in range(M.n):
        rows = o.Li[o.Lp[k]:o.Lp[k + 1]]
        c = rows.size
        t = np.arange(1, c)
        ext = col2s[rows[1:]] != col2s[k]
        total += int(np.sum(2 * (c - t)[ext]))
    assert info.update_flops == total
    assert info.update_flops < info.flops == o.flops_exact


def _auto(M):
    return S.Solver(M.n, M.Ap, M.Ai, flags=S.SYM_FLAG_HOST_ONLY, ordering="auto")


@pytest.mark.parametrize("maker", [lambda r: w.laplace2d5(40, r), lambda r: w.conduct3d(14, r, "star"),
                                   lambda r: w.conduct3d(10, r, "box"), lambda r: w.dd2d9(40, r),
                                   lambda r: w.erdos_renyi(1500, 6, r), lambda r: w.random_spd_pattern(400, 0.01, r)])
def test_auto_ordering_symbolic_bit_exact(maker):
    """SYM_ORDER_AUTO yields a permutation; given that permutation, the independent oracle
    reproduces every integer output of the inspector bit for bit."""
    M = maker(np.random.default_rng(71))
    s = _auto(M)
    info = s.info()
    perm = s.export("perm")
    assert np.array_equal(np.sort(perm), np.arange(M.n))
    assert info.ordering_method in (S.SYM_ORDER_METHOD_MD, S.SYM_ORDER_METHOD_ND)
    assert info.flops == min(info.ordering_flops_md, info.ordering_flops_nd)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, perm, want_rel=True)
    for mine, theirs in PAIRS:
        a = s.export(mine)
        b = getattr(o, theirs)
        assert np.array_equal(a, b), mine


def test_auto_ordering_fill_against_references():
    """Fill (nnz(L)) of the automatic ordering: on 2D and 3D stencil grids at most 1.5x that of the
    geometric nested dissection the workloads use, and on Erdos-Renyi graphs (no geometry) below
    that of reverse Cuthill-McKee."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    rng = np.random.default_rng(73)
    for M in (w.laplace2d5(96, rng), w.dd2d9(64, rng), w.conduct3d(24, rng, "star"), w.conduct3d(16, rng, "box")):
        auto = _auto(M).info().nnz_l
        geom = S.Solver(M.n, M.Ap, M.Ai, M.perm, flags=S.SYM_FLAG_HOST_ONLY).info().nnz_l
        assert auto <= 1.5 * geom, (auto, geom)
    for n, d in ((3000, 4), (3000, 12)):
        M = w.erdos_renyi(n, d, rng)
        L = sp.csc_matrix((M.Ax, M.Ai, M.Ap), shape=(n, n))
        rcm = reverse_cuthill_mckee((L + L.T).tocsr(), symmetric_mode=True).astype(np.int32)
        auto = _auto(M).info().nnz_l
        ref = S.Solver(M.n, M.Ap, M.Ai, rcm, flags=S.SYM_FLAG_HOST_ONLY).info().nnz_l
        assert auto < ref, (auto, ref)


def test_auto_ordering_special_structures():
    """Degenerate patterns: empty, diagonal (no edges), a path, and a dense matrix."""
    s = S.Solver(0, np.zeros(1, np.int64), np.zeros(0, np.int32), flags=S.SYM_FLAG_HOST_ONLY, ordering="auto")
    assert s.info().n == 0
    n = 50
    diag = _auto(w.Matrix(n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int32), np.ones(n)))
    assert diag.info().nnz_l == n
    u = np.arange(n - 1)
    Ap, Ai, Ax = w.lower_csc(n, u, u + 1, -np.ones(n - 1), 3 * np.ones(n))
    path = _auto(w.Matrix(n, Ap, Ai, Ax)).info()
    assert path.nnz_l == 2 * n - 1  # a path orders without fill
    M = w.random_spd_pattern(40, 1.0, np.random.default_rng(3))
    assert _auto(M).info().nnz_l == 40 * 41 // 2
