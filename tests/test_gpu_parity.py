"""GPU parity: the CUDA path (through the C ABI) against the CPU FP64 oracle.

Tolerances. Spec bounds for FP64: ||L L^T - A||_F / ||A||_F <= 1e-12 and normwise backward
error <= 1e-13 for every solve. Entry-wise, both factors are backward stable with
||dA|| <= c n^{1/2} u ||A|| for a small c; by the perturbation bound for the Cholesky factor
(||dL||_F / ||L||_2 <= kappa_2(A) ||dA||_F / ||A||_2 up to a constant) two such factors differ
by at most about kappa(A) * 1e-15 relative to max|L|. The matrices below have kappa <= 1e5, so
entry-wise agreement is required to ENTRY_RTOL = 1e-10 of max|L|.
"""
import numpy as np
import pytest

import oracle
import workloads as w
from tests.helpers import exports, panels_on_pattern

pytestmark = pytest.mark.gpu

ENTRY_RTOL = 1e-10
FACTOR_TOL = 1e-12
BERR_TOL = 1e-13


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _lib():
    import paper_1705_06575_gb300 as S
    return S


def check_matrix(torch, M, nrhs=1, kmax=-1, seed=0, solve_oracle=True):
    """Factor M on the GPU and compare with the oracle; returns a dict of measured errors."""
    S = _lib()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    # symbolic parity (bit exact)
    assert np.array_equal(s.export("perm"), o.perm)
    assert np.array_equal(s.export("super"), o.sn)
    Ax = torch.from_numpy(M.Ax).cuda()
    s.factor(Ax)
    Lx = s.factor_panels()
    rc = o.factor(M.Ax, kmax)
    assert rc == 0
    vals, outside = panels_on_pattern(exports(s), Lx, o.Lp, o.Li)
    assert outside == 0.0, "values outside the exact pattern must stay exactly zero"
    res = {}
    if kmax < 0 or kmax >= M.n:
        ref = o.Lx
        err = np.abs(vals - ref).max() / np.abs(ref).max()
        res["entry"] = err
        res["factor_resid"] = o.factor_residual_with(M.Ax, vals)
    else:
        # leading kmax x kmax block: the oracle computed exactly those rows
        cols = np.repeat(np.arange(M.n), np.diff(o.Lp))
        sel = (cols < kmax) & (o.Li < kmax)
        ref = o.Lx[sel]
        err = np.abs(vals[sel] - ref).max() / np.abs(ref).max()
        res["entry"] = err
        res["factor_resid"] = o.factor_residual_with(M.Ax, vals, kmax)
    assert res["entry"] <= ENTRY_RTOL, res
    assert res["factor_resid"] <= FACTOR_TOL, res
    rng = np.random.default_rng(seed)
    B = w.rhs(M.n, nrhs, rng)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()  # row q = right-hand side q
    Xt = s.solve(Bt if nrhs > 1 else Bt[0])
    torch.cuda.synchronize()
    X = Xt.cpu().numpy()
    X = X.T if nrhs > 1 else X[:, None]
    res["berr"] = oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X)
    assert res["berr"] <= BERR_TOL, res
    if solve_oracle and (kmax < 0 or kmax >= M.n):
        Xo = o.solve(B)
        res["x_vs_oracle"] = np.abs(X - Xo).max() / np.abs(Xo).max()
    s.close()
    return res


def test_laplace2d5_64(torch_cuda):
    r = check_matrix(torch_cuda, w.cfg("laplace2d5_64"), nrhs=1)
    assert r["x_vs_oracle"] < 1e-10


def test_laplace2d5_64_four_rhs(torch_cuda):
    check_matrix(torch_cuda, w.cfg("laplace2d5_64"), nrhs=4)


def test_many_rhs_two_passes(torch_cuda):
    check_matrix(torch_cuda, w.laplace2d5(24, np.random.default_rng(3)), nrhs=11)


@pytest.mark.parametrize("n,density,seed", [(300, 0.02, 1), (700, 0.01, 2), (1500, 0.004, 3)])
def test_random_patterns_natural_order(torch_cuda, n, density, seed):
    M = w.random_spd_pattern(n, density, np.random.default_rng(seed))
    check_matrix(torch_cuda, M, nrhs=2)


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 200, 333])
def test_dense(torch_cuda, n):
    """One supernode: multi-tile POTRF / TRSM / GEMM with a ragged last tile."""
    M = w.random_spd_pattern(n, 1.0, np.random.default_rng(n))
    check_matrix(torch_cuda, M, nrhs=3)


def test_diagonal_and_tridiagonal(torch_cuda):
    n = 500
    Ap = np.arange(n + 1, dtype=np.int64)
    Ai = np.arange(n, dtype=np.int32)
    M = w.Matrix(n, Ap, Ai, np.linspace(1.0, 3.0, n))
    check_matrix(torch_cuda, M)
    u = np.arange(n - 1)
    Ap, Ai, Ax = w.lower_csc(n, u, u + 1, -np.ones(n - 1), 2.5 * np.ones(n))
    check_matrix(torch_cuda, w.Matrix(n, Ap, Ai, Ax))


def test_pivot_square_roots_within_two_ulp(torch_cuda):
    """Diagonal matrices: every L_jj is a pivot square root computed by the POTRF kernel's
    Newton-Raphson reciprocal square root; it must match IEEE sqrt within 2 ulp over a wide
    range of magnitudes (including values outside the single-precision range)."""
    torch = torch_cuda
    S = _lib()
    rng = np.random.default_rng(17)
    d = np.concatenate([10.0 ** rng.uniform(-300, 300, 2000), rng.uniform(0.5, 2.0, 2000),
                        10.0 ** rng.uniform(-29, 29, 2000)])
    n = d.size
    Ap = np.arange(n + 1, dtype=np.int64)
    Ai = np.arange(n, dtype=np.int32)
    s = S.Solver(n, Ap, Ai)
    s.factor(torch.from_numpy(d).cuda())
    Lx = s.factor_panels()
    perm = s.export("perm")
    lx = s.export("lxptr")
    got = Lx[lx[:-1]]  # one 1 x 1 panel per column, in the final order
    ref = np.sqrt(d[perm])
    ulp = np.abs(got - ref) / np.spacing(ref)
    assert ulp.max() <= 2.0, ulp.max()


def test_grids_nested_dissection(torch_cuda):
    rng = np.random.default_rng(7)
    check_matrix(torch_cuda, w.dd2d9(48, rng), nrhs=2)
    check_matrix(torch_cuda, w.conduct3d(16, rng, "star"), nrhs=1)
    check_matrix(torch_cuda, w.conduct3d(12, rng, "box"), nrhs=1)


def test_refactor_new_values_same_handle(torch_cuda):
    torch = torch_cuda
    S = _lib()
    M = w.laplace2d5(40, np.random.default_rng(11))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    for t in range(3):
        Ax = M.Ax * (1.0 + 0.1 * t)
        Ax = Ax + (np.arange(Ax.size) % 7) * 1e-3 * t
        s.factor(torch.from_numpy(Ax).cuda())
        o.factor(Ax)
        vals, _ = panels_on_pattern(exports(s), s.factor_panels(), o.Lp, o.Li)
        assert np.abs(vals - o.Lx).max() / np.abs(o.Lx).max() <= ENTRY_RTOL


def test_not_spd_reports_first_column(torch_cuda):
    torch = torch_cuda
    S = _lib()
    M = w.laplace2d5(20, np.random.default_rng(5))
    Ax = M.Ax.copy()
    diag_pos = M.Ap[:-1]
    Ax[diag_pos[137]] = -5.0
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(Ax) == oracle.ERR_NOT_SPD
    with pytest.raises(S.SymError) as ei:
        s.factor(torch.from_numpy(Ax).cuda())
    assert ei.value.code == S.SYM_ERR_NOT_SPD
    assert s.error_column() == o.perm[o.err_col]
    # a solve after a failed factorization is refused, then a good factorization recovers
    with pytest.raises(S.SymError):
        s.solve(torch.zeros(M.n, dtype=torch.float64, device="cuda"))
    s.factor(torch.from_numpy(M.Ax).cuda())
    assert s.error_column() == -1


def test_empty_matrix(torch_cuda):
    torch = torch_cuda
    S = _lib()
    s = S.Solver(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    s.factor(torch.zeros(1, dtype=torch.float64, device="cuda"))
    assert s.info().nsuper == 0


def test_host_pointer_variants(torch_cuda):
    S = _lib()
    M = w.laplace2d5(30, np.random.default_rng(9))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.factor_host(M.Ax)
    B = w.rhs(M.n, 3, np.random.default_rng(1))
    X = s.solve_host(B)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= BERR_TOL


def test_user_stream(torch_cuda):
    torch = torch_cuda
    M = w.laplace2d5(32, np.random.default_rng(2))
    S = _lib()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    st = torch.cuda.Stream()
    s.set_stream(st)
    with torch.cuda.stream(st):
        Ax = torch.from_numpy(M.Ax).cuda()
        b = torch.from_numpy(w.rhs(M.n, 1, np.random.default_rng(0))[:, 0]).cuda()
    st.synchronize()
    s.factor(Ax)
    x = s.solve(b)
    st.synchronize()
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, b.cpu().numpy(), x.cpu().numpy()) <= BERR_TOL


def test_lookahead_matches_one_stream_bit_for_bit(torch_cuda):
    """The two-stream (lookahead) factor performs each tile's arithmetic in the same order as
    the one-stream run of the same list, so the two factors agree bit for bit; both match the
    oracle. The 3D grid has separators several column tiles wide, so the lookahead chain, its
    row-half split and the auxiliary-stream updates all run."""
    torch = torch_cuda
    S = _lib()
    M = w.conduct3d(20, np.random.default_rng(5), "star")
    Ax = torch.from_numpy(M.Ax).cuda()
    panels = []
    for flags in (0, S.SYM_FLAG_ONE_STREAM, 0):
        s = S.Solver(M.n, M.Ap, M.Ai, M.perm, flags=flags)
        assert max(s.export("super")[1:] - s.export("super")[:-1]) > 3 * 64
        for _ in range(2):  # the second call replays the captured graph
            s.factor(Ax)
        panels.append(s.factor_panels().copy())
        s.close()
    assert np.array_equal(panels[0], panels[1])
    assert np.array_equal(panels[0], panels[2])
    check_matrix(torch, M, nrhs=1)


def test_conduct3d27_40_full(torch_cuda):
    """27-point 40^3 (n = 64,000; dense separator supernodes up to ~2400 columns, where the
    lookahead chain, the row-half split and the cluster updates run at full size): the whole
    factor entry-wise against the oracle's complete up-looking factorization (2.6e10 flops),
    the full factor residual, and the solve by backward error and against the oracle's x."""
    r = check_matrix(torch_cuda, w.cfg("conduct3d27_40"), nrhs=2)
    assert r["x_vs_oracle"] < 1e-10, r


def test_conduct3d7_64_full_size(torch_cuda):
    """The benchmark workload (64^3, 7-point, 4 right-hand sides) in the launch configuration the
    benchmark times: leading 20000 columns entry-wise against the oracle, the leading-block
    factor residual, and the backward error of all four solves."""
    check_matrix(torch_cuda, w.cfg("conduct3d7_64"), nrhs=4, kmax=20000, solve_oracle=False)


@pytest.mark.parametrize("maker", [lambda r: w.erdos_renyi(3000, 8, r), lambda r: w.conduct3d(18, r, "star")])
def test_auto_ordering_factor_and_solve(torch_cuda, maker):
    """The inspector's own ordering (SYM_ORDER_AUTO) on a graph without geometry and on a grid:
    the factor entry-wise against the oracle run with the same final permutation, and the solve."""
    torch = torch_cuda
    S = _lib()
    M = maker(np.random.default_rng(31))
    s = S.Solver(M.n, M.Ap, M.Ai, ordering="auto")
    perm = s.export("perm")
    o = oracle.Oracle(M.n, M.Ap, M.Ai, perm)
    assert np.array_equal(s.export("super"), o.sn)
    s.factor(torch.from_numpy(M.Ax).cuda())
    assert o.factor(M.Ax) == 0
    vals, outside = panels_on_pattern(exports(s), s.factor_panels(), o.Lp, o.Li)
    assert outside == 0.0
    assert np.abs(vals - o.Lx).max() <= ENTRY_RTOL * np.abs(o.Lx).max()
    assert o.factor_residual_with(M.Ax, vals) <= FACTOR_TOL
    B = w.rhs(M.n, 2, np.random.default_rng(2))
    X = s.solve_host(B)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= BERR_TOL
    s.close()


def test_autotune_one_matrix(torch_cuda):
    """The autotuner on one matrix: its tunable launches are exactly the schedule's clustered
    FP64 updates and small-tile POTRF / TRTRI launches; whatever forms it keeps, the factor still
    matches the oracle entry by entry and the solve's backward error stays within bound."""
    torch = torch_cuda
    S = _lib()
    M = w.cfg("laplace2d5_64")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    raw = s.export("factor_launches").reshape(-1, 5)
    kind, cluster, tb = raw[:, 0] & 0xffffffff, raw[:, 3] & 0xffffffff, raw[:, 4] >> 32
    want = int(np.sum(((kind == 1) & (cluster > 1) & (tb != 32)) | ((tb == 32) & ((kind == 2) | (kind == 5)))))
    assert want > 0 and np.any((kind == 1) & (cluster > 1))
    Ax = torch.from_numpy(M.Ax).cuda()
    s.factor(Ax)
    L0 = s.factor_panels().copy()
    tuned, changed = S.sym_autotune(s.h, 1, Ax, M.nnz, 2)
    assert tuned == want and 0 <= changed <= tuned
    s.factor(Ax)
    L1 = s.factor_panels()
    assert np.abs(L1 - L0).max() <= 1e-13 * np.abs(L0).max()
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax, -1) == 0
    vals, outside = panels_on_pattern(exports(s), L1, o.Lp, o.Li)
    assert outside == 0.0 and np.abs(vals - o.Lx).max() <= ENTRY_RTOL * np.abs(o.Lx).max()
    B = w.rhs(M.n, 1, np.random.default_rng(3))
    x = s.solve(torch.from_numpy(np.ascontiguousarray(B[:, 0])).cuda()).cpu().numpy()
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, x[:, None]) <= BERR_TOL


@pytest.mark.parametrize("maker", [lambda r: w.laplace2d5(40, r), lambda r: w.conduct3d(12, r, "star")])
@pytest.mark.parametrize("precision", [None, "mixed"])
def test_fused_narrow_levels_one_matrix(torch_cuda, maker, precision):
    """A single matrix solving one or two right-hand sides runs each level of supernodes of at most
    32 columns as one launch per direction (one warp per supernode, rows spread over the lanes):
    the forward sums, steps and pushes, the backward gathers and steps; its factor runs a level as
    one launch (POTRF + TRSM + TRTRI) where the autotuner finds that faster. Solutions agree with
    the separate launches' to rounding (the fused backward gather sums its rows in another order)
    and match the oracle."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = maker(np.random.default_rng(21))
    fused = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision=precision)
    apart = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision=precision, flags=S.SYM_FLAG_NO_FUSED_LEVELS)
    assert (fused.export("batch_panel").reshape(-1, 4)[:, 0] == 1).sum() >= 3
    assert (fused.export("fwd_panel").reshape(-1, 4)[:, 0] == 1).sum() >= 3
    Ax = torch.from_numpy(M.Ax).cuda()
    tuned, _ = S.sym_autotune(fused.h, 1, Ax, M.nnz, 1)
    assert tuned >= 3  # at least the fused levels were timed
    Bh = w.rhs(M.n, 2, np.random.default_rng(4))
    B = torch.from_numpy(np.ascontiguousarray(Bh.T)).cuda()
    out = []
    for s in (fused, apart):
        s.factor(Ax)
        X = torch.empty_like(B)
        S.sym_solve_multi(s.h, 2, B, M.n, X, M.n)
        torch.cuda.synchronize()
        out.append((s.factor_panels().copy(), X.cpu().numpy()))
    tol = BERR_TOL if precision is None else 1e-12
    for L, X in out:
        assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, Bh, X.T) <= tol
    if precision is None:
        assert np.abs(out[0][1] - out[1][1]).max() <= 1e-12 * np.abs(out[1][1]).max()
        o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
        o.factor(M.Ax)
        Lb, outside = panels_on_pattern(exports(fused), out[0][0], o.Lp, o.Li)
        assert outside == 0.0 and np.abs(Lb - o.Lx).max() <= ENTRY_RTOL * np.abs(o.Lx).max()
