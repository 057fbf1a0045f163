"""GPU parity of batched refactorization (many value sets on one pattern) and of uneven batches
(a block-diagonal union of different grids analyzed once)."""
import numpy as np
import pytest

import oracle
import workloads as w
from tests.helpers import exports, panels_on_pattern

pytestmark = pytest.mark.gpu

ENTRY_RTOL = 1e-10
BERR_TOL = 1e-13
REFINED_BERR = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_batch_matches_single_factorizations(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    nb, nrhs = 6, 3
    M, vals = w.same_pattern_batch(lambda r: w.dd2d9(24, r), nb, 40)
    stride = M.nnz + 5  # padded rows
    V = np.zeros((nb, stride))
    V[:, :M.nnz] = vals
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    S.sym_factor_batch(s.h, nb, torch.from_numpy(V).cuda(), stride)
    rng = np.random.default_rng(1)
    B = np.stack([w.rhs(M.n, nrhs, rng).T for _ in range(nb)])  # (nb, nrhs, n): row = one RHS
    Bt = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Xt = torch.empty_like(Bt)
    S.sym_solve_batch(s.h, nb, nrhs, Bt, M.n, nrhs * M.n, Xt, M.n, nrhs * M.n)
    torch.cuda.synchronize()
    X = Xt.cpu().numpy()
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    sx = exports(s)
    for b in range(nb):
        assert oracle.backward_error(M.n, M.Ap, M.Ai, vals[b], B[b].T, X[b].T) <= BERR_TOL
        o.factor(vals[b])
        Lb, outside = panels_on_pattern(sx, S.sym_get_batch_factor_host(s.h, b), o.Lp, o.Li)
        assert outside == 0.0
        assert np.abs(Lb - o.Lx).max() <= ENTRY_RTOL * np.abs(o.Lx).max()
    # a single factorization of matrix 4 gives the batch's panels up to rounding: a lone matrix
    # spreads the tiles of its short update launches over thread-block clusters (partial sums
    # added in rank order), the batch keeps one CTA per tile; each is deterministic
    single = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    single.factor(torch.from_numpy(vals[4]).cuda())
    a, b = single.factor_panels(), S.sym_get_batch_factor_host(s.h, 4)
    assert np.abs(a - b).max() <= 1e-13 * np.abs(b).max()
    single.factor(torch.from_numpy(vals[4]).cuda())
    assert np.array_equal(single.factor_panels(), a)


def test_batch_reports_each_failing_matrix(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    nb = 5
    M, vals = w.same_pattern_batch(lambda r: w.laplace2d5(16, r), nb, 7)
    vals = vals.copy()
    vals[1, M.Ap[33]] = -1.0
    vals[3, M.Ap[200]] = -2.0
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    with pytest.raises(S.SymError) as e:
        S.sym_factor_batch(s.h, nb, torch.from_numpy(vals).cuda(), M.nnz)
    assert e.value.code == S.SYM_ERR_NOT_SPD
    cols = S.sym_batch_error_columns(s.h, nb)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    for b in range(nb):
        rc = o.factor(vals[b])
        assert cols[b] == (o.perm[o.err_col] if rc == oracle.ERR_NOT_SPD else -1)
    assert cols[0] == -1 and cols[1] >= 0 and cols[3] >= 0


def test_mixed_precision_batch(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    nb = 4
    M, vals = w.same_pattern_batch(lambda r: w.conduct3d(10, r, "star"), nb, 3)
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    S.sym_factor_batch(s.h, nb, torch.from_numpy(vals).cuda(), M.nnz)
    B = np.stack([w.rhs(M.n, 2, np.random.default_rng(b)).T for b in range(nb)])
    Bt = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    Xt = torch.empty_like(Bt)
    S.sym_solve_batch(s.h, nb, 2, Bt, M.n, 2 * M.n, Xt, M.n, 2 * M.n)
    torch.cuda.synchronize()
    X = Xt.cpu().numpy()
    for b in range(nb):
        assert oracle.backward_error(M.n, M.Ap, M.Ai, vals[b], B[b].T, X[b].T) <= REFINED_BERR


def test_uneven_batch_as_block_diagonal(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    rng = np.random.default_rng(11)
    mats, sides = w.uneven_grid_batch(7, rng, lo=12, hi=70)
    U = w.block_diagonal(mats)
    s = S.Solver(U.n, U.Ap, U.Ai, U.perm)
    s.factor(torch.from_numpy(U.Ax).cuda())
    b = w.rhs(U.n, 1, np.random.default_rng(2))[:, 0]
    x = s.solve(torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    x = x.cpu().numpy()
    off = 0
    for M in mats:
        seg = slice(off, off + M.n)
        assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, b[seg], x[seg]) <= BERR_TOL
        off += M.n


def test_autotune_keeps_results(torch_cuda):
    """The batch autotuner times both kernel forms of the batch's small-tile launches and keeps the
    faster; whatever it picks, every matrix's factor still matches the oracle, and refactoring
    with the tuned plan agrees with the untuned one up to rounding (the forms add in other
    orders)."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    nb = 8
    M, vals = w.same_pattern_batch(lambda r: w.dd2d9(28, r), nb, 50)
    V = torch.from_numpy(np.ascontiguousarray(vals)).cuda()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    S.sym_factor_batch(s.h, nb, V, M.nnz)
    before = [S.sym_get_batch_factor_host(s.h, b).copy() for b in range(nb)]
    tuned, changed = S.sym_autotune(s.h, nb, V, M.nnz, 2)
    assert tuned > 0 and 0 <= changed <= tuned
    S.sym_factor_batch(s.h, nb, V, M.nnz)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    sx = exports(s)
    for b in range(nb):
        after = S.sym_get_batch_factor_host(s.h, b)
        assert np.abs(after - before[b]).max() <= 1e-13 * np.abs(before[b]).max()
        o.factor(vals[b])
        Lb, outside = panels_on_pattern(sx, after, o.Lp, o.Li)
        assert outside == 0.0 and np.abs(Lb - o.Lx).max() <= ENTRY_RTOL * np.abs(o.Lx).max()
    # tuning the handle for one matrix keeps the batch's choice (the two are stored apart): the
    # batch's factors are bit-identical afterwards
    tuned_batch = [S.sym_get_batch_factor_host(s.h, b).copy() for b in range(nb)]
    tuned1, _ = S.sym_autotune(s.h, 1, V, M.nnz, 1)
    assert tuned1 > 0
    S.sym_factor_batch(s.h, nb, V, M.nnz)
    for b in range(nb):
        assert np.array_equal(S.sym_get_batch_factor_host(s.h, b), tuned_batch[b])


@pytest.mark.parametrize("precision", [None, "mixed"])
def test_fused_narrow_levels_match_separate_launches(torch_cuda, precision):
    """A batch factors each level of narrow supernodes in one launch (lanes = matrices, 1 to 8 lanes
    per matrix on this pattern, 37 matrices: ragged lane groups), and an FP64 batch solves each such
    level in one launch per direction. The panels equal, bit for bit, those of the level's separate
    POTRF, TRSM and TRTRI launches; the solutions agree with the separate solve launches' to
    rounding (the fused backward gather sums its rows in another order) and match the oracle.
    Single matrices fuse the same levels (the mixed-precision batch's refined solves)."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    nb, nrhs = 37, 2
    M, vals = w.same_pattern_batch(lambda r: w.dd2d9(48, r), nb, 60)
    V = torch.from_numpy(vals).cuda()
    fused = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision=precision)
    apart = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision=precision, flags=S.SYM_FLAG_NO_FUSED_LEVELS)
    assert (fused.export("batch_panel").reshape(-1, 4)[:, 0] == 1).sum() >= 4
    assert (fused.export("fwd_panel").reshape(-1, 4)[:, 0] == 1).sum() >= 3
    assert (fused.export("bwd_panel").reshape(-1, 4)[:, 0] == 1).sum() >= 3
    B = torch.from_numpy(np.stack([w.rhs(M.n, nrhs, np.random.default_rng(b)).T for b in range(nb)])).cuda()
    out = []
    for s in (fused, apart):
        S.sym_factor_batch(s.h, nb, V, M.nnz)
        X = torch.empty_like(B)
        S.sym_solve_batch(s.h, nb, nrhs, B, M.n, nrhs * M.n, X, M.n, nrhs * M.n)
        torch.cuda.synchronize()
        out.append(([S.sym_get_batch_factor_host(s.h, b).copy() for b in range(nb)], X.cpu().numpy()))
    for b in range(nb):
        assert np.array_equal(out[0][0][b], out[1][0][b])
    if precision is None:  # (a mixed-precision batch is refined one matrix at a time; both reach
        # the refinement's backward error, checked below)
        assert np.abs(out[0][1] - out[1][1]).max() <= 1e-12 * np.abs(out[1][1]).max()
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    sx = exports(fused)
    Bh = B.cpu().numpy()
    for b in (0, 31, 32, nb - 1):
        assert oracle.backward_error(M.n, M.Ap, M.Ai, vals[b], Bh[b].T, out[0][1][b].T) <= (
            BERR_TOL if precision is None else REFINED_BERR)
        if precision is None:
            o.factor(vals[b])
            Lb, outside = panels_on_pattern(sx, out[0][0][b], o.Lp, o.Li)
            assert outside == 0.0 and np.abs(Lb - o.Lx).max() <= ENTRY_RTOL * np.abs(o.Lx).max()
