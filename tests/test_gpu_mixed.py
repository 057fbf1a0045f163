"""GPU parity of the mixed-precision form: FP32 factor and FP64 conjugate-gradient refinement
preconditioned by it.

Tolerances. The FP32 factor is compared with the oracle's FP64 factor entry-wise to
MIXED_ENTRY_RTOL = 1e-4 of max|L| (u32 = 6e-8 times the perturbation bound kappa(A) <= 1e3 for
these cases) and by ||L L^T - A||_F / ||A||_F <= 1e-6. Every refined solve must reach the
spec bound for the mixed form, normwise backward error <= 1e-12, measured on the host.
"""
import numpy as np
import pytest

import oracle
import workloads as w
from tests.helpers import exports, panels_on_pattern

pytestmark = pytest.mark.gpu

MIXED_ENTRY_RTOL = 1e-4
MIXED_FACTOR_TOL = 1e-6
REFINED_BERR = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def solve_refined(torch, s, M, nrhs, seed=0):
    B = w.rhs(M.n, nrhs, np.random.default_rng(seed))
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xt = s.solve(Bt if nrhs > 1 else Bt[0])
    torch.cuda.synchronize()
    X = Xt.cpu().numpy()
    X = X.T if nrhs > 1 else X[:, None]
    return B, X


def test_mixed_factor_and_refined_solve(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.cfg("laplace2d5_64")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.factor(torch.from_numpy(M.Ax).cuda())
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax) == 0
    vals, outside = panels_on_pattern(exports(s), s.factor_panels(), o.Lp, o.Li)
    assert outside == 0.0
    assert np.abs(vals - o.Lx).max() <= MIXED_ENTRY_RTOL * np.abs(o.Lx).max()
    assert o.factor_residual_with(M.Ax, vals) <= MIXED_FACTOR_TOL
    B, X = solve_refined(torch, s, M, 4)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= REFINED_BERR
    it, be = s.refinement_info()
    assert 1 <= it <= 10 and be <= REFINED_BERR
    Xo = o.solve(B)
    assert np.abs(X - Xo).max() <= 1e-9 * np.abs(Xo).max()


@pytest.mark.parametrize("maker,nrhs", [
    (lambda: w.dd2d9(48, np.random.default_rng(2)), 1),
    (lambda: w.conduct3d(20, np.random.default_rng(3), "star"), 70),   # two refinement chunks
    (lambda: w.conduct3d(12, np.random.default_rng(4), "box"), 3),
    (lambda: w.random_spd_pattern(900, 0.006, np.random.default_rng(5)), 2),
])
def test_mixed_refined_backward_error(torch_cuda, maker, nrhs):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.factor(torch.from_numpy(M.Ax).cuda())
    B, X = solve_refined(torch, s, M, nrhs, seed=nrhs)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= REFINED_BERR


def test_mixed_ill_conditioned_coefficient_jumps(torch_cuda):
    """Vector PDE with coefficient jumps 1 / 1e2 / 1e4 by subdomain: kappa far above 1/u32 for
    plain refinement; preconditioned CG still reaches the FP64 bound."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.vector3d27(10, np.random.default_rng(6), sub=3)
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.set_refinement(1e-12, 300)
    s.factor(torch.from_numpy(M.Ax).cuda())
    B, X = solve_refined(torch, s, M, 2, seed=9)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= REFINED_BERR


def test_mixed_iteration_limit_reports_no_convergence(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.conduct3d(10, np.random.default_rng(8), "star")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.set_refinement(1e-30, 2)  # unreachable tolerance
    s.factor(torch.from_numpy(M.Ax).cuda())
    b = torch.from_numpy(w.rhs(M.n, 1, np.random.default_rng(0))[:, 0]).cuda()
    with pytest.raises(S.SymError) as e:
        s.solve(b)
    assert e.value.code == S.SYM_ERR_NO_CONVERGENCE
    assert s.refinement_info()[0] == 2


def test_mixed_not_spd(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.laplace2d5(16, np.random.default_rng(5))
    Ax = M.Ax.copy()
    Ax[M.Ap[:-1][77]] = -3.0
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(Ax) == oracle.ERR_NOT_SPD
    with pytest.raises(S.SymError) as e:
        s.factor(torch.from_numpy(Ax).cuda())
    assert e.value.code == S.SYM_ERR_NOT_SPD
    assert s.error_column() == o.perm[o.err_col]


# ---------------------------------------------------------------------------------------------
# FP64 pivots of the FP32 factor and the breakdown ratio min_k d_k / C_kk

def oracle_pivot_ratios(o, M):
    """Exact FP64 ratios d_k / C_kk = L_kk^2 / C_kk of the oracle's factor (permuted order)."""
    d = o.Lx[o.Lp[:-1]] ** 2
    ckk = M.Ax[M.Ap[:-1]][o.perm]
    return d / ckk


def dense_matrix(A):
    """A dense symmetric matrix as the library's input (full lower triangle, CSC)."""
    n = A.shape[0]
    rows = [np.arange(j, n) for j in range(n)]
    Ap = np.concatenate([[0], np.cumsum([r.size for r in rows])]).astype(np.int64)
    Ai = np.concatenate(rows).astype(np.int32)
    Ax = np.concatenate([A[j:, j] for j in range(n)])
    return w.Matrix(n, Ap, Ai, Ax, np.arange(n, dtype=np.int32))


def arrow_block(v, s):
    """The dense matrix [[I, v], [v^T, v.v + s]]: its exact factor is [[I, 0], [v^T, sqrt(s)]], so
    every pivot is 1 except the last, d = s, and min_k d_k / C_kk = s / (v.v + s). With v
    representable in FP32 the tile's multipliers are exact, and the FP64 pivot chain (C_nn in
    FP64, the squares subtracted in FP64) recovers s to FP64 rounding of v.v; an FP32 chain would
    lose several percent of s in the rounding of C_nn and of the sum of squares (n u32 v.v)."""
    n = v.size + 1
    A = np.eye(n)
    A[-1, :-1] = v
    A[:-1, -1] = v
    A[-1, -1] = float(v @ v) + s
    return dense_matrix(A)


def fp32_values(rng, size, lo=0.5, hi=1.0):
    return rng.uniform(lo, hi, size).astype(np.float32).astype(np.float64)


def panel_diagonal(s):
    """The stored diagonal L_kk of the factor (permuted order), from its panels."""
    sup, rowptr, lxptr = s.export("super"), s.export("rowptr"), s.export("lxptr")
    Lx = s.factor_panels()
    d = np.empty(int(sup[-1]))
    for J in range(sup.size - 1):
        f, l = int(sup[J]), int(sup[J + 1])
        nr = int(rowptr[J + 1] - rowptr[J])
        panel = Lx[lxptr[J]:lxptr[J + 1]].reshape(l - f, nr)
        d[f:l] = panel[np.arange(l - f), np.arange(l - f)]
    return d


@pytest.mark.parametrize("maker", [lambda: w.cfg("laplace2d5_64"),
                                   lambda: w.conduct3d(12, np.random.default_rng(4), "box"),
                                   lambda: w.vector3d27(10, np.random.default_rng(6), sub=3)])
def test_pivot_ratio_matches_oracle_and_flag_clear(torch_cuda, maker):
    """Well-conditioned and coefficient-jump cases (the last with jumps 1 / 1e2 / 1e4):
    - the reported minimum is min_k L_kk^2 / C_kk of the factor's own stored diagonal (the FP64
      pivot rounded once to FP32 by its square root: within 2^-22 relative), at that column;
    - it agrees with the oracle's exact ratio within the FP32 factor's forward-error bound:
      |L_kk - L*_kk| <= delta = 5e-4 max|L| (the bound the tensor-core factor tests use) gives
      |ratio_k - ratio*_k| <= (2 L*_kk delta + delta^2) / C_kk;
    - the breakdown flag stays clear."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.factor(torch.from_numpy(M.Ax).cuda())
    r, col, bd = s.pivot_info()
    assert not bd
    perm = s.export("perm")
    ckk = M.Ax[M.Ap[:-1]][perm]
    own = panel_diagonal(s) ** 2 / ckk
    k = int(np.nonzero(perm == col)[0][0])  # the reported column in permuted numbering
    assert abs(r - own.min()) <= 5e-7 * own.min() and abs(own[k] - r) <= 5e-7 * r
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax) == 0
    exact = oracle_pivot_ratios(o, M)
    delta = 5e-4 * np.abs(o.Lx).max()
    lkk = o.Lx[o.Lp[:-1]]
    bound = float(np.max((2 * lkk * delta + delta ** 2) / ckk))
    assert abs(r - exact.min()) <= bound, (r, exact.min(), bound)


@pytest.mark.parametrize("n", [48, 64])
def test_pivot_breakdown_flag_on_near_singular_matrix(torch_cuda, n):
    """A dense matrix one pivot away from singular (exact ratio s / C_nn = 3e-6, below the
    default threshold 2^-16): the FP64 pivot chain of the FP32 factor reports the exact ratio to
    FP64 rounding of v.v relative to s (1e-8; an FP32 chain is off by percents here), flags
    breakdown at the last column, the FP64 refinement still reaches the backward-error bound, and
    a lower threshold clears the flag."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    v = fp32_values(np.random.default_rng(21 + n), n - 1)
    vv = float(v @ v)
    sh = 3e-6 * vv / (1 - 3e-6)
    M = arrow_block(v, sh)
    exact = sh / (vv + sh)
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.set_refinement(1e-12, 300)
    s.factor(torch.from_numpy(M.Ax).cuda())
    r, col, bd = s.pivot_info()
    assert bd and col == n - 1
    assert abs(r - exact) <= 1e-8 * exact, (r, exact)
    B, X = solve_refined(torch, s, M, 1, seed=3)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= REFINED_BERR
    S.sym_set_pivot_threshold(s.h, 1e-7)
    assert not s.pivot_info()[2]


def test_pivot_ratio_per_matrix_of_a_batch(torch_cuda):
    """A batch of two 24 x 24 dense matrices (diagonal tiles of order <= 32: the warp-per-tile
    POTRF with its own FP64 pivot chain): the near-singular one is flagged at its last column,
    the well-conditioned one is not; each ratio matches its exact value."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    v = fp32_values(np.random.default_rng(22), 23)
    vv = float(v @ v)
    sh = 2e-6 * vv / (1 - 2e-6)
    M1 = arrow_block(v, sh)
    M2 = arrow_block(v, 4.0 * vv)  # last pivot 4 v.v: ratio 0.8; the others 1
    s = S.Solver(M1.n, M1.Ap, M1.Ai, M1.perm, precision="mixed")
    vals = torch.from_numpy(np.stack([M1.Ax, M2.Ax])).cuda()
    S.sym_factor_batch(s.h, 2, vals, M1.nnz)
    r1, c1, bd1 = S.sym_pivot_info(s.h, 0)
    r2, c2, bd2 = S.sym_pivot_info(s.h, 1)
    assert bd1 and c1 == 23 and not bd2 and c2 == 23
    assert abs(r1 - sh / (vv + sh)) <= 1e-8 * r1
    assert abs(r2 - 0.8) <= 1e-6


def test_autotune_mixed_precision(torch_cuda):
    """The autotuner on an FP32 factor (tensor-core or SIMT updates of full tiles, one-CTA or
    one-warp small-tile POTRF/TRTRI, per launch): whatever forms it keeps, the FP32 factor stays
    within the FP32 forward-error bound of the oracle's, and the refined solve reaches 1e-12."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.cfg("conduct3d7_48")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.set_refinement(1e-12, 100)
    Ax = torch.from_numpy(M.Ax).cuda()
    tuned, changed = S.sym_autotune(s.h, 1, Ax, M.nnz, 2)
    assert tuned > 0 and 0 <= changed <= tuned
    s.factor(Ax)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    kmax = 20000
    assert o.factor(M.Ax, kmax) == 0
    vals, outside = panels_on_pattern(exports(s), s.factor_panels(), o.Lp, o.Li)
    cols = np.repeat(np.arange(M.n), np.diff(o.Lp))
    sel = (cols < kmax) & (o.Li < kmax)
    assert outside == 0.0
    assert np.abs(vals[sel] - o.Lx[sel]).max() <= 5e-4 * np.abs(o.Lx[sel]).max()
    B, X = solve_refined(torch, s, M, 2)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= REFINED_BERR
