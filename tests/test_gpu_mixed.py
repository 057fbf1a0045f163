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


def near_singular(n, target, rng):
    """B + s I with B = G G^T of rank n - 1, s chosen by bisection (on the oracle's FP64 factor)
    so that min_k d_k / C_kk is close to target."""
    G = rng.standard_normal((n, n - 1))
    Bm = G @ G.T
    lo, hi = 0.0, 1.0
    for _ in range(60):
        s = 0.5 * (lo + hi)
        M = dense_matrix(Bm + s * np.eye(n))
        o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
        assert o.factor(M.Ax) == 0
        r = oracle_pivot_ratios(o, M).min()
        if r > target:
            hi = s
        else:
            lo = s
    return M, o


@pytest.mark.parametrize("maker", [lambda: w.cfg("laplace2d5_64"),
                                   lambda: w.conduct3d(12, np.random.default_rng(4), "box"),
                                   lambda: w.vector3d27(10, np.random.default_rng(6), sub=3)])
def test_pivot_ratio_matches_oracle_and_flag_clear(torch_cuda, maker):
    """Well-conditioned and coefficient-jump cases (the latter with jumps 1 / 1e2 / 1e4): the FP64
    pivots of the FP32 factor give min d_k / C_kk within FP32 accuracy of the oracle's exact
    ratio, at a column whose exact ratio is that small, and the breakdown flag stays clear."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = maker()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.factor(torch.from_numpy(M.Ax).cuda())
    r, col, bd = s.pivot_info()
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax) == 0
    ratios = oracle_pivot_ratios(o, M)
    rmin = ratios.min()
    tol = 1e-3 * rmin + 1e-5
    assert abs(r - rmin) <= tol, (r, rmin)
    k = int(np.nonzero(o.perm == col)[0][0])  # the reported column in permuted numbering
    assert ratios[k] <= rmin + 2 * tol
    assert not bd


def test_pivot_breakdown_flag_on_near_singular_matrix(torch_cuda):
    """A dense 48 x 48 matrix shifted just off singularity (exact min d_k / C_kk = 3e-6, below the
    default threshold 2^-16): the FP64 pivot chain reports a ratio close to the exact one, the
    flag trips, the FP64 refinement still reaches the backward-error bound, and a lower
    threshold clears the flag."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M, o = near_singular(48, 3e-6, np.random.default_rng(21))
    rmin = oracle_pivot_ratios(o, M).min()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.set_refinement(1e-12, 300)
    s.factor(torch.from_numpy(M.Ax).cuda())
    r, col, bd = s.pivot_info()
    assert bd
    assert abs(r - rmin) <= 0.3 * rmin, (r, rmin)
    B, X = solve_refined(torch, s, M, 1, seed=3)
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X) <= REFINED_BERR
    S.sym_set_pivot_threshold(s.h, 1e-7)
    assert not s.pivot_info()[2]


def test_pivot_ratio_per_matrix_of_a_batch(torch_cuda):
    """A batch of two 24 x 24 dense matrices (diagonal tiles of order <= 32: the warp-per-tile
    POTRF with its own FP64 pivot chain): the near-singular one is flagged, the other is not,
    each with its own ratio."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M1, o1 = near_singular(24, 2e-6, np.random.default_rng(22))
    G = np.random.default_rng(23).standard_normal((24, 24))
    M2 = dense_matrix(G @ G.T + 24 * np.eye(24))
    o2 = oracle.Oracle(M2.n, M2.Ap, M2.Ai, M2.perm)
    assert o2.factor(M2.Ax) == 0
    s = S.Solver(M1.n, M1.Ap, M1.Ai, M1.perm, precision="mixed")
    vals = torch.from_numpy(np.stack([M1.Ax, M2.Ax])).cuda()
    S.sym_factor_batch(s.h, 2, vals, M1.nnz)
    r1, _, bd1 = S.sym_pivot_info(s.h, 0)
    r2, _, bd2 = S.sym_pivot_info(s.h, 1)
    e1 = oracle_pivot_ratios(o1, M1).min()
    e2 = oracle_pivot_ratios(o2, M2).min()
    assert bd1 and not bd2
    assert abs(r1 - e1) <= 0.3 * e1 and abs(r2 - e2) <= 1e-4 * e2, (r1, e1, r2, e2)
