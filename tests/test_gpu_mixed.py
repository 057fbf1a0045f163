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
