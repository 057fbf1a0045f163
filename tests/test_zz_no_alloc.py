"""sym_solve_multi_noalloc: the solve for callers that may not allocate device memory.

It must give the same results as sym_solve_multi (the allocating entry point) on consecutive
calls, since every call reuses the same fixed work array, and it must refuse sizes above its
documented limit without issuing any work. This file is collected last on purpose."""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu

ENTRY_RTOL = 1e-10  # the entry-wise tolerance of the GPU parity tests
BERR_TOL = 1e-13


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_noalloc_solve_matches_allocating_solve(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.laplace2d5(48, np.random.default_rng(123))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.factor(torch.from_numpy(M.Ax).cuda())
    rng = np.random.default_rng(5)
    for call in range(2):  # two calls in a row share (and overwrite) the fixed work array
        nrhs = 3 + call
        B = w.rhs(M.n, nrhs, rng)
        Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
        X_ref = torch.empty_like(Bt)
        X_new = torch.full_like(Bt, float("nan"))
        S.sym_solve_multi(s.h, nrhs, Bt, M.n, X_ref, M.n)
        S.sym_solve_multi_noalloc(s.h, nrhs, Bt, M.n, X_new, M.n)
        torch.cuda.synchronize()
        xr = X_ref.cpu().numpy().T
        xn = X_new.cpu().numpy().T
        assert np.abs(xn - xr).max() <= ENTRY_RTOL * np.abs(xr).max()
        assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, xn) <= BERR_TOL
    s.close()


def test_noalloc_solve_rejects_sizes_over_the_limit(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.laplace2d5(32, np.random.default_rng(1))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.factor(torch.from_numpy(M.Ax).cuda())
    nrhs = S.SYM_NOALLOC_MAX_WORK // M.n + 1
    B = torch.zeros((nrhs, M.n), dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    with pytest.raises(S.SymError) as e:
        S.sym_solve_multi_noalloc(s.h, nrhs, B, M.n, X, M.n)
    assert e.value.code == S.SYM_ERR_LIMIT
    s.close()
