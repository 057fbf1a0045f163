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


def test_noalloc_first_solve_allocates_nothing(torch_cuda):
    """The entry point as the first solve of a freshly factored handle (its one-time set-up path),
    then a second call: the device's free memory is the same before and after the second call,
    and both results match the oracle's solution."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.laplace2d5(40, np.random.default_rng(7))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.factor(torch.from_numpy(M.Ax).cuda())
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax) == 0
    rng = np.random.default_rng(9)
    B = w.rhs(M.n, 2, rng)
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    Xo = o.solve(B)
    X = torch.full_like(Bt, float("nan"))
    S.sym_solve_multi_noalloc(s.h, 2, Bt, M.n, X, M.n)  # first solve of this handle
    torch.cuda.synchronize()
    x1 = X.cpu().numpy().T
    assert np.abs(x1 - Xo).max() <= ENTRY_RTOL * np.abs(Xo).max()
    X.fill_(float("nan"))
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    S.sym_solve_multi_noalloc(s.h, 2, Bt, M.n, X, M.n)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    x2 = X.cpu().numpy().T
    assert np.abs(x2 - Xo).max() <= ENTRY_RTOL * np.abs(Xo).max()
    s.close()


def test_noalloc_solve_at_exactly_the_limit(torch_cuda):
    """n * nrhs equal to SYM_NOALLOC_MAX_WORK is accepted and uses the whole array: a 32 x 32 grid
    (n = 1024) with 1024 right-hand sides, each solved to the backward-error bound."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.laplace2d5(32, np.random.default_rng(13))
    nrhs = S.SYM_NOALLOC_MAX_WORK // M.n
    assert nrhs * M.n == S.SYM_NOALLOC_MAX_WORK
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.factor(torch.from_numpy(M.Ax).cuda())
    B = w.rhs(M.n, nrhs, np.random.default_rng(17))
    Bt = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    X = torch.full_like(Bt, float("nan"))
    S.sym_solve_multi_noalloc(s.h, nrhs, Bt, M.n, X, M.n)
    torch.cuda.synchronize()
    xn = X.cpu().numpy().T
    assert np.isfinite(xn).all()
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, xn) <= BERR_TOL
    s.close()


def test_noalloc_solve_needs_an_fp64_factor(torch_cuda):
    """A mixed-precision handle (FP32 factor, refined solve) is refused with SYM_ERR_STATE."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.laplace2d5(24, np.random.default_rng(19))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.factor(torch.from_numpy(M.Ax).cuda())
    B = torch.zeros((1, M.n), dtype=torch.float64, device="cuda")
    X = torch.zeros_like(B)
    with pytest.raises(S.SymError) as e:
        S.sym_solve_multi_noalloc(s.h, 1, B, M.n, X, M.n)
    assert e.value.code == S.SYM_ERR_STATE
    s.close()
