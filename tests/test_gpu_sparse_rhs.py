"""GPU parity of the sparse right-hand-side forward solve over reach sets (VI-Prune + VS-Block)."""
import numpy as np
import pytest

import oracle
import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("maker,nb", [
    (lambda: w.cfg("laplace2d5_64"), 3),
    (lambda: w.cfg("laplace2d5_64"), 200),
    (lambda: w.conduct3d(16, np.random.default_rng(3), "star"), 8),
    (lambda: w.conduct3d(10, np.random.default_rng(4), "box"), 1),
    (lambda: w.random_spd_pattern(900, 0.006, np.random.default_rng(5)), 30),
])
def test_sparse_lower_solve_matches_oracle(torch_cuda, maker, nb):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = maker()
    rng = np.random.default_rng(nb + 1)
    bidx = rng.choice(M.n, size=nb, replace=False).astype(np.int32)
    bvals = rng.standard_normal(nb)
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    s.factor(torch.from_numpy(M.Ax).cuda())
    r = S.Reach(s.h, bidx)
    x = torch.full((r.size(),), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):  # the reach is reused: two solves in a row
        r.solve(torch.from_numpy(bvals).cuda(), x)
    torch.cuda.synchronize()
    xg = x.cpu().numpy()
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    o.factor(M.Ax)
    iperm = np.empty(M.n, dtype=np.int64)
    iperm[o.perm] = np.arange(M.n)
    reach, xo = o.sparse_lsolve(iperm[bidx].astype(np.int32), bvals)
    cols = r.export(0)
    assert np.array_equal(cols, np.sort(reach))
    ref = xo[cols]
    assert np.abs(xg - ref).max() <= 1e-12 * np.abs(ref).max()
    r.close()


def test_sparse_solve_after_refactorization(torch_cuda):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.laplace2d5(40, np.random.default_rng(9))
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm)
    bidx = np.array([5, 700, 1599], dtype=np.int32)
    s.factor(torch.from_numpy(M.Ax).cuda())
    r = S.Reach(s.h, bidx)
    Ax2 = M.Ax * 1.5
    s.factor(torch.from_numpy(Ax2).cuda())  # new values, same pattern: the reach stays valid
    x = torch.empty(r.size(), dtype=torch.float64, device="cuda")
    r.solve(torch.tensor([1.0, -2.0, 0.5], dtype=torch.float64, device="cuda"), x)
    torch.cuda.synchronize()
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    o.factor(Ax2)
    iperm = np.empty(M.n, dtype=np.int64)
    iperm[o.perm] = np.arange(M.n)
    reach, xo = o.sparse_lsolve(iperm[bidx].astype(np.int32), np.array([1.0, -2.0, 0.5]))
    ref = xo[r.export(0)]
    assert np.abs(x.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()
    r.close()
