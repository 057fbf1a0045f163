"""GPU tests of the tensor-core (tcgen05) path of the FP32 factor.

* The layout check: one kind::tf32 tile product through the library's operand layout and
  descriptors reproduces A B^T exactly on integer data (every product and partial sum is an
  integer below 2^11, exact in TF32 inputs and FP32 accumulation).
* The FP32 factor with tensor-core updates against the oracle's FP64 factor. Each operand x is
  split into two TF32 values, hi = RN(x) and lo = RN(x - hi) with 11 significant bits each, so
  |x - hi - lo| <= 2^-22 |x| and a product a b is formed with relative error <= 2^-21 (all four
  partial products are exact), against 2^-24 for an FP32 multiply; the tensor core's sums run
  over at most 64 MMAs of K = 8 before they are added in FP32. The backward-stable measure scales
  with that unit: ||L L^T - A||_F / ||A||_F <= MIXED_FACTOR_TOL = 1e-6 for the SIMT factor and
  8 times that, TC_FACTOR_TOL = 8e-6, for the split. The entry-wise difference from the exact
  factor is a forward error, about kappa(A) u, and kappa reaches ~1e4 on these 3D grids with
  their 1e-3 diagonal shift; ENTRY_RTOL = 5e-4 of max|L| bounds both factors. Both must refine
  to the FP64 backward-error bound, and they agree with each other to the same entry bound.
"""
import numpy as np
import pytest

import oracle
import workloads as w
from tests.helpers import exports, panels_on_pattern

pytestmark = pytest.mark.gpu

ENTRY_RTOL = 5e-4
MIXED_FACTOR_TOL = 1e-6
TC_FACTOR_TOL = 8e-6
REFINED_BERR = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def test_tc_tile_product_layout(torch_cuda):
    import paper_1705_06575_gb300 as S
    rng = np.random.default_rng(11)
    A = rng.integers(-8, 9, size=(128, 32)).astype(np.float32)
    B = rng.integers(-8, 9, size=(64, 32)).astype(np.float32)
    D = S.sym_tc_probe(A, B)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.array_equal(D.astype(np.float64), ref)


def test_tc_tile_product_split_precision(torch_cuda):
    """Values with all 24 significand bits: the hi/lo split the update uses, done here on the host
    (round to 10 stored bits, nearest), multiplied as [A_hi; A_lo] (B_hi + B_lo)^T on the tensor
    cores, reproduces A B^T to FP32 accuracy."""
    import paper_1705_06575_gb300 as S
    rng = np.random.default_rng(12)

    def tf32(x):
        b = x.astype(np.float32).view(np.uint32).astype(np.uint64)
        b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)  # round half away from zero on |x|
        return b.view(np.float32)

    A = rng.standard_normal((64, 32)).astype(np.float32)
    B = rng.standard_normal((64, 32)).astype(np.float32)
    Ah = tf32(A)
    Al = tf32(A - Ah)
    Bh = tf32(B)
    Bl = tf32(B - Bh)
    Dh = S.sym_tc_probe(np.vstack([Ah, Al]), Bh)
    Dl = S.sym_tc_probe(np.vstack([Ah, Al]), Bl)
    C = (Dh[:64] + Dh[64:]).astype(np.float64) + (Dl[:64] + Dl[64:]).astype(np.float64)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    scale = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    # a dropped partial product would leave ~2^-12 |a||b|; FP32 accumulation of 32 terms ~32 u32
    assert np.all(np.abs(C - ref) <= 1e-5 * scale)


@pytest.mark.parametrize("maker", [
    lambda: w.conduct3d(20, np.random.default_rng(21), "star"),   # separators of 400 columns
    lambda: w.conduct3d(12, np.random.default_rng(22), "box"),    # dense 27-point separators
    lambda: w.dd2d9(40, np.random.default_rng(23)),               # 2D 9-point
])
def test_tc_factor_against_oracle(torch_cuda, maker):
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = maker()
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax) == 0
    Ax = torch.from_numpy(M.Ax).cuda()
    got, err = {}, {}
    bounds = {"tc": TC_FACTOR_TOL, "simt": MIXED_FACTOR_TOL}
    for name, flags in (("tc", 0), ("simt", S.SYM_FLAG_NO_TENSOR_CORES)):
        s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed", flags=flags)
        s.factor(Ax)
        vals, outside = panels_on_pattern(exports(s), s.factor_panels(), o.Lp, o.Li)
        assert outside == 0.0
        B = w.rhs(M.n, 2, np.random.default_rng(5))
        X = s.solve(torch.from_numpy(np.ascontiguousarray(B.T)).cuda()).cpu().numpy().T
        err[name] = (np.abs(vals - o.Lx).max() / np.abs(o.Lx).max(), o.factor_residual_with(M.Ax, vals),
                     oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X), s.refinement_info()[0])
        got[name] = vals
        s.close()
    print(err)
    for name, (ent, res, berr, _) in err.items():
        assert ent <= ENTRY_RTOL, name
        assert res <= bounds[name], name
        assert berr <= REFINED_BERR, name
    # the two FP32 factors differ by rounding only
    assert np.abs(got["tc"] - got["simt"]).max() <= ENTRY_RTOL * np.abs(o.Lx).max()


def test_tc_factor_is_deterministic(torch_cuda):
    """Every tile's entries accumulate in one fixed order on the tensor cores: a repeated
    factorization gives the same bits."""
    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.conduct3d(16, np.random.default_rng(31), "star")
    Ax = torch.from_numpy(M.Ax).cuda()
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    s.factor(Ax)
    L1 = s.factor_panels().copy()
    s.factor(Ax)
    L2 = s.factor_panels()
    assert np.array_equal(L1, L2)
    s.close()


def test_tensor_core_wait_runs_out_and_handle_recovers(torch_cuda):
    """Failure path of the bounded waits: with the MMAs withheld (nothing ever arrives on the
    update kernel's mbarriers) and a 20 us limit, every wait runs out, the kernel frees its tensor
    memory and the factorization returns SYM_ERR_TIMEOUT quickly; the solve is then refused, and
    the same handle factors and solves normally once the limit is restored."""
    import time

    torch = torch_cuda
    import paper_1705_06575_gb300 as S
    M = w.conduct3d(16, np.random.default_rng(12), "star")
    s = S.Solver(M.n, M.Ap, M.Ai, M.perm, precision="mixed")
    assert max(np.diff(s.export("super"))) > 64  # 64-wide tiles: the tensor-core update runs
    Ax = torch.from_numpy(M.Ax).cuda()
    s.factor(Ax)
    S.sym_set_tc_wait(s.h, 20_000, 1)
    t0 = time.perf_counter()
    with pytest.raises(S.SymError) as e:
        s.factor(Ax)
    assert e.value.code == S.SYM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    b = torch.from_numpy(w.rhs(M.n, 1, np.random.default_rng(1))[:, 0]).cuda()
    with pytest.raises(S.SymError) as e2:
        s.solve(b)
    assert e2.value.code == S.SYM_ERR_STATE
    S.sym_set_tc_wait(s.h, 1_000_000_000, 0)
    s.set_refinement(1e-12, 100)
    s.factor(Ax)
    x = s.solve(b)
    torch.cuda.synchronize()
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, b.cpu().numpy(), x.cpu().numpy()) <= 1e-12
