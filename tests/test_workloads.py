"""CPU checks of the seeded synthetic inputs: each generator produces the recipe it states (value
ranges, stencil, diagonal rule), a valid lower-triangle CSC, an ordering that is a permutation,
and the same matrix for the same seed."""
import numpy as np
import pytest

import workloads as w


def full(M):
    A = w.csc_to_dense(M)
    assert np.array_equal(A, A.T)
    return A


def check_csc(M):
    assert M.Ap[0] == 0 and M.Ap[-1] == M.Ai.size == M.Ax.size
    for j in range(M.n):
        rows = M.Ai[M.Ap[j]:M.Ap[j + 1]]
        assert rows[0] == j and np.all(np.diff(rows) > 0)  # diagonal first, rows increasing


def test_laplace2d5_recipe():
    M = w.laplace2d5(12, np.random.default_rng(0))
    check_csc(M)
    A = full(M)
    d = np.diag(A)
    off = A - np.diag(d)
    assert np.all((d >= 4.0) & (d <= 4.1))
    nz = off[off != 0]
    assert np.all((nz >= -1.1) & (nz <= -0.9))
    deg = (off != 0).sum(1)
    assert deg.max() == 4 and deg.min() == 2  # 5-point stencil: corners have two neighbours
    assert np.array_equal(np.sort(M.perm), np.arange(M.n))


@pytest.mark.parametrize("kind,maxdeg", [("star", 6), ("box", 26)])
def test_conduct3d_recipe(kind, maxdeg):
    M = w.conduct3d(5, np.random.default_rng(1), kind)
    check_csc(M)
    A = full(M)
    off = A - np.diag(np.diag(A))
    nz = off[off != 0]
    assert np.all((nz >= -2.0) & (nz <= -0.5))
    assert (off != 0).sum(1).max() == maxdeg
    # A_ii = sum of incident conductivities + 1e-3: every row sums to the shift
    assert np.allclose(A.sum(1), 1e-3, rtol=0, atol=1e-12)
    assert np.array_equal(np.sort(M.perm), np.arange(M.n))


def test_dd2d9_recipe():
    M = w.dd2d9(9, np.random.default_rng(2))
    check_csc(M)
    A = full(M)
    d = np.diag(A)
    off = A - np.diag(d)
    assert (off != 0).sum(1).max() == 8
    assert np.allclose(d, 1.05 * np.abs(off).sum(1), rtol=1e-14, atol=0)


def test_vector3d27_is_spd_with_its_jumps():
    M = w.vector3d27(4, np.random.default_rng(3), sub=2)
    check_csc(M)
    A = full(M)
    assert M.n == 3 * 4 ** 3
    ev = np.linalg.eigvalsh(A)
    assert ev[0] > 0
    # the shift term is 1e-3 c per node, c in {1, 1e2, 1e4}: the spread of the diagonal reflects it
    d = np.diag(A)
    assert d.max() / d.min() > 1e3
    # dofs of one node stay consecutive in the ordering
    p = M.perm.reshape(-1, 3)
    assert np.all(p[:, 1] == p[:, 0] + 1) and np.all(p[:, 2] == p[:, 0] + 2)


def test_seeds_are_deterministic_and_distinct():
    a = w.cfg("conduct3d7_48")
    b = w.cfg("conduct3d7_48")
    assert np.array_equal(a.Ax, b.Ax) and np.array_equal(a.Ai, b.Ai)
    c = w.cfg("conduct3d7_48", matrix_index=1)
    assert np.array_equal(a.Ai, c.Ai) and not np.array_equal(a.Ax, c.Ax)


def test_same_pattern_batch_shares_the_pattern():
    M, vals = w.same_pattern_batch(lambda r: w.dd2d9(8, r), 5, 7)
    assert vals.shape == (5, M.nnz)
    assert np.array_equal(vals[0], M.Ax)
    assert len({tuple(v[:5]) for v in vals}) == 5


def test_block_diagonal_union_of_uneven_grids():
    mats, sides = w.uneven_grid_batch(4, np.random.default_rng(4), lo=5, hi=9)
    U = w.block_diagonal(mats)
    check_csc(U)
    assert U.n == sum(m.n for m in mats)
    assert np.array_equal(np.sort(U.perm), np.arange(U.n))
    # no entry couples two blocks
    off = 0
    for m in mats:
        for j in range(off, off + m.n):
            rows = U.Ai[U.Ap[j]:U.Ap[j + 1]]
            assert rows.min() >= off and rows.max() < off + m.n
        off += m.n
