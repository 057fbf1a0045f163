"""Pins of the CPU FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: closed forms, textbook or
library routines (numpy's dense Cholesky and eigensolver), brute-force elimination on tiny
inputs, and the definitions the paper gives (etree, Eq. (1), the supernode rule).
"""
import numpy as np
import pytest

import oracle
import workloads as w


def dense_of(M):
    return w.csc_to_dense(M)


def permuted_dense(M, perm):
    A = dense_of(M)
    return A[np.ix_(perm, perm)]


def brute_fill(C):
    """Boolean Gaussian elimination on a dense bitmap: the exact pattern of L (no cancellation)."""
    n = C.shape[0]
    G = C != 0
    for k in range(n):
        rows = np.nonzero(G[k + 1:, k])[0] + k + 1
        for i in rows:
            G[i, rows] = True
            G[rows, i] = True
    return np.tril(G)


def oracle_pattern(o):
    n = o.n
    P = np.zeros((n, n), dtype=bool)
    for j in range(n):
        P[o.Li[o.Lp[j]:o.Lp[j + 1]], j] = True
    return P


def tridiag(n, d=2.0, e=-1.0):
    u = np.arange(n - 1)
    Ap, Ai, Ax = w.lower_csc(n, u, u + 1, np.full(n - 1, e), np.full(n, d))
    return w.Matrix(n, Ap, Ai, Ax)


# ---------------------------------------------------------------------------------------------
# Numeric factor

@pytest.mark.parametrize("n,density,seed", [(5, 1.0, 0), (8, 0.5, 1), (12, 0.3, 2), (12, 1.0, 3),
                                            (10, 0.2, 4)])
def test_factor_matches_dense_cholesky(n, density, seed):
    rng = np.random.default_rng(seed)
    M = w.random_spd_pattern(n, density, rng)
    perm = rng.permutation(n).astype(np.int32)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, perm)
    assert o.factor(M.Ax) == 0
    C = permuted_dense(M, o.perm)
    Lref = np.linalg.cholesky(C)
    L = o.L_dense()
    assert np.abs(L - Lref).max() <= 1e-14 * np.abs(Lref).max()
    # the stored pattern covers every nonzero of the dense factor
    assert np.all((np.abs(Lref) > 1e-300) <= (L != 0) | (np.abs(Lref) < 1e-14))


def test_laplace1d_closed_form():
    """tridiag(-1, 2, -1): L_kk = sqrt((k+1)/k), L_{k+1,k} = -sqrt(k/(k+1)) (1-based k)."""
    n = 50
    M = tridiag(n)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, None)
    assert np.array_equal(o.perm, np.arange(n))  # a path etree postorders to itself
    assert o.factor(M.Ax) == 0
    L = o.L_dense()
    k = np.arange(1, n + 1, dtype=np.float64)
    assert np.allclose(np.diag(L), np.sqrt((k + 1) / k), rtol=1e-15, atol=0)
    assert np.allclose(np.diag(L, -1), -np.sqrt(k[:-1] / (k[:-1] + 1)), rtol=1e-15, atol=0)


def test_leading_block_factor_is_exact():
    """Stopping after k rows gives the Cholesky factor of the leading k x k block."""
    rng = np.random.default_rng(8)
    M = w.random_spd_pattern(40, 0.2, rng)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, None)
    o.factor(M.Ax, kmax=17)
    C = permuted_dense(M, o.perm)
    Lref = np.linalg.cholesky(C[:17, :17])
    L = o.L_dense()[:17, :17]
    assert np.abs(L - Lref).max() <= 1e-14 * np.abs(Lref).max()


def test_not_spd_first_column():
    """The first non-positive leading minor (numpy's eigvalsh of the leading blocks) is the
    column the oracle reports."""
    rng = np.random.default_rng(4)
    for trial in range(10):
        M = w.random_spd_pattern(15, 0.4, rng)
        Ax = M.Ax.copy()
        j = int(rng.integers(0, 15))
        Ax[M.Ap[j]] = -Ax[M.Ap[j]]
        o = oracle.Oracle(M.n, M.Ap, M.Ai, None)
        rc = o.factor(Ax)
        C = permuted_dense(w.Matrix(M.n, M.Ap, M.Ai, Ax), o.perm)
        first_bad = next(k for k in range(15) if np.linalg.eigvalsh(C[:k + 1, :k + 1]).min() <= 0)
        assert rc == oracle.ERR_NOT_SPD
        assert o.err_col == first_bad


def test_solve_and_backward_error():
    rng = np.random.default_rng(3)
    M = w.laplace2d5(20, rng)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    o.factor(M.Ax)
    A = dense_of(M)
    xstar = rng.standard_normal((M.n, 2))
    B = A @ xstar
    X = o.solve(B)
    assert np.abs(X - xstar).max() <= 1e-12 * np.abs(xstar).max()
    assert np.allclose(X, np.linalg.solve(A, B), rtol=1e-12, atol=1e-12)
    eta = oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X)
    assert eta <= 1e-15
    # the definition ||b - Ax||_inf / (||A||_inf ||x||_inf + ||b||_inf), max over columns, on a
    # perturbed solution whose residual is far above rounding
    X2 = X + 1e-6 * rng.standard_normal(X.shape)
    r = B - A @ X2
    ref = max(np.abs(r[:, c]).max() / (np.abs(A).sum(1).max() * np.abs(X2[:, c]).max() + np.abs(B[:, c]).max())
              for c in range(2))
    assert oracle.backward_error(M.n, M.Ap, M.Ai, M.Ax, B, X2) == pytest.approx(ref, rel=1e-9)


def test_factor_residual_definition():
    rng = np.random.default_rng(6)
    M = w.random_spd_pattern(30, 0.2, rng)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, None)
    o.factor(M.Ax)
    C = permuted_dense(M, o.perm)
    L = o.L_dense()
    ref = np.linalg.norm(L @ L.T - C) / np.linalg.norm(C)
    assert o.factor_residual() == pytest.approx(ref, rel=1e-3, abs=1e-17)
    # a planted error of known size is measured exactly
    Lx = o.Lx.copy()
    Lx[o.Lp[3]] += 1e-3
    L2 = L.copy()
    L2[3, 3] += 1e-3
    ref2 = np.linalg.norm(L2 @ L2.T - C) / np.linalg.norm(C)
    assert o.factor_residual_with(M.Ax, Lx) == pytest.approx(ref2, rel=1e-9)


def test_cfg1_is_spd_and_factors():
    """The 64x64 5-point workload (diagonal 4+U(0,0.1), off-diagonal -U(0.9,1.1)) is not
    diagonally dominant by construction; check seed 0 is SPD with a dense eigensolver."""
    M = w.cfg("laplace2d5_64")
    lam = np.linalg.eigvalsh(dense_of(M))
    assert lam.min() > 0
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.factor(M.Ax) == 0
    assert o.factor_residual() <= 1e-15


# ---------------------------------------------------------------------------------------------
# Symbolic structure

@pytest.mark.parametrize("n,density,seed", [(6, 0.4, 0), (20, 0.15, 1), (40, 0.08, 2), (64, 0.05, 3),
                                            (64, 0.02, 4), (30, 0.5, 5)])
def test_pattern_and_etree_brute_force(n, density, seed):
    rng = np.random.default_rng(seed)
    M = w.random_spd_pattern(n, density, rng)
    perm = rng.permutation(n).astype(np.int32)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, perm)
    C = permuted_dense(M, o.perm)
    G = brute_fill(C)
    assert np.array_equal(oracle_pattern(o), G)
    assert np.array_equal(o.colcount, G.sum(0))
    for j in range(n):
        below = np.nonzero(G[j + 1:, j])[0]
        assert o.parent[j] == (j + 1 + below[0] if below.size else -1)  # min{i > j : L_ij != 0}
        assert o.parent[j] == -1 or o.parent[j] > j
    assert o.row_patterns_agree()


def test_postorder_properties():
    rng = np.random.default_rng(12)
    M = w.random_spd_pattern(60, 0.05, rng)
    perm0 = rng.permutation(60).astype(np.int32)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, perm0)
    assert np.array_equal(np.sort(o.perm), np.arange(60))
    # every subtree is a contiguous range ending at its root
    n = o.n
    size = np.ones(n, dtype=int)
    for j in range(n):
        if o.parent[j] >= 0:
            size[o.parent[j]] += size[j]
    for j in range(n):
        desc = {j}
        for k in range(j - 1, -1, -1):
            if o.parent[k] in desc:
                desc.add(k)
        assert desc == set(range(j - size[j] + 1, j + 1))
    # fill is invariant under the postorder: same count as the given order without it
    G0 = brute_fill(permuted_dense(M, perm0))
    assert o.nnzL == G0.sum()


def test_special_cases():
    n = 30
    # tridiagonal: path etree, c_j = 2 (last 1), flops 4(n-1)+1
    T = tridiag(n)
    o = oracle.Oracle(T.n, T.Ap, T.Ai, None)
    assert np.array_equal(o.parent, np.r_[np.arange(1, n), -1])
    assert np.array_equal(o.colcount, np.r_[np.full(n - 1, 2), 1])
    assert o.flops_exact == 4 * (n - 1) + 1
    # dense: one fundamental supernode, c_j = n - j, flops n(n+1)(2n+1)/6
    D = w.random_spd_pattern(n, 1.0, np.random.default_rng(0))
    o = oracle.Oracle(D.n, D.Ap, D.Ai, None, relax=None)
    assert np.array_equal(o.fsn, [0, n])
    assert np.array_equal(o.colcount, n - np.arange(n))
    assert o.flops_exact == n * (n + 1) * (2 * n + 1) // 6
    # diagonal: n singleton roots, all at level 0
    Ap = np.arange(n + 1, dtype=np.int64)
    Ai = np.arange(n, dtype=np.int32)
    o = oracle.Oracle(n, Ap, Ai, None)
    assert np.all(o.parent == -1) and np.all(o.level == 0) and o.nsn == n
    # arrowhead (dense last row and column): star etree, no fill
    u = np.arange(n - 1)
    Ap, Ai, Ax = w.lower_csc(n, u, np.full(n - 1, n - 1), -np.ones(n - 1), np.full(n, float(n)))
    o = oracle.Oracle(n, Ap, Ai, None, relax=None)
    assert np.array_equal(o.parent, np.r_[np.full(n - 1, n - 1), -1])
    assert o.nnzL == Ap[-1]
    # k x k 5-point grid in natural order: the factor fills the envelope (row i starts at its
    # first nonzero column f_i: i-k for i >= k, i-1 in the first grid row), so
    # c_j = j + 3 for j <= k-2 and min(k, n-1-j) + 1 for j >= k-1
    for k in (3, 7, 10):
        u, v, _ = w.grid_edges((k, k), "star")
        Ap, Ai, Ax = w.lower_csc(k * k, u, v, -np.ones(u.size), np.full(k * k, 4.0))
        o = oracle.Oracle(k * k, Ap, Ai, None)
        nn = k * k
        j = np.arange(nn)
        ref = np.where(j <= k - 2, j + 3, np.minimum(k, nn - 1 - j) + 1)
        assert np.array_equal(o.colcount, ref)


def test_fundamental_supernode_rule():
    """Inside a fundamental supernode L_{j-1} minus {j-1} equals L_j, each column is the only
    child of the next, and the supernodes are maximal under the rule."""
    rng = np.random.default_rng(21)
    for trial in range(6):
        M = w.random_spd_pattern(50, 0.06 + 0.03 * trial, rng)
        o = oracle.Oracle(M.n, M.Ap, M.Ai, None, relax=None)
        P = oracle_pattern(o)
        nchild = np.bincount(o.parent[o.parent >= 0], minlength=o.n)
        starts = set(o.fsn[:-1].tolist())
        for j in range(1, o.n):
            same = np.array_equal(P[j + 1:, j - 1], P[j + 1:, j]) and P[j, j - 1]
            rule = o.parent[j - 1] == j and nchild[j] == 1 and o.colcount[j - 1] == o.colcount[j] + 1
            # inside a fundamental supernode the structure nests (L_{j-1} minus {j-1} = L_j); the
            # rule is exactly that nesting plus "j-1 is the only child of j"
            assert (not rule) or same
            assert rule == (same and nchild[j] == 1)
            assert (j not in starts) == rule
        assert o.nsn == len(o.fsn) - 1  # no amalgamation requested


def _storage(rows_count, nc):
    return nc * rows_count - nc * (nc - 1) // 2


def test_amalgamation_rule_brute_force():
    """Re-derive the zero counts of every amalgamated supernode from the dense filled pattern and
    check the partition is a fixed point of the rule."""
    relax = oracle.DEFAULT_RELAX
    rng = np.random.default_rng(31)
    for trial in range(5):
        M = w.random_spd_pattern(60, 0.04 + 0.02 * trial, rng)
        o = oracle.Oracle(M.n, M.Ap, M.Ai, rng.permutation(60).astype(np.int32), relax=relax)
        P = oracle_pattern(o)
        fund = set(o.fsn.tolist())
        # each amalgamated supernode is a union of consecutive fundamental ones
        assert set(o.sn.tolist()) <= fund
        sets = []
        for J in range(o.nsn):
            f, l = o.sn[J], o.sn[J + 1]
            rows = np.nonzero(P[:, f:l].any(1))[0]
            assert np.array_equal(rows, o.sri[o.srp[J]:o.srp[J + 1]])
            total = _storage(rows.size, l - f)
            true = int(P[:, f:l].sum())
            sets.append((f, l, rows, total, true))
        # fixed point: no adjacent pair that the rule allows to merge is left unmerged
        for J in range(o.nsn - 1):
            f, l, rows, _, true1 = sets[J]
            f2, l2, rows2, _, true2 = sets[J + 1]
            if o.parent[l - 1] != l:
                continue
            mrows = np.union1d(rows, rows2)
            nc = l2 - f
            total = _storage(mrows.size, nc)
            z = total - (true1 + true2)
            ok = (nc <= relax[0] or (nc <= relax[1] and z * 1000 <= relax[3] * total) or
                  (nc <= relax[2] and z * 1000 <= relax[4] * total) or z * 1000 <= relax[5] * total)
            assert not ok, (J, nc, z, total)


def _rule(relax, nc, z, total):
    """The amalgamation rule as stated in the library's interface (sym_options)."""
    return (nc <= relax[0] or (nc <= relax[1] and z * 1000 <= relax[3] * total) or
            (nc <= relax[2] and z * 1000 <= relax[4] * total) or z * 1000 <= relax[5] * total)


def _replay_merges(o, P, relax):
    """Apply the oracle's logged merges to its fundamental supernodes in log order. For each
    merge, check that the two supernodes are adjacent and eligible (the absorbed one's last
    column has the other's first column as etree parent), and re-derive from the dense filled
    pattern P the merged column count, the trapezoid size and its explicit zeros. Returns the
    merges the rule does not accept and the partition the replay ends with."""
    n = o.n
    starts = [int(x) for x in o.fsn[:-1]]
    rejected = []
    for fS, fP in o.merges.tolist():
        i = starts.index(fS)
        assert i + 1 < len(starts) and starts[i + 1] == fP, "merge of non-adjacent supernodes"
        assert o.parent[fP - 1] == fP, "merge of a supernode whose last column's parent is elsewhere"
        end = starts[i + 2] if i + 2 < len(starts) else n
        rows = np.nonzero(P[:, fS:end].any(1))[0]
        nc = end - fS
        total = _storage(rows.size, nc)
        z = total - int(P[:, fS:end].sum())
        if not _rule(relax, nc, z, total):
            rejected.append((fS, fP, nc, z, total))
        del starts[i + 1]
    return rejected, starts + [n]


def _amalgamation_cases():
    rng = np.random.default_rng(53)
    cases = []
    for trial in range(6):
        M = w.random_spd_pattern(70, 0.03 + 0.015 * trial, rng)
        cases.append((M, rng.permutation(70).astype(np.int32)))
    for side in (9, 13):
        M = w.laplace2d5(side, rng)
        cases.append((M, M.perm))
    M = w.conduct3d(6, rng, "box")
    cases.append((M, M.perm))
    return cases


def test_amalgamation_merges_replay():
    """Accept side of the amalgamation rule: every merge the oracle made, replayed from the
    fundamental supernodes in its order, is one the rule accepts on the zero counts of the dense
    filled pattern (brute-force elimination), and the replay ends at the oracle's partition.
    With the fixed-point test below (reject side), a wrong merge in either direction fails."""
    relax = oracle.DEFAULT_RELAX
    total_merges = 0
    for M, perm in _amalgamation_cases():
        o = oracle.Oracle(M.n, M.Ap, M.Ai, perm, relax=relax)
        P = brute_fill(permuted_dense(M, o.perm))
        assert np.array_equal(P, oracle_pattern(o))
        rejected, part = _replay_merges(o, P, relax)
        assert rejected == []
        assert np.array_equal(np.array(part), o.sn)
        total_merges += len(o.merges)
    assert total_merges > 50  # the cases exercise the rule, not just fundamental supernodes


@pytest.mark.parametrize("plant", ["ORC_PLANT_DROP_Z_CLAUSE", "ORC_PLANT_OR_FOR_AND"])
def test_amalgamation_planted_over_merge_is_caught(plant):
    """Copies of the oracle compiled with a wrong rule (a zero-fraction clause dropped, or || for
    &&) make merges that the replay flags."""
    relax = oracle.DEFAULT_RELAX
    caught = 0
    for M, perm in _amalgamation_cases():
        o = oracle.Oracle(M.n, M.Ap, M.Ai, perm, relax=relax, defines=(plant,))
        P = brute_fill(permuted_dense(M, o.perm))
        rejected, _ = _replay_merges(o, P, relax)
        caught += len(rejected)
    assert caught > 0


def test_amalgamation_limits():
    """Closed forms of the rule's extremes. Column thresholds of n accept every eligible merge, so
    supernodes end exactly where the next column is not the etree parent of the last one. All
    thresholds zero accept only merges that add no explicit zero."""
    rng = np.random.default_rng(59)
    for M, perm in _amalgamation_cases():
        n = M.n
        o = oracle.Oracle(M.n, M.Ap, M.Ai, perm, relax=(n, n, n, 0, 0, 0))
        breaks = [0] + [j for j in range(1, n) if o.parent[j - 1] != j] + [n]
        assert np.array_equal(o.sn, np.array(breaks))
        o0 = oracle.Oracle(M.n, M.Ap, M.Ai, perm, relax=(0, 0, 0, 0, 0, 0))
        P = brute_fill(permuted_dense(M, o0.perm))
        for f, l in zip(o0.sn[:-1], o0.sn[1:]):
            rows = np.nonzero(P[:, f:l].any(1))[0]
            assert _storage(rows.size, l - f) == int(P[:, f:l].sum())  # no explicit zeros
        rejected, part = _replay_merges(o0, P, (0, 0, 0, 0, 0, 0))
        assert rejected == [] and np.array_equal(np.array(part), o0.sn)


def test_row_patterns_check_rejects_corrupted_structure():
    """The etree row-walk check returns a mismatch when the etree or a column pattern is wrong
    (the mistake is planted in the oracle's own arrays, on the CPU)."""
    import ctypes as ct
    rng = np.random.default_rng(61)
    M = w.laplace2d5(10, rng)
    for what in ("parent", "Li"):
        o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
        assert o.row_patterns_agree()
        if what == "parent":
            # re-hang a column with a non-root parent onto a later column
            j = int(np.nonzero(o.parent[:-2] >= 0)[0][3])
            arr = (ct.c_int32 * o.n).from_address(o._lib.orc_parent(o._h))
            arr[j] = min(int(o.parent[j]) + 1, o.n - 1) if o.parent[j] + 1 < o.n else int(o.parent[j]) - 1
        else:
            # move one off-diagonal row index of a column to another row below the diagonal
            j = next(c for c in range(o.n) if o.Lp[c + 1] - o.Lp[c] >= 3)
            arr = (ct.c_int32 * int(o.nnzL)).from_address(o._lib.orc_Li(o._h))
            p = int(o.Lp[j]) + 1
            free_rows = np.setdiff1d(np.arange(j + 1, o.n), o.Li[o.Lp[j]:o.Lp[j + 1]])
            arr[p] = int(free_rows[0])
        assert not o.row_patterns_agree(), what


def test_descendants_maps_levels():
    rng = np.random.default_rng(41)
    M = w.laplace2d5(18, rng)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm, want_rel=True)
    ns = o.nsn
    rows = [o.sri[o.srp[J]:o.srp[J + 1]] for J in range(ns)]
    for J in range(ns):
        f, l = o.sn[J], o.sn[J + 1]
        ref = [K for K in range(J) if np.any((rows[K] >= f) & (rows[K] < l))]
        got = o.dk[o.dp[J]:o.dp[J + 1]].tolist()
        assert got == ref
        for q in range(o.dp[J], o.dp[J + 1]):
            K = o.dk[q]
            r0 = int(o.dr0[q])
            assert rows[K][r0] >= f and (r0 == 0 or rows[K][r0 - 1] < f)
            assert o.dnin[q] == int(np.sum((rows[K] >= f) & (rows[K] < l)))
            rel = o.rel[o.relp[q]:o.relp[q + 1]]
            assert np.array_equal(rows[J][rel], rows[K][r0:])  # round trip
    # levels: leaves 0, else 1 + max over children; lists ascending within a level
    for J in range(ns):
        kids = np.nonzero(o.sparent == J)[0]
        assert o.level[J] == (0 if kids.size == 0 else 1 + o.level[kids].max())
    for l in range(o.nlev):
        s = o.lvl[o.lvp[l]:o.lvp[l + 1]]
        assert np.all(np.diff(s) > 0) and np.all(o.level[s] == l)


def test_sizing_cfg1():
    """Sizing (not a parity target): with the nested-dissection rule the 64x64 5-point grid
    gives nnz(L) = 89,164 and 3.73e6 flops."""
    M = w.cfg("laplace2d5_64")
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    assert o.nnzL == 89164
    assert abs(o.flops - 3.73e6) / 3.73e6 < 0.01


def test_validation():
    n = 3
    good_Ap = np.array([0, 2, 3, 4])
    good_Ai = np.array([0, 2, 1, 2])
    assert oracle.validate(n, good_Ap, good_Ai) == 0
    assert oracle.validate(n, good_Ap, np.array([2, 0, 1, 2])) == oracle.ERR_INVALID  # diag not first
    assert oracle.validate(n, np.array([0, 2, 2, 3]), np.array([0, 2, 2])) == oracle.ERR_INVALID  # no diag
    assert oracle.validate(n, good_Ap, np.array([0, 3, 1, 2])) == oracle.ERR_INVALID  # out of range
    assert oracle.validate(n, np.array([0, 3, 4, 5]), np.array([0, 2, 2, 1, 2])) == oracle.ERR_INVALID  # dup
    with pytest.raises(ValueError):
        oracle.Oracle(n, good_Ap, good_Ai, np.array([0, 0, 1], dtype=np.int32))  # not a permutation


def test_planted_mistakes_are_caught():
    """A wrong sign, a dropped term or a transposed operand in a factor is visible in the checks
    the parity tests use (factor residual and backward error)."""
    rng = np.random.default_rng(2)
    M = w.laplace2d5(12, rng)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    o.factor(M.Ax)
    base = o.factor_residual_with(M.Ax, o.Lx)
    assert base < 1e-15
    off = np.setdiff1d(np.arange(o.nnzL), o.Lp[:-1])
    wrong_sign = o.Lx.copy()
    wrong_sign[off[5]] *= -1
    dropped = o.Lx.copy()
    dropped[off[10]] = 0.0
    for bad in (wrong_sign, dropped):
        assert o.factor_residual_with(M.Ax, bad) > 1e-4


def test_reach_set_brute_force_and_topological_order():
    """Reach_L(beta) equals the closure of beta under the edges j -> i (L_ij != 0), computed by
    boolean matrix powers, and the returned order is topological (every edge goes forward)."""
    rng = np.random.default_rng(51)
    for trial in range(6):
        M = w.random_spd_pattern(60, 0.04 + 0.02 * trial, rng)
        o = oracle.Oracle(M.n, M.Ap, M.Ai, rng.permutation(60).astype(np.int32))
        G = oracle_pattern(o).astype(np.int64)
        np.fill_diagonal(G, 0)
        beta = rng.choice(60, size=3, replace=False).astype(np.int32)
        v = np.zeros(60, dtype=np.int64)
        v[beta] = 1
        for _ in range(60):  # closure under x -> G x (column j reaches rows of column j)
            v = np.minimum(1, v + G @ v)
        r = o.reach(beta)
        assert set(r.tolist()) == set(np.nonzero(v)[0].tolist())
        pos = {int(j): t for t, j in enumerate(r)}
        for j in r:
            for i in np.nonzero(G[:, j])[0]:
                assert pos[int(i)] > pos[int(j)]


def test_sparse_lower_solve_matches_dense_triangular_solve():
    rng = np.random.default_rng(52)
    M = w.laplace2d5(20, rng)
    o = oracle.Oracle(M.n, M.Ap, M.Ai, M.perm)
    o.factor(M.Ax)
    L = o.L_dense()
    beta = rng.choice(M.n, size=4, replace=False).astype(np.int32)
    bvals = rng.standard_normal(4)
    r, x = o.sparse_lsolve(beta, bvals)
    b = np.zeros(M.n)
    b[beta] = bvals
    ref = np.linalg.solve(L, b)
    assert np.abs(x - ref).max() <= 1e-13 * np.abs(ref).max()
    outside = np.setdiff1d(np.arange(M.n), r)
    assert np.all(ref[outside] == 0.0)  # the solution vanishes outside the reach set


def test_mlp_gradient_matches_finite_differences():
    """The reference MLP's chain-rule gradient agrees with central differences of its loss."""
    from oracle import mlp
    rng = np.random.default_rng(61)
    nin, h, N = 5, 7, 23
    theta = rng.standard_normal(mlp.nparams(nin, h)) * 0.5
    X = rng.standard_normal((N, nin))
    t = rng.standard_normal(N)
    g = mlp.gradient(theta, X, t, nin, h)
    eps = 1e-6
    fd = np.empty_like(theta)
    for i in range(theta.size):
        tp, tm = theta.copy(), theta.copy()
        tp[i] += eps
        tm[i] -= eps
        fd[i] = (mlp.loss(tp, X, t, nin, h) - mlp.loss(tm, X, t, nin, h)) / (2 * eps)
    assert np.abs(g - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())
    # a planted mistake (dropping the ReLU mask of the first layer) is detected
    W1, b1, W2, b2, w3, b3 = mlp.unpack(theta, nin, h)
    y, (Xc, z1, h1, z2, h2) = mlp.forward(theta, X, nin, h)
    dy = 2.0 * (y - t) / N
    dz2 = np.outer(dy, w3) * (z2 > 0)
    wrong_dW1 = (dz2 @ W2).T @ X  # no mask
    assert np.abs(wrong_dW1.ravel() - g[:h * nin]).max() > 1e-6 or np.all(z1 > 0)
