"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This module generates matrices, right-hand sides and fill-reducing orderings. It holds none of the
factorization's arithmetic: no elimination tree, no fill, no supernodes, no numeric factor. Both
the CPU oracle and the CUDA path receive its output as plain arrays.

Storage convention (the input format of the factorization, Sec. 2.1 and Sec. 4.2 of the paper):
the lower triangle of a symmetric matrix in compressed sparse column form, 0-based, with
``Ap`` int64 column pointers (length n+1), ``Ai`` int32 row indices (strictly increasing within a
column, the diagonal first) and ``Ax`` float64 values.

Value recipes (the paper's SuiteSparse matrices are not available; these stand in for them):

* ``laplace2d5``: 2D 5-point grid, diagonal 4+U(0,0.1) per row, off-diagonal -U(0.9,1.1) per edge.
* ``conduct3d``: 3D 7- or 27-point grid, per-edge conductivity w~U(0.5,2.0), A_ij=-w,
  A_ii = sum of the incident w + shift (1e-3).
* ``dd2d9``: 2D 9-point grid, w~U(0.5,2.0), A_ij=-w, A_ii = 1.05 * sum_j |A_ij|.
* ``vector3d27``: 3 unknowns per node, 27-point coupling, A = sum_e c_e (e_i-e_j)(e_i-e_j)^T (x) B_e
  + 1e-3 diag(c) (x) I_3 with B_e = I_3 + d_e d_e^T, coefficient jumps 1/1e2/1e4 by subdomain.
* ``erdos_renyi``: random graph, off-diagonal -U(0.5,2.0), A_ii = f * sum_j |A_ij|, f~U(1.01,1.5).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "grid_edges", "nd_perm", "lower_csc", "laplace2d5", "conduct3d", "dd2d9", "vector3d27",
    "erdos_renyi", "rhs", "Matrix", "csc_to_dense", "random_spd_pattern", "cfg",
]


class Matrix:
    """Lower-triangular CSC matrix plus the ordering it should be factored with."""

    def __init__(self, n, Ap, Ai, Ax, perm=None, name=""):
        self.n = int(n)
        self.Ap = np.ascontiguousarray(Ap, dtype=np.int64)
        self.Ai = np.ascontiguousarray(Ai, dtype=np.int32)
        self.Ax = None if Ax is None else np.ascontiguousarray(Ax, dtype=np.float64)
        self.perm = None if perm is None else np.ascontiguousarray(perm, dtype=np.int32)
        self.name = name

    @property
    def nnz(self):
        return int(self.Ap[-1])


def grid_node_ids(dims):
    """Node id of each grid point, lexicographic with the first coordinate slowest."""
    return np.arange(int(np.prod(dims)), dtype=np.int64).reshape(dims)


def _offsets(ndim, kind):
    """Half of the stencil offsets (the lexicographically positive ones)."""
    if kind == "star":  # 5-point (2D) / 7-point (3D)
        offs = [tuple(1 if k == d else 0 for k in range(ndim)) for d in range(ndim)]
    elif kind == "box":  # 9-point (2D) / 27-point (3D)
        import itertools
        offs = []
        for o in itertools.product((-1, 0, 1), repeat=ndim):
            if any(o) and next(v for v in o if v != 0) > 0:
                offs.append(o)
    else:
        raise ValueError(kind)
    return offs


def grid_edges(dims, kind):
    """All undirected edges (i, j), i != j, of a star or box stencil on a grid.

    Returns two int64 arrays (u, v) and the unit direction of each edge (for vector problems).
    """
    dims = tuple(int(d) for d in dims)
    ids = grid_node_ids(dims)
    us, vs, dirs = [], [], []
    for off in _offsets(len(dims), kind):
        src = tuple(slice(max(0, -o), d - max(0, o)) for o, d in zip(off, dims))
        dst = tuple(slice(max(0, o), d - max(0, -o)) for o, d in zip(off, dims))
        u = ids[src].ravel()
        v = ids[dst].ravel()
        us.append(u)
        vs.append(v)
        d = np.asarray(off, dtype=np.float64)
        dirs.append(np.broadcast_to(d / np.linalg.norm(d), (u.size, len(dims))))
    return np.concatenate(us), np.concatenate(vs), np.concatenate(dirs)


def nd_perm(dims, dof=1):
    """Geometric nested dissection of a grid (the ordering the paper leaves unstated).

    ND(box): if the largest extent is <= 2 or the volume is <= 8, list the box lexicographically.
    Otherwise cut the first dimension d of largest extent at m = (lo+hi)//2, order [lo, m) first,
    then [m+1, hi), then the plane x_d = m. A one-plane separator splits star and box stencils.
    perm[k] is the original index placed at position k. With dof > 1 the unknowns of one node
    stay consecutive.
    """
    dims = tuple(int(d) for d in dims)
    ids = grid_node_ids(dims)
    out = []
    stack = [tuple((0, d) for d in dims)]
    # Explicit stack of work items: a box to split, or a block of ids to emit.
    work = [("box", stack[0])]
    while work:
        kind, item = work.pop()
        if kind == "emit":
            out.append(item)
            continue
        box = item
        ext = [hi - lo for lo, hi in box]
        vol = int(np.prod(ext))
        if vol == 0:
            continue
        if max(ext) <= 2 or vol <= 8:
            out.append(ids[tuple(slice(lo, hi) for lo, hi in box)].ravel())
            continue
        d = int(np.argmax(ext))
        lo, hi = box[d]
        m = (lo + hi) // 2
        left = tuple((lo, m) if k == d else b for k, b in enumerate(box))
        right = tuple((m + 1, hi) if k == d else b for k, b in enumerate(box))
        plane = tuple(slice(m, m + 1) if k == d else slice(b[0], b[1]) for k, b in enumerate(box))
        # LIFO: push in reverse order of processing.
        work.append(("emit", ids[plane].ravel()))
        work.append(("box", right))
        work.append(("box", left))
    p = np.concatenate(out).astype(np.int64)
    assert p.size == ids.size
    if dof > 1:
        p = (p[:, None] * dof + np.arange(dof)[None, :]).ravel()
    return p.astype(np.int32)


def lower_csc(n, u, v, w, diag):
    """Assemble the lower triangle (CSC, diagonal first, rows sorted) from edges and a diagonal.

    Each undirected edge (u, v) with weight w contributes A[max, min] = w. Duplicate edges are
    summed.
    """
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    r = np.maximum(u, v)
    c = np.minimum(u, v)
    rows = np.concatenate([np.arange(n, dtype=np.int64), r])
    cols = np.concatenate([np.arange(n, dtype=np.int64), c])
    vals = np.concatenate([np.asarray(diag, dtype=np.float64), np.asarray(w, dtype=np.float64)])
    key = cols * n + rows
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    sums = np.add.reduceat(vals, start)
    cc = uniq // n
    rr = uniq % n
    Ap = np.zeros(n + 1, dtype=np.int64)
    np.add.at(Ap, cc + 1, 1)
    Ap = np.cumsum(Ap)
    return Ap, rr.astype(np.int32), sums


def _seed(cfg_index, matrix_index=0):
    return np.random.default_rng(1000 * cfg_index + matrix_index)


def laplace2d5(side, rng):
    """2D 5-point grid: diagonal 4+U(0,0.1), off-diagonal -U(0.9,1.1) (symmetric, per edge)."""
    dims = (side, side)
    n = side * side
    u, v, _ = grid_edges(dims, "star")
    w = -rng.uniform(0.9, 1.1, size=u.size)
    diag = 4.0 + rng.uniform(0.0, 0.1, size=n)
    Ap, Ai, Ax = lower_csc(n, u, v, w, diag)
    return Matrix(n, Ap, Ai, Ax, nd_perm(dims), name=f"laplace2d5_{side}")


def conduct3d(side, rng, kind="star", shift=1e-3):
    """3D conductivity grid: edges w~U(0.5,2.0), A_ij=-w, A_ii = sum of incident w + shift."""
    dims = (side, side, side)
    n = side ** 3
    u, v, _ = grid_edges(dims, kind)
    w = rng.uniform(0.5, 2.0, size=u.size)
    diag = np.full(n, shift)
    np.add.at(diag, u, w)
    np.add.at(diag, v, w)
    Ap, Ai, Ax = lower_csc(n, u, v, -w, diag)
    return Matrix(n, Ap, Ai, Ax, nd_perm(dims), name=f"conduct3d_{kind}_{side}")


def dd2d9(side, rng, factor=1.05):
    """2D 9-point grid: w~U(0.5,2.0), A_ij=-w, A_ii = factor * sum_j |A_ij|."""
    dims = (side, side)
    n = side * side
    u, v, _ = grid_edges(dims, "box")
    w = rng.uniform(0.5, 2.0, size=u.size)
    s = np.zeros(n)
    np.add.at(s, u, w)
    np.add.at(s, v, w)
    Ap, Ai, Ax = lower_csc(n, u, v, -w, factor * s)
    return Matrix(n, Ap, Ai, Ax, nd_perm(dims), name=f"dd2d9_{side}")


def vector3d27(side, rng, sub=12, jumps=(1.0, 1e2, 1e4), shift=1e-3):
    """3 unknowns per node, 27-point coupling, coefficient jumps by cubic subdomains of `sub`^3.

    A = sum_e c_e (e_i - e_j)(e_i - e_j)^T (x) B_e + shift * diag(c) (x) I_3, B_e = I + d d^T,
    c_e = min of the endpoint coefficients. SPD by construction.
    """
    dims = (side, side, side)
    nn = side ** 3
    nsub = -(-side // sub)
    coef_sub = rng.choice(np.asarray(jumps), size=(nsub, nsub, nsub))
    g = np.arange(side) // sub
    coef = coef_sub[g[:, None, None], g[None, :, None], g[None, None, :]].ravel()
    u, v, dirs = grid_edges(dims, "box")
    ce = np.minimum(coef[u], coef[v])
    B = np.eye(3)[None, :, :] + dirs[:, :, None] * dirs[:, None, :]
    blk = ce[:, None, None] * B  # edge block
    n = 3 * nn
    # node-diagonal blocks
    D = np.zeros((nn, 3, 3))
    np.add.at(D, u, blk)
    np.add.at(D, v, blk)
    D += (shift * coef)[:, None, None] * np.eye(3)[None]
    rows, cols, vals = [], [], []
    a, b = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    # off-diagonal node blocks: A[3u+a, 3v+b] = -blk[a,b]
    rows.append((3 * u[:, None, None] + a[None]).ravel())
    cols.append((3 * v[:, None, None] + b[None]).ravel())
    vals.append((-blk).ravel())
    # within-node blocks (strictly lower part; the diagonal goes separately)
    lo = a > b
    rows.append((3 * np.arange(nn)[:, None] + a[lo][None]).ravel())
    cols.append((3 * np.arange(nn)[:, None] + b[lo][None]).ravel())
    vals.append(D[:, lo].ravel())
    diag = D[:, np.arange(3), np.arange(3)].ravel()
    Ap, Ai, Ax = lower_csc(n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals), diag)
    return Matrix(n, Ap, Ai, Ax, nd_perm(dims, dof=3), name=f"vector3d27_{side}")


def erdos_renyi(n, avg_degree, rng):
    """Random graph with about n*avg_degree/2 edges; off-diagonal -U(0.5,2.0),
    A_ii = f * sum_j |A_ij| with f ~ U(1.01, 1.5). No ordering is attached."""
    m = int(round(n * avg_degree / 2))
    u = rng.integers(0, n, size=m)
    v = rng.integers(0, n, size=m)
    keep = u != v
    u, v = u[keep], v[keep]
    a, b = np.minimum(u, v), np.maximum(u, v)
    key = np.unique(a.astype(np.int64) * n + b)
    u, v = key // n, key % n
    w = rng.uniform(0.5, 2.0, size=u.size)
    s = np.zeros(n)
    np.add.at(s, u, w)
    np.add.at(s, v, w)
    f = rng.uniform(1.01, 1.5)
    s = np.where(s == 0, 1.0, s)
    Ap, Ai, Ax = lower_csc(n, u, v, -w, f * s)
    return Matrix(n, Ap, Ai, Ax, None, name=f"er_{n}_{avg_degree}")


def random_spd_pattern(n, density, rng, dominance=1.5):
    """Small random SPD matrix (diagonally dominant) for exhaustive tests."""
    mask = rng.random((n, n)) < density
    mask = np.tril(mask, -1)
    r, c = np.nonzero(mask)
    w = rng.uniform(0.5, 2.0, size=r.size)
    s = np.zeros(n)
    np.add.at(s, r, w)
    np.add.at(s, c, w)
    diag = dominance * s + 1.0
    Ap, Ai, Ax = lower_csc(n, r, c, -w, diag)
    return Matrix(n, Ap, Ai, Ax, None, name=f"rand_{n}")


def wide_block(nblock, ntail, rng):
    """Natural-order pattern with one wide supernode: columns 0..nblock-1 are coupled densely and
    every row of a first tail (ntail rows after the block) to column 0; a second tail of ntail rows
    is coupled to the first tail's first column only. The factor's first supernode then has nblock
    columns and the first tail as its rows below the diagonal block, and amalgamation with its
    parent would add nblock * ntail explicit zeros. Diagonally dominant."""
    n = nblock + 2 * ntail
    r, c = np.tril_indices(nblock, -1)
    r = np.concatenate([r, np.arange(nblock, nblock + ntail), np.arange(nblock + ntail, n)])
    c = np.concatenate([c, np.zeros(ntail, dtype=r.dtype), np.full(ntail, nblock, dtype=r.dtype)])
    wv = rng.uniform(0.5, 2.0, size=r.size)
    s = np.zeros(n)
    np.add.at(s, r, wv)
    np.add.at(s, c, wv)
    Ap, Ai, Ax = lower_csc(n, r, c, -wv, 1.5 * s + 1.0)
    return Matrix(n, Ap, Ai, Ax, None, name=f"wide_{nblock}_{ntail}")


def rhs(n, nrhs, rng):
    """Dense right-hand sides, column-major (n x nrhs), entries N(0,1)."""
    return np.asfortranarray(rng.standard_normal((n, nrhs)))


def csc_to_dense(M):
    """Full symmetric dense copy of a lower-CSC matrix (small n only)."""
    A = np.zeros((M.n, M.n))
    for j in range(M.n):
        for p in range(M.Ap[j], M.Ap[j + 1]):
            i = M.Ai[p]
            A[i, j] = M.Ax[p]
            A[j, i] = M.Ax[p]
    return A


def block_diagonal(mats):
    """One matrix whose diagonal blocks are the given matrices (an uneven batch). Its ordering
    places each block's own ordering in its own index range."""
    n = sum(M.n for M in mats)
    Ap = [np.zeros(1, dtype=np.int64)]
    Ai, Ax, perm = [], [], []
    off_n = 0
    off_nz = 0
    for M in mats:
        Ap.append(M.Ap[1:] + off_nz)
        Ai.append(M.Ai.astype(np.int64) + off_n)
        Ax.append(M.Ax)
        perm.append((M.perm if M.perm is not None else np.arange(M.n)).astype(np.int64) + off_n)
        off_n += M.n
        off_nz += M.nnz
    return Matrix(n, np.concatenate(Ap), np.concatenate(Ai), np.concatenate(Ax), np.concatenate(perm),
                  name=f"blockdiag_{len(mats)}")


def uneven_grid_batch(count, rng, lo=32, hi=256):
    """Uneven batch of 2D 5-point grids with sides uniform in lo..hi (values as laplace2d5)."""
    sides = rng.integers(lo, hi + 1, size=count)
    return [laplace2d5(int(s), rng) for s in sides], sides


def same_pattern_batch(maker, count, seed):
    """count value sets on one pattern: maker(rng) must build the same pattern for every rng.
    Returns the first matrix and a (count, nnz) array of values."""
    first = maker(np.random.default_rng(seed))
    vals = np.empty((count, first.nnz))
    vals[0] = first.Ax
    for b in range(1, count):
        M = maker(np.random.default_rng(seed + b))
        assert M.nnz == first.nnz
        vals[b] = M.Ax
    return first, vals


def rcm_perm(M):
    """Reverse Cuthill-McKee ordering (scipy) for patterns without geometry."""
    import scipy.sparse as sp
    from scipy.sparse.csgraph import reverse_cuthill_mckee
    L = sp.csc_matrix((np.ones(M.nnz), M.Ai, M.Ap), shape=(M.n, M.n))
    G = (L + L.T).tocsr()
    return np.ascontiguousarray(reverse_cuthill_mckee(G, symmetric_mode=True), dtype=np.int32)


def pattern_suite(count, seed):
    """A mix of generated SPD patterns for the cost model: 2D 5/9-point grids (sides 24..160),
    3D 7/27-point grids (sides 8..32), 3-dof 27-point grids (sides 5..12) and Erdos-Renyi graphs
    (n 800..4000, average degree 4..16, reverse Cuthill-McKee order). Pattern i uses the seed
    seed + i, so disjoint seed ranges give disjoint sets."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed + i)
        kind = i % 7
        if kind == 0:
            M = laplace2d5(int(rng.integers(24, 161)), rng)
        elif kind == 1:
            M = dd2d9(int(rng.integers(24, 161)), rng)
        elif kind == 2:
            M = conduct3d(int(rng.integers(8, 33)), rng, "star")
        elif kind == 3:
            M = conduct3d(int(rng.integers(8, 25)), rng, "box")
        elif kind == 4:
            M = vector3d27(int(rng.integers(5, 13)), rng, sub=4)
        elif kind == 5:
            M = conduct3d(int(rng.integers(10, 29)), rng, "star", shift=1e-2)
        else:
            M = erdos_renyi(int(rng.integers(800, 4001)), int(rng.integers(4, 17)), rng)
            M.perm = rcm_perm(M)
        M.name = f"suite{seed + i}_{M.name}"
        out.append(M)
    return out


# The learned-schedule suite at its stated sizes: 2D 5/9-point and 3D 7/27-point grids of sides
# 32..128 and Erdos-Renyi graphs with n in 50,000..200,000 and average degree 4..16 (made SPD by
# a dominance factor U(1.01, 1.5)). Pattern i has seed seed + i; disjoint seed ranges give
# disjoint sets. Specs are cheap; a matrix is built only for a spec that is kept.
SUITE5_KINDS = ("grid2d5", "grid2d9", "grid3d7", "grid3d27", "er")


def suite5_spec(i, seed):
    rng = np.random.default_rng(seed + i)
    kind = SUITE5_KINDS[i % len(SUITE5_KINDS)]
    if kind == "er":
        return {"kind": kind, "n": int(rng.integers(50000, 200001)), "degree": int(rng.integers(4, 17)),
                "seed": seed + i}
    return {"kind": kind, "side": int(rng.integers(32, 129)), "seed": seed + i}


def suite5_estimate_flops(spec):
    """Factor flops (sum c_j^2) of a spec before it is built, from measured anchors of the same
    families under their orderings: 3D 7-point 5.7e9 at side 32, 3D 27-point 2.6e10 at side 40,
    both growing as side^6 (nested dissection); 2D grids stay below 1e9 at side 128; Erdos-Renyi at
    n = 50,000 and degree 4 (the smallest of the suite) 4.6e11 under minimum degree, larger n and
    degree only add fill."""
    k = spec["kind"]
    if k == "grid3d7":
        return 5.7e9 * (spec["side"] / 32.0) ** 6
    if k == "grid3d27":
        return 2.6e10 * (spec["side"] / 40.0) ** 6
    if k == "er":
        return 4.6e11 * (spec["n"] / 50000.0) ** 2 * (spec["degree"] / 4.0)
    return 1e9 * (spec["side"] / 128.0) ** 3


def suite5_build(spec):
    rng = np.random.default_rng(spec["seed"])
    k = spec["kind"]
    if k == "grid2d5":
        M = laplace2d5(spec["side"], rng)
    elif k == "grid2d9":
        M = dd2d9(spec["side"], rng)
    elif k == "grid3d7":
        M = conduct3d(spec["side"], rng, "star")
    elif k == "grid3d27":
        M = conduct3d(spec["side"], rng, "box")
    else:
        M = erdos_renyi(spec["n"], spec["degree"], rng)
        M.perm = rcm_perm(M)
    M.name = f"suite5_{spec['seed']}_{M.name}"
    return M


def cfg(name, matrix_index=0):
    """The named workloads with their seeds (1000 * config index + matrix index)."""
    if name == "laplace2d5_64":
        return laplace2d5(64, _seed(0, matrix_index))
    if name == "conduct3d7_64":
        return conduct3d(64, _seed(1, matrix_index), "star")
    if name == "conduct3d7_48":  # the smaller case of the same family, for profiler captures
        return conduct3d(48, _seed(1, 48 + matrix_index), "star")
    if name == "conduct3d27_40":
        return conduct3d(40, _seed(1, 1 + matrix_index), "box")
    if name == "dd2d9_128":
        return dd2d9(128, _seed(2, matrix_index))
    if name == "vector3d27_48":
        return vector3d27(48, _seed(3, matrix_index))
    raise KeyError(name)
