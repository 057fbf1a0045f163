"""Test helpers: map the library's supernodal panels onto the oracle's column pattern."""
import numpy as np


def panels_on_pattern(sx, Lx, Lp, Li):
    """Values of the panel storage Lx at the entries (Li, column) of the pattern Lp/Li.

    sx: dict of the library's exports (super, rowptr, rows, lxptr). Also returns the largest
    magnitude stored outside the pattern (amalgamation padding and the strict upper part of the
    diagonal blocks), which must be exactly zero.
    """
    sup, rowptr, rows, lxptr = sx["super"], sx["rowptr"], sx["rows"], sx["lxptr"]
    out = np.empty(Li.size, dtype=np.float64)
    outside = 0.0
    for J in range(sup.size - 1):
        f, l = int(sup[J]), int(sup[J + 1])
        nc = l - f
        R = rows[rowptr[J]:rowptr[J + 1]]
        nr = R.size
        panel = Lx[lxptr[J]:lxptr[J + 1]].reshape(nc, nr)  # row c of the view = column f + c
        lo, hi = Lp[f], Lp[l]
        rr = Li[lo:hi]
        cc = np.repeat(np.arange(nc), np.diff(Lp[f:l + 1]))
        pos = np.searchsorted(R, rr)
        assert np.all(R[pos] == rr), "pattern entry missing from the supernode's rows"
        out[lo:hi] = panel[cc, pos]
        mask = np.ones((nc, nr), dtype=bool)
        mask[cc, pos] = False
        if mask.any():
            outside = max(outside, float(np.abs(panel[mask]).max()))
    return out, outside


def exports(solver):
    return {k: solver.export(k) for k in ("super", "rowptr", "rows", "lxptr", "perm")}
