"""Python view of the CPU FP64 oracle (``sym_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg use it. The product path (``paper_1705_06575_gb300``) never imports it, and it imports nothing
from the product. It is built with plain ``gcc`` into ``oracle/_build/liborc.so``.

Parity notes: every function is pinned by the ``-m "not gpu"`` tests in ``tests/test_oracle.py``
against closed forms, brute-force elimination and library routines (numpy's dense Cholesky).
"""
from __future__ import annotations

import ctypes as ct
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liborc.so")
_lock = threading.Lock()
_libs = {}

# Amalgamation parameters: nrelax0..2 (column counts), zrelax0..2 (zero fraction, per mille).
DEFAULT_RELAX = (4, 16, 48, 800, 100, 50)

ERR_INVALID = -1
ERR_NOT_SPD = -2


def build(force=False, defines=()):
    """Compile the oracle with gcc (no CUDA involved). ``defines`` builds a separate copy with
    those preprocessor symbols (the planted-mistake copies the pin tests use)."""
    so = _SO if not defines else os.path.join(_HERE, "_build", "liborc_" + "_".join(defines).lower() + ".so")
    os.makedirs(os.path.dirname(so), exist_ok=True)
    src = os.path.join(_HERE, "sym_oracle.c")
    if not force and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    tmp = so + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC"] + [f"-D{d}" for d in defines] +
                          ["-o", tmp, src, "-lm"])
    os.replace(tmp, so)
    return so


def _load(defines=()):
    key = tuple(defines)
    with _lock:
        if key in _libs:
            return _libs[key]
        lib = ct.CDLL(build(defines=key))
        P = ct.c_void_p
        i64, i32 = ct.c_int64, ct.c_int32
        lib.orc_validate.argtypes = [i64, P, P]
        lib.orc_validate.restype = ct.c_int
        lib.orc_analyze.argtypes = [i64, P, P, P, P, ct.c_int, ct.POINTER(P)]
        lib.orc_analyze.restype = ct.c_int
        lib.orc_analyze_rules.argtypes = [i64, P, P, P, P, i32, P, i64, ct.c_int, ct.POINTER(P)]
        lib.orc_analyze_rules.restype = ct.c_int
        lib.orc_free.argtypes = [P]
        lib.orc_factor.argtypes = [P, P, i64]
        lib.orc_factor.restype = ct.c_int
        lib.orc_solve.argtypes = [P, i64, P, P]
        lib.orc_solve.restype = ct.c_int
        lib.orc_factor_residual.argtypes = [P, P, i64]
        lib.orc_factor_residual.restype = ct.c_double
        lib.orc_factor_residual_with.argtypes = [P, P, P, i64]
        lib.orc_factor_residual_with.restype = ct.c_double
        lib.orc_backward_error.argtypes = [i64, P, P, P, i64, P, P]
        lib.orc_backward_error.restype = ct.c_double
        lib.orc_reach.argtypes = [P, i64, P, P]
        lib.orc_reach.restype = i64
        lib.orc_sparse_lsolve.argtypes = [P, i64, P, i64, P, P, P]
        lib.orc_sparse_lsolve.restype = None
        lib.orc_row_patterns_check.argtypes = [P]
        lib.orc_row_patterns_check.restype = ct.c_int
        for name, rt in [("n", i64), ("nnzL", i64), ("nfsn", i32), ("nsn", i32), ("nsrows", i64),
                         ("npairs", i64), ("nrel", i64), ("nlev", i32), ("err_col", i64), ("nmerge", i64)]:
            f = getattr(lib, "orc_" + name)
            f.argtypes = [P]
            f.restype = rt
        for name in ["perm", "parent", "Lp", "Li", "Lx", "Cp", "Ci", "Cmap", "fsn", "sn", "srp",
                     "sri", "sparent", "dp", "dk", "dr0", "dnin", "relp", "rel", "level", "lvp",
                     "lvl", "merges"]:
            f = getattr(lib, "orc_" + name)
            f.argtypes = [P]
            f.restype = P
        _libs[key] = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ct.c_void_p)


def _view(addr, count, dtype):
    if count == 0 or not addr:
        return np.zeros(0, dtype=dtype)
    buf = (ct.c_char * (int(count) * np.dtype(dtype).itemsize)).from_address(addr)
    return np.frombuffer(buf, dtype=dtype).copy()


def validate(n, Ap, Ai):
    lib = _load()
    Ap = np.ascontiguousarray(Ap, dtype=np.int64)
    Ai = np.ascontiguousarray(Ai, dtype=np.int32)
    return lib.orc_validate(int(n), _ptr(Ap), _ptr(Ai))


class Oracle:
    """Symbolic analysis (every integer output of the inspector) plus the numeric factor."""

    def __init__(self, n, Ap, Ai, perm0=None, relax=DEFAULT_RELAX, want_rel=False, defines=(), rules=None,
                 fund_rule=None):
        """rules (records {amalgamate, nrelax0..2, zrelax0..2}) with fund_rule (one index per
        fundamental supernode) replace relax by per-supernode amalgamation rules."""
        lib = _load(defines)
        self._lib = lib
        self.n = int(n)
        self.Ap = np.ascontiguousarray(Ap, dtype=np.int64)
        self.Ai = np.ascontiguousarray(Ai, dtype=np.int32)
        p0 = None if perm0 is None else np.ascontiguousarray(perm0, dtype=np.int32)
        rl = None if relax is None else np.ascontiguousarray(relax, dtype=np.int32)
        h = ct.c_void_p()
        if rules is not None:
            R = np.ascontiguousarray(rules, dtype=np.int32).reshape(-1, 7)
            F = np.ascontiguousarray(fund_rule, dtype=np.int32)
            rc = lib.orc_analyze_rules(self.n, _ptr(self.Ap), _ptr(self.Ai), _ptr(p0), _ptr(R), R.shape[0], _ptr(F),
                                       F.size, 1 if want_rel else 0, ct.byref(h))
        else:
            rc = lib.orc_analyze(self.n, _ptr(self.Ap), _ptr(self.Ai), _ptr(p0), _ptr(rl),
                                 1 if want_rel else 0, ct.byref(h))
        if rc != 0:
            raise ValueError(f"oracle analyze failed: {rc}")
        self._h = h
        self._read_symbolic()

    def _read_symbolic(self):
        lib, h, n = self._lib, self._h, self.n
        self.nnzL = lib.orc_nnzL(h)
        self.perm = _view(lib.orc_perm(h), n, np.int32)
        self.parent = _view(lib.orc_parent(h), n, np.int32)
        self.Lp = _view(lib.orc_Lp(h), n + 1, np.int64)
        self.Li = _view(lib.orc_Li(h), self.nnzL, np.int32)
        self.colcount = np.diff(self.Lp)
        nnzA = int(self.Ap[-1])
        self.Cp = _view(lib.orc_Cp(h), n + 1, np.int64)
        self.Ci = _view(lib.orc_Ci(h), nnzA, np.int32)
        self.Cmap = _view(lib.orc_Cmap(h), nnzA, np.int64)
        nf = lib.orc_nfsn(h)
        self.fsn = _view(lib.orc_fsn(h), nf + 1, np.int32)
        ns = lib.orc_nsn(h)
        self.nsn = ns
        self.sn = _view(lib.orc_sn(h), ns + 1, np.int32)
        self.srp = _view(lib.orc_srp(h), ns + 1, np.int64)
        self.sri = _view(lib.orc_sri(h), lib.orc_nsrows(h), np.int32)
        self.sparent = _view(lib.orc_sparent(h), ns, np.int32)
        npairs = lib.orc_npairs(h)
        self.dp = _view(lib.orc_dp(h), ns + 1, np.int64)
        self.dk = _view(lib.orc_dk(h), npairs, np.int32)
        self.dr0 = _view(lib.orc_dr0(h), npairs, np.int64)
        self.dnin = _view(lib.orc_dnin(h), npairs, np.int32)
        nrel = lib.orc_nrel(h)
        self.relp = _view(lib.orc_relp(h), npairs + 1, np.int64) if nrel else None
        self.rel = _view(lib.orc_rel(h), nrel, np.int32) if nrel else None
        self.level = _view(lib.orc_level(h), ns, np.int32)
        nl = lib.orc_nlev(h)
        self.nlev = nl
        self.lvp = _view(lib.orc_lvp(h), nl + 1, np.int32)
        self.lvl = _view(lib.orc_lvl(h), ns, np.int32)
        # amalgamation log: (first column of the absorbed supernode, first column of the one it
        # merged into, at the time of the merge), in the order the merges were made
        self.merges = _view(lib.orc_merges(h), 2 * lib.orc_nmerge(h), np.int32).reshape(-1, 2)
        self.flops = int(np.sum(self.colcount.astype(np.float64) ** 2))
        self.flops_exact = int(np.sum(self.colcount.astype(np.int64) ** 2))
        self.Lx = None
        self.err_col = -1

    def row_patterns_agree(self):
        """Etree row walks (Sec. 3.2) reproduce the transpose of the Eq. (1) column patterns."""
        return self._lib.orc_row_patterns_check(self._h) == 0

    def factor(self, Ax, kmax=-1):
        """Up-looking numeric factor; returns 0, or ERR_NOT_SPD with ``err_col`` set."""
        self._Ax = np.ascontiguousarray(Ax, dtype=np.float64)
        rc = self._lib.orc_factor(self._h, _ptr(self._Ax), int(kmax))
        self.err_col = self._lib.orc_err_col(self._h)
        self.Lx = _view(self._lib.orc_Lx(self._h), self.nnzL, np.float64)
        return rc

    def solve(self, B):
        B = np.asfortranarray(B, dtype=np.float64)
        if B.ndim == 1:
            B = B[:, None]
        X = np.zeros_like(B, order="F")
        self._lib.orc_solve(self._h, B.shape[1], _ptr(B), _ptr(X))
        return X

    def factor_residual(self, Ax=None, kmax=0):
        Ax = self._Ax if Ax is None else np.ascontiguousarray(Ax, dtype=np.float64)
        return self._lib.orc_factor_residual(self._h, _ptr(Ax), int(kmax))

    def reach(self, beta):
        """Reach_L(beta) (permuted numbering) in a topological order (reverse DFS finishing)."""
        beta = np.ascontiguousarray(beta, dtype=np.int32)
        out = np.zeros(self.n, dtype=np.int32)
        nr = self._lib.orc_reach(self._h, beta.size, _ptr(beta), _ptr(out))
        return out[:nr].copy()

    def sparse_lsolve(self, beta, bvals, reach=None):
        """Solve L x = b for b with entries bvals at beta (permuted numbering); returns (reach,
        dense x with zeros outside the reach)."""
        beta = np.ascontiguousarray(beta, dtype=np.int32)
        bvals = np.ascontiguousarray(bvals, dtype=np.float64)
        r = self.reach(beta) if reach is None else np.ascontiguousarray(reach, dtype=np.int32)
        x = np.zeros(self.n)
        self._lib.orc_sparse_lsolve(self._h, r.size, _ptr(r), beta.size, _ptr(beta), _ptr(bvals), _ptr(x))
        return r, x

    def factor_residual_with(self, Ax, Lx, kmax=0):
        """||L L^T - C||_F / ||C||_F for values Lx given on this oracle's pattern."""
        Ax = np.ascontiguousarray(Ax, dtype=np.float64)
        Lx = np.ascontiguousarray(Lx, dtype=np.float64)
        assert Lx.size == self.nnzL
        return self._lib.orc_factor_residual_with(self._h, _ptr(Ax), _ptr(Lx), int(kmax))

    def L_dense(self):
        L = np.zeros((self.n, self.n))
        for j in range(self.n):
            L[self.Li[self.Lp[j]:self.Lp[j + 1]], j] = self.Lx[self.Lp[j]:self.Lp[j + 1]]
        return L

    def close(self):
        if self._h:
            self._lib.orc_free(self._h)
            self._h = ct.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def backward_error(n, Ap, Ai, Ax, B, X):
    lib = _load()
    B = np.asfortranarray(B, dtype=np.float64)
    X = np.asfortranarray(X, dtype=np.float64)
    if B.ndim == 1:
        B, X = B[:, None], X[:, None]
    Ap = np.ascontiguousarray(Ap, dtype=np.int64)
    Ai = np.ascontiguousarray(Ai, dtype=np.int32)
    Ax = np.ascontiguousarray(Ax, dtype=np.float64)
    return lib.orc_backward_error(int(n), _ptr(Ap), _ptr(Ai), _ptr(Ax), B.shape[1], _ptr(B), _ptr(X))
