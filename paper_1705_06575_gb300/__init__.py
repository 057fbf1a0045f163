"""GB300 supernodal Cholesky (numeric phase of decoupled sparse Cholesky, after Sympiler).

Thin Python binding of the C ABI in ``include/sym.h``: the functions below have the same names
and arguments as the C entry points and only marshal arguments (numpy arrays for host data,
``torch.Tensor`` or raw integers for device pointers). Every step of the factorization and the
solve runs in the CUDA kernels of ``_build/libsym.so``; there is no Python or CPU fallback. If
the library cannot be built or loaded the import of the binding fails with an error.
"""
from __future__ import annotations

import ctypes as ct
import threading

import numpy as np

from . import build as _build

__all__ = [
    "SymError", "sym_options", "sym_stats", "sym_options_default", "sym_analyze",
    "sym_analyze_perm", "sym_set_stream", "sym_factor", "sym_factor_async", "sym_status",
    "sym_factor_host", "sym_solve", "sym_solve_multi", "sym_solve_host", "sym_info",
    "sym_last_error_column", "sym_get_factor_host", "sym_export", "sym_free", "load", "Solver",
    "EXPORTS", "sym_profile", "sym_profile_read", "sym_profile_launches", "sym_fma_peak", "sym_tc_probe", "sym_solve_host_ptr", "KINDS",
    "sym_solve_multi_noalloc", "sym_set_refinement", "sym_refinement_info", "sym_pivot_info",
    "sym_set_pivot_threshold", "sym_set_tc_wait", "sym_analyze_rules", "sym_autotune", "sym_factor_batch",
    "sym_batch_error_columns", "sym_solve_batch", "sym_get_batch_factor_host", "Reach", "MLP",
]

SYM_OK = 0
SYM_ERR_INVALID = -1
SYM_ERR_NOT_SPD = -2
SYM_ERR_CUDA = -3
SYM_ERR_OOM = -4
SYM_ERR_STATE = -5
SYM_ERR_TIMEOUT = -6
SYM_ERR_LIMIT = -7
SYM_ERR_NO_CONVERGENCE = -8
SYM_PREC_FP64 = 0
SYM_PREC_MIXED = 1
SYM_ORDER_NATURAL = 0
SYM_ORDER_GIVEN = 1
SYM_ORDER_AUTO = 2
SYM_ORDER_METHOD_MD = 3
SYM_ORDER_METHOD_ND = 4
SYM_FLAG_HOST_ONLY = 1
SYM_FLAG_NO_GRAPHS = 2
SYM_FLAG_ONE_STREAM = 4
SYM_FLAG_NO_TENSOR_CORES = 8
SYM_FLAG_NO_FUSED_LEVELS = 16

# name -> (code, numpy dtype)
EXPORTS = {
    "perm": (1, np.int32), "parent": (2, np.int32), "colcount": (3, np.int64),
    "fsuper": (4, np.int32), "super": (5, np.int32), "rowptr": (6, np.int64),
    "rows": (7, np.int32), "sparent": (8, np.int32), "descptr": (9, np.int64),
    "desc": (10, np.int32), "descr0": (11, np.int64), "descnin": (12, np.int32),
    "relptr": (13, np.int64), "rel": (14, np.int32), "level": (15, np.int32),
    "levelptr": (16, np.int32), "levellist": (17, np.int32), "lxptr": (18, np.int64),
    "factor_launches": (19, np.int64), "fwd_launches": (20, np.int64), "bwd_launches": (21, np.int64),
    "tasks": (22, np.int32), "upd_tasks": (23, np.int64), "upd_entries": (24, np.int64),
    "contrib_ptr": (25, np.int64), "contrib": (26, np.int32), "batch_panel": (27, np.int32),
    "fwd_panel": (28, np.int32), "bwd_panel": (29, np.int32),
}


class SymError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


class sym_options(ct.Structure):
    _fields_ = [("ordering", ct.c_int32), ("amalgamate", ct.c_int32), ("nrelax", ct.c_int32 * 3),
                ("zrelax_permille", ct.c_int32 * 3), ("flags", ct.c_uint32),
                ("precision", ct.c_int32), ("reserved", ct.c_int32 * 7)]


class sym_stats(ct.Structure):
    _fields_ = [("n", ct.c_int64), ("nnz_a", ct.c_int64), ("nnz_l", ct.c_int64),
                ("storage_l", ct.c_int64), ("flops", ct.c_double), ("solve_flops", ct.c_double),
                ("nsuper_fund", ct.c_int32), ("nsuper", ct.c_int32), ("nlevels", ct.c_int32),
                ("max_ncols", ct.c_int32), ("npairs", ct.c_int64), ("nlaunch_factor", ct.c_int64),
                ("nlaunch_solve", ct.c_int64), ("analyze_seconds", ct.c_double),
                ("device_bytes", ct.c_int64), ("upd_tasks", ct.c_int64), ("upd_entries", ct.c_int64),
                ("dense_tasks", ct.c_int64), ("exec_flops", ct.c_double), ("update_flops", ct.c_double),
                ("ordering_method", ct.c_int32), ("reserved0", ct.c_int32), ("ordering_flops_md", ct.c_double),
                ("ordering_flops_nd", ct.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load():
    """Build (if stale) and load the CUDA library; raise if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ct.CDLL(_build.build())
        P, i64, i32, I = ct.c_void_p, ct.c_int64, ct.c_int32, ct.c_int
        sigs = {
            "sym_options_default": ([ct.POINTER(sym_options)], I),
            "sym_analyze": ([i64, P, P, ct.POINTER(P)], I),
            "sym_analyze_perm": ([i64, P, P, P, ct.POINTER(sym_options), ct.POINTER(P)], I),
            "sym_set_stream": ([P, P], I),
            "sym_factor": ([P, P], I),
            "sym_factor_async": ([P, P], I),
            "sym_status": ([P], I),
            "sym_factor_host": ([P, P], I),
            "sym_solve": ([P, P, P], I),
            "sym_solve_multi": ([P, i32, P, i64, P, i64], I),
            "sym_solve_host": ([P, i32, P, i64, P, i64], I),
            "sym_info": ([P, ct.POINTER(sym_stats)], I),
            "sym_last_error_column": ([P, ct.POINTER(i64)], I),
            "sym_get_factor_host": ([P, P], I),
            "sym_export": ([P, i32, P], i64),
            "sym_error_string": ([I], ct.c_char_p),
            "sym_last_error_string": ([], ct.c_char_p),
            "sym_free": ([P], None),
            "sym_profile": ([P, i32], I),
            "sym_profile_read": ([P, i32, ct.POINTER(ct.c_double), ct.POINTER(i64),
                                  ct.POINTER(ct.c_double)], I),
            "sym_fma_peak": ([i32, ct.POINTER(ct.c_double)], I),
            "sym_tc_probe": ([P, P, P, ct.c_uint32, ct.c_uint32], I),
            "sym_profile_launches": ([P, i32, P], i64),
            "sym_solve_multi_noalloc": ([P, i32, P, i64, P, i64], I),
            "sym_set_refinement": ([P, ct.c_double, i32], I),
            "sym_factor_batch": ([P, i32, P, i64], I),
            "sym_reach_analyze": ([P, i64, P, ct.POINTER(P)], I),
            "sym_reach_size": ([P], i64),
            "sym_reach_indices": ([P, P], I),
            "sym_reach_export": ([P, i32, P], i64),
            "sym_solve_lower_sparse": ([P, P, P, P], I),
            "sym_reach_free": ([P], None),
            "sym_mlp_create": ([i32, i32, ct.c_uint64, ct.POINTER(P)], I),
            "sym_mlp_nparams": ([P], i64),
            "sym_mlp_set_params": ([P, P], I),
            "sym_mlp_get_params": ([P, P], I),
            "sym_mlp_predict": ([P, i64, P, P], I),
            "sym_mlp_gradient": ([P, i64, P, P, P, P], I),
            "sym_mlp_train": ([P, i64, P, P, i32, ct.c_float, P], I),
            "sym_mlp_free": ([P], None),
            "sym_batch_error_columns": ([P, P], I),
            "sym_solve_batch": ([P, i32, i32, P, i64, i64, P, i64, i64], I),
            "sym_get_batch_factor_host": ([P, i32, P], I),
            "sym_refinement_info": ([P, ct.POINTER(i32), ct.POINTER(ct.c_double)], I),
            "sym_pivot_info": ([P, i32, ct.POINTER(ct.c_double), ct.POINTER(i64), ct.POINTER(i32)], I),
            "sym_set_pivot_threshold": ([P, ct.c_double], I),
            "sym_set_tc_wait": ([P, ct.c_uint64, i32], I),
            "sym_analyze_rules": ([i64, P, P, P, ct.POINTER(sym_options), i32, P, i64, P, ct.POINTER(P)], I),
            "sym_autotune": ([P, i32, P, i64, i32, ct.POINTER(i32), ct.POINTER(i32)], I),
        }
        for name, (args, res) in sigs.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(rc):
    if rc < 0:
        lib = load()
        raise SymError(rc, lib.sym_last_error_string().decode() or lib.sym_error_string(rc).decode())
    return rc


def _host(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _dptr(x):
    """Device address of a torch tensor (or an int address)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def sym_options_default():
    o = sym_options()
    _check(load().sym_options_default(ct.byref(o)))
    return o


def sym_analyze(n, Ap, Ai):
    Ap, Ai = _host(Ap, np.int64), _host(Ai, np.int32)
    h = ct.c_void_p()
    _check(load().sym_analyze(int(n), Ap.ctypes.data, Ai.ctypes.data, ct.byref(h)))
    return h


def sym_analyze_perm(n, Ap, Ai, perm=None, opt=None):
    Ap, Ai = _host(Ap, np.int64), _host(Ai, np.int32)
    pp = None if perm is None else _host(perm, np.int32)
    h = ct.c_void_p()
    _check(load().sym_analyze_perm(int(n), Ap.ctypes.data, Ai.ctypes.data,
                                   None if pp is None else pp.ctypes.data,
                                   None if opt is None else ct.byref(opt), ct.byref(h)))
    return h


def sym_analyze_rules(n, Ap, Ai, perm, opt, rules, fund_rule):
    """Inspector with one amalgamation rule per fundamental supernode: rules is an (R, 7) int32
    table {amalgamate, nrelax[3], zrelax_permille[3]}, fund_rule one row index per fundamental
    supernode of this pattern and ordering."""
    Ap, Ai = _host(Ap, np.int64), _host(Ai, np.int32)
    pp = None if perm is None else _host(perm, np.int32)
    R = np.ascontiguousarray(rules, dtype=np.int32).reshape(-1, 7)
    F = np.ascontiguousarray(fund_rule, dtype=np.int32)
    h = ct.c_void_p()
    _check(load().sym_analyze_rules(int(n), Ap.ctypes.data, Ai.ctypes.data, None if pp is None else pp.ctypes.data,
                                    None if opt is None else ct.byref(opt), int(R.shape[0]), R.ctypes.data,
                                    int(F.size), F.ctypes.data, ct.byref(h)))
    return h


def sym_set_stream(h, stream):
    """stream: a torch.cuda.Stream, a raw cudaStream_t integer, or None (legacy default)."""
    s = getattr(stream, "cuda_stream", stream)
    return _check(load().sym_set_stream(h, s))


def sym_factor(h, Ax):
    return _check(load().sym_factor(h, _dptr(Ax)))


def sym_factor_async(h, Ax):
    return _check(load().sym_factor_async(h, _dptr(Ax)))


def sym_status(h):
    return _check(load().sym_status(h))


def sym_factor_host(h, Ax):
    """Ax: a numpy array, or the integer address of host memory (pinned or pageable)."""
    if isinstance(Ax, int):
        return _check(load().sym_factor_host(h, Ax))
    Ax = _host(Ax, np.float64)
    return _check(load().sym_factor_host(h, Ax.ctypes.data))


def sym_solve(h, b, x):
    return _check(load().sym_solve(h, _dptr(b), _dptr(x)))


def sym_solve_multi(h, nrhs, B, ldb, X, ldx):
    return _check(load().sym_solve_multi(h, int(nrhs), _dptr(B), int(ldb), _dptr(X), int(ldx)))


SYM_NOALLOC_MAX_WORK = 1048576


def sym_solve_multi_noalloc(h, nrhs, B, ldb, X, ldx):
    """sym_solve_multi without any allocation (work block in the library's fixed device array)."""
    return _check(load().sym_solve_multi_noalloc(h, int(nrhs), _dptr(B), int(ldb), _dptr(X), int(ldx)))


def sym_solve_host(h, B):
    """Host right-hand sides (n or n x nrhs); returns X with the same shape."""
    B = np.asarray(B, dtype=np.float64)
    one = B.ndim == 1
    Bf = np.asfortranarray(B[:, None] if one else B)
    X = np.zeros_like(Bf, order="F")
    n = Bf.shape[0]
    _check(load().sym_solve_host(h, Bf.shape[1], Bf.ctypes.data, n, X.ctypes.data, n))
    return X[:, 0] if one else X


def sym_solve_host_ptr(h, nrhs, B, ldb, X, ldx):
    """Host-pointer solve with raw integer addresses (for pinned buffers)."""
    return _check(load().sym_solve_host(h, int(nrhs), B, int(ldb), X, int(ldx)))


SYM_PROFILE_OFF, SYM_PROFILE_ON, SYM_PROFILE_RESET = 0, 1, 2
KINDS = {"scatter": 0, "update": 1, "potrf": 2, "trsm": 3, "gemm": 4, "trtri": 5, "fgather": 11,
         "fstep": 12, "fpush": 13, "bgather": 14, "bstep": 15, "fsum": 16, "perm": 17}


def sym_profile(h, mode):
    return _check(load().sym_profile(h, int(mode)))


def sym_profile_launches(h, which=0):
    """Per-launch milliseconds of the last profiled factor (which=0) or solve (which=1)."""
    lib = load()
    cnt = lib.sym_profile_launches(h, int(which), None)
    if cnt < 0:
        _check(int(cnt))
    out = np.zeros(max(int(cnt), 0), dtype=np.float64)
    if cnt:
        _check(int(lib.sym_profile_launches(h, int(which), out.ctypes.data)))
    return out


def sym_profile_read(h, kind):
    """(milliseconds, launches, algorithmic flops) accumulated for one kernel kind."""
    ms, nl, fl = ct.c_double(), ct.c_int64(), ct.c_double()
    _check(load().sym_profile_read(h, int(kind), ct.byref(ms), ct.byref(nl), ct.byref(fl)))
    return ms.value, nl.value, fl.value


def sym_fma_peak(precision=64):
    g = ct.c_double()
    _check(load().sym_fma_peak(int(precision), ct.byref(g)))
    return g.value


def sym_tc_probe(A, B, lbo=128, sbo=1024):
    """D = A B^T through one tcgen05 kind::tf32 tile product (A: 128 x 32, B: 64 x 32 float32)."""
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    if A.shape != (128, 32) or B.shape != (64, 32):
        raise ValueError("A must be 128 x 32 and B 64 x 32")
    D = np.empty((128, 64), dtype=np.float32)
    _check(load().sym_tc_probe(A.ctypes.data, B.ctypes.data, D.ctypes.data, int(lbo), int(sbo)))
    return D


def sym_set_refinement(h, tol, max_iter):
    return _check(load().sym_set_refinement(h, float(tol), int(max_iter)))


def sym_refinement_info(h):
    """(iterations, backward error) of the last mixed-precision solve."""
    it, be = ct.c_int32(), ct.c_double()
    _check(load().sym_refinement_info(h, ct.byref(it), ct.byref(be)))
    return it.value, be.value


def sym_pivot_info(h, index=0):
    """(min_k d_k / C_kk, its column, breakdown flag) of the last mixed-precision factorization."""
    r, col, bd = ct.c_double(), ct.c_int64(), ct.c_int32()
    _check(load().sym_pivot_info(h, int(index), ct.byref(r), ct.byref(col), ct.byref(bd)))
    return r.value, col.value, bool(bd.value)


def sym_set_pivot_threshold(h, threshold):
    return _check(load().sym_set_pivot_threshold(h, float(threshold)))


def sym_autotune(h, nbatch, Ax, stride, reps=3):
    """Time both kernel forms of a batch's tunable launches and keep the faster; returns
    (tunable launches, launches switched to their second form)."""
    tuned, changed = ct.c_int32(), ct.c_int32()
    _check(load().sym_autotune(h, int(nbatch), _dptr(Ax), int(stride), int(reps), ct.byref(tuned),
                               ct.byref(changed)))
    return tuned.value, changed.value


def sym_set_tc_wait(h, limit_ns, withhold_mma=0):
    return _check(load().sym_set_tc_wait(h, int(limit_ns), int(withhold_mma)))


def sym_factor_batch(h, nbatch, Ax, stride):
    """Ax: device tensor (nbatch, stride) or address; matrix b's values at Ax + b * stride."""
    return _check(load().sym_factor_batch(h, int(nbatch), _dptr(Ax), int(stride)))


def sym_batch_error_columns(h, nbatch):
    out = np.zeros(nbatch, dtype=np.int64)
    _check(load().sym_batch_error_columns(h, out.ctypes.data))
    return out


def sym_solve_batch(h, nbatch, nrhs, B, ldb, bstride, X, ldx, xstride):
    return _check(load().sym_solve_batch(h, int(nbatch), int(nrhs), _dptr(B), int(ldb), int(bstride), _dptr(X),
                                         int(ldx), int(xstride)))


def sym_get_batch_factor_host(h, index):
    st = sym_info(h)
    out = np.zeros(st.storage_l, dtype=np.float64)
    _check(load().sym_get_batch_factor_host(h, int(index), out.ctypes.data))
    return out


class MLP:
    """The cost model network (owning wrapper of sym_mlp); X and t are torch CUDA float32 tensors."""

    def __init__(self, nin, hidden, seed=0):
        self.nin, self.hidden = int(nin), int(hidden)
        m = ct.c_void_p()
        _check(load().sym_mlp_create(self.nin, self.hidden, ct.c_uint64(seed), ct.byref(m)))
        self.m = m
        self.nparams = int(load().sym_mlp_nparams(m))

    def get_params(self):
        out = np.zeros(self.nparams, dtype=np.float32)
        _check(load().sym_mlp_get_params(self.m, out.ctypes.data))
        return out

    def set_params(self, theta):
        theta = np.ascontiguousarray(theta, dtype=np.float32)
        assert theta.size == self.nparams
        _check(load().sym_mlp_set_params(self.m, theta.ctypes.data))

    def predict(self, X):
        y = X.new_empty(X.shape[0])
        _check(load().sym_mlp_predict(self.m, X.shape[0], _dptr(X), _dptr(y)))
        return y

    def gradient(self, X, t):
        g = np.zeros(self.nparams, dtype=np.float32)
        loss = ct.c_float()
        _check(load().sym_mlp_gradient(self.m, X.shape[0], _dptr(X), _dptr(t), g.ctypes.data, ct.byref(loss)))
        return g, loss.value

    def train(self, X, t, steps, lr):
        loss = ct.c_float()
        _check(load().sym_mlp_train(self.m, X.shape[0], _dptr(X), _dptr(t), int(steps), ct.c_float(lr), ct.byref(loss)))
        return loss.value

    def close(self):
        if self.m:
            load().sym_mlp_free(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Reach:
    """Reach set of a sparse right-hand-side pattern (owning wrapper of sym_reach)."""

    def __init__(self, h, bidx):
        self.h = h
        self.bidx = np.ascontiguousarray(bidx, dtype=np.int32)
        r = ct.c_void_p()
        _check(load().sym_reach_analyze(h, self.bidx.size, self.bidx.ctypes.data, ct.byref(r)))
        self.r = r

    def size(self):
        return _check(load().sym_reach_size(self.r))

    def indices(self):
        out = np.zeros(self.size(), dtype=np.int32)
        if out.size:
            _check(load().sym_reach_indices(self.r, out.ctypes.data))
        return out

    def export(self, what):
        lib = load()
        cnt = _check(lib.sym_reach_export(self.r, int(what), None))
        out = np.zeros(cnt, dtype=np.int32)
        if cnt:
            _check(lib.sym_reach_export(self.r, int(what), out.ctypes.data))
        return out

    def solve(self, bvals, xvals):
        """Device tensors: bvals (len(bidx)), xvals (size())."""
        return _check(load().sym_solve_lower_sparse(self.h, self.r, _dptr(bvals), _dptr(xvals)))

    def close(self):
        if self.r:
            load().sym_reach_free(self.r)
            self.r = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sym_info(h):
    s = sym_stats()
    _check(load().sym_info(h, ct.byref(s)))
    return s


def sym_last_error_column(h):
    c = ct.c_int64()
    _check(load().sym_last_error_column(h, ct.byref(c)))
    return c.value


def sym_get_factor_host(h):
    st = sym_info(h)
    out = np.zeros(st.storage_l, dtype=np.float64)
    _check(load().sym_get_factor_host(h, out.ctypes.data))
    return out


def sym_export(h, what):
    code, dt = EXPORTS[what]
    lib = load()
    cnt = _check(lib.sym_export(h, code, None))
    out = np.zeros(cnt, dtype=dt)
    if cnt:
        _check(lib.sym_export(h, code, out.ctypes.data))
    return out


def sym_free(h):
    if h:
        load().sym_free(h)


class Solver:
    """Owning wrapper of one handle: analyze on construction, free on close."""

    def __init__(self, n, Ap, Ai, perm=None, opt=None, host_only=False, precision=None, flags=0, ordering=None,
                 rules=None):
        """perm: a fill-reducing ordering (SYM_ORDER_GIVEN); ordering="auto" lets the inspector
        compute one (SYM_ORDER_AUTO); rules = (table, fund_rule): one amalgamation rule per
        fundamental supernode (sym_analyze_rules)."""
        if opt is None:
            opt = sym_options_default()
        opt.flags |= int(flags)
        if precision is not None:
            opt.precision = SYM_PREC_MIXED if precision in ("mixed", SYM_PREC_MIXED) else SYM_PREC_FP64
        if perm is not None:
            opt.ordering = SYM_ORDER_GIVEN
        if ordering in ("auto", SYM_ORDER_AUTO):
            opt.ordering = SYM_ORDER_AUTO
            perm = None
        if host_only:
            opt.flags |= SYM_FLAG_HOST_ONLY
        self.n = int(n)
        if rules is not None:
            self.h = sym_analyze_rules(n, Ap, Ai, perm, opt, rules[0], rules[1])
        else:
            self.h = sym_analyze_perm(n, Ap, Ai, perm, opt)

    def info(self):
        return sym_info(self.h)

    def export(self, what):
        return sym_export(self.h, what)

    def set_stream(self, stream):
        sym_set_stream(self.h, stream)

    def factor(self, Ax):
        return sym_factor(self.h, Ax)

    def factor_async(self, Ax):
        return sym_factor_async(self.h, Ax)

    def status(self):
        return sym_status(self.h)

    def factor_host(self, Ax):
        return sym_factor_host(self.h, Ax)

    def solve(self, B, X=None):
        """Device solve. B, X: torch float64 tensors of shape (n,) or (nrhs, n) rows = columns
        of the column-major block (each row of the tensor is one right-hand side)."""
        if X is None:
            X = B.new_empty(B.shape)
        if B.dim() == 1:
            sym_solve(self.h, B, X)
        else:
            sym_solve_multi(self.h, B.shape[0], B, B.stride(0), X, X.stride(0))
        return X

    def solve_host(self, B):
        return sym_solve_host(self.h, B)

    def factor_panels(self):
        return sym_get_factor_host(self.h)

    def profile(self, mode):
        sym_profile(self.h, mode)

    def profile_read(self, kind):
        return sym_profile_read(self.h, KINDS[kind] if isinstance(kind, str) else kind)

    def set_refinement(self, tol, max_iter):
        sym_set_refinement(self.h, tol, max_iter)

    def refinement_info(self):
        return sym_refinement_info(self.h)

    def pivot_info(self, index=0):
        return sym_pivot_info(self.h, index)

    def error_column(self):
        return sym_last_error_column(self.h)

    def close(self):
        if self.h:
            sym_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
