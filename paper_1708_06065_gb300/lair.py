"""Python binding of liblair.so (include/lair.h): argument marshalling only.

Every computation runs inside the CUDA library; this module converts arguments
(numpy arrays for host buffers, torch CUDA tensors for device buffers) into the C
structs and pointers of the ABI and turns status codes into exceptions. Importing
it loads the library and raises if it has not been built: there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblair.so")

LAIR_OK = 0
STATUS_NAMES = ["OK", "INVALID_ARG", "NOT_SQUARE", "UNSORTED_CSR", "DUPLICATE_ENTRY", "ZERO_DIAGONAL",
                "COARSENING_STALLED", "NOT_CONVERGED", "NAN", "OOM", "ARENA_OVERFLOW", "DEVICE_TIMEOUT", "CUDA",
                "UNSUPPORTED"]
CF_RS, CF_PMIS, CF_USER, CF_AUTO = 0, 1, 2, 3
P_LAIP, P_ONEPOINT = 0, 1
R_LAIR, R_NEUMANN = 0, 1
RELAX_FFC, RELAX_FCF, RELAX_FF = 0, 1, 2
FP64, MIXED = 0, 1
STATIONARY, FGMRES = 0, 1


class LairError(RuntimeError):
    def __init__(self, status, msg):
        self.status = status
        super().__init__(f"lair status {STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else status}: {msg}")


class lair_csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p),
                ("val", C.c_void_p), ("on_device", C.c_int)]


class lair_options(C.Structure):
    _fields_ = [("cf_mode", C.c_int), ("cf_user", C.c_void_p), ("distance", C.c_int), ("theta", C.c_double),
                ("theta_cf", C.c_double), ("strength_abs", C.c_int), ("interp", C.c_int), ("relax", C.c_int),
                ("lump_tol", C.c_double), ("lump_level0", C.c_int), ("precision", C.c_int),
                ("coarse_max", C.c_int), ("max_levels", C.c_int), ("block_size", C.c_int),
                ("rs_block", C.c_int), ("pmis_seed", C.c_uint64), ("fgmres_restart", C.c_int),
                ("stream", C.c_void_p), ("timing", C.c_int), ("restriction", C.c_int),
                ("nodal", C.c_int), ("autotune", C.c_int), ("wait_polls", C.c_int)]


class lair_report(C.Structure):
    _fields_ = [("iters", C.c_int), ("final_rel", C.c_double), ("setup_ms", C.c_double), ("solve_ms", C.c_double),
                ("nlevels", C.c_int), ("singular_R", C.c_int64), ("singular_P", C.c_int64),
                ("op_complexity", C.c_double), ("cycle_complexity", C.c_double), ("hist", C.c_void_p),
                ("hist_cap", C.c_int), ("hist_len", C.c_int)]


class lair_kernel_timer(C.Structure):
    _fields_ = [("name", C.c_char * 40), ("launches", C.c_int64), ("total_ms", C.c_double),
                ("bytes_per_launch", C.c_double)]


class lair_level_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("nc", C.c_int64), ("nnz_R", C.c_int64),
                ("nnz_P", C.c_int64), ("is_coarsest", C.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(LIB_PATH)
    p = C.c_void_p
    sig = {
        "lair_options_default": (C.c_int, [C.POINTER(lair_options)]),
        "lair_setup": (C.c_int, [C.POINTER(lair_csr), C.POINTER(lair_options), C.POINTER(p)]),
        "lair_solve": (C.c_int, [p, p, p, C.c_double, C.c_int, C.c_int, C.POINTER(lair_report)]),
        "lair_refresh": (C.c_int, [p, p]),
        "lair_precond_apply": (C.c_int, [p, p, p]),
        "lair_adjoint": (C.c_int, [p, p, p, C.c_double, C.c_int, C.c_int, C.POINTER(lair_report)]),
        "lair_grad_A": (C.c_int, [p, p, p, p]),
        "lair_hierarchy_info": (C.c_int, [p, C.POINTER(lair_level_info), C.c_int, C.POINTER(C.c_int)]),
        "lair_export_csr": (C.c_int, [p, C.c_int, C.c_int, p, p, p]),
        "lair_export_cf": (C.c_int, [p, C.c_int, p, p, p, p]),
        "lair_kernel_launches": (C.c_int64, [p]),
        "lair_kernel_timers": (C.c_int, [p, C.POINTER(lair_kernel_timer), C.c_int, C.POINTER(C.c_int)]),
        "lair_local_solve_noalloc": (C.c_int, [C.c_int64, C.c_int32, p, p, p, p, p]),
        "lair_setup_batched": (C.c_int, [C.POINTER(lair_csr), C.c_int, p, C.POINTER(lair_options), C.POINTER(p)]),
        "lair_solve_batched": (C.c_int, [p, p, p, C.c_double, C.c_int, C.c_int, p, p]),
        "lair_batch_setup_solve": (C.c_int, [C.c_int, C.POINTER(lair_csr), p, p, C.POINTER(lair_options), C.c_double,
                                             C.c_int, C.c_int, p, p]),
        "lair_free": (None, [p]),
        "lair_status_string": (C.c_char_p, [C.c_int]),
        "lair_last_error": (C.c_char_p, [p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()


def _on_device(a):
    """True for a CUDA tensor; numpy arrays and CPU tensors (pinned or not) are host memory."""
    return not isinstance(a, np.ndarray) and bool(getattr(a, "is_cuda", False))


def _ptr(a):
    """Data pointer of a numpy array (host) or a torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _vec(a, n):
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous or a.shape != (n,):
            raise ValueError("vectors must be contiguous float64 of length n")
        return a
    import torch
    if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
        raise ValueError("vectors must be contiguous float64 of length n")
    return a


def options(**kw) -> lair_options:
    o = lair_options()
    lib.lair_options_default(C.byref(o))
    for k, v in kw.items():
        if k == "cf_user":
            continue
        if k == "stream":
            v = v.cuda_stream if hasattr(v, "cuda_stream") else v
        setattr(o, k, v)
    return o


@dataclass
class Report:
    status: int
    iters: int
    final_rel: float
    setup_ms: float
    solve_ms: float
    nlevels: int
    singular_R: int
    singular_P: int
    op_complexity: float
    cycle_complexity: float
    hist: np.ndarray = field(default_factory=lambda: np.zeros(0))


class Hierarchy:
    """An lAIR hierarchy on the GPU: ``Hierarchy(row_ptr, col, val, **options)``.

    row_ptr (int64), col (int32) and val (float64) are numpy arrays (host) or torch
    CUDA tensors (device). Options are the fields of ``lair_options``.
    """

    def __init__(self, row_ptr, col, val, cf_user=None, **kw):
        self._h = C.c_void_p()
        n = len(row_ptr) - 1
        nnz = len(col)
        on_dev = _on_device(row_ptr)
        self._keep = [row_ptr, col, val]
        A = lair_csr(n, nnz, _ptr(row_ptr), _ptr(col), _ptr(val), int(on_dev))
        o = options(**kw)
        if cf_user is not None:
            cfu = np.ascontiguousarray(cf_user, np.int8)
            self._keep.append(cfu)
            o.cf_user = cfu.ctypes.data
            o.cf_mode = CF_USER
        self.n, self.nnz = n, nnz
        self.opts = o
        st = lib.lair_setup(C.byref(A), C.byref(o), C.byref(self._h))
        self._keep = None
        if st != LAIR_OK:
            msg = self.last_error()
            self.close()
            raise LairError(st, msg)

    @classmethod
    def batched(cls, row_ptr, col, val, sys_offsets, **kw):
        """One hierarchy for independent systems stored as one block-diagonal CSR."""
        self = cls.__new__(cls)
        self._h = C.c_void_p()
        self.n, self.nnz = len(row_ptr) - 1, len(col)
        on_dev = _on_device(row_ptr)
        A = lair_csr(self.n, self.nnz, _ptr(row_ptr), _ptr(col), _ptr(val), int(on_dev))
        offs = np.ascontiguousarray(sys_offsets, np.int64)
        self.nsys = len(offs) - 1
        self.opts = options(**kw)
        st = lib.lair_setup_batched(C.byref(A), self.nsys, offs.ctypes.data, C.byref(self.opts), C.byref(self._h))
        if st != LAIR_OK:
            msg = self.last_error()
            self.close()
            raise LairError(st, msg)
        return self

    def solve_batched(self, b, x=None, tol=1e-8, max_iter=500, cycle=STATIONARY, raise_on_nc=False):
        """Per-system solves (stationary refinement or FGMRES); returns (x, iters[nsys], rel[nsys], status)."""
        b = _vec(b, self.n)
        if x is None:
            x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.new_zeros(self.n)
        x = _vec(x, self.n)
        its = np.zeros(self.nsys, np.int32)
        rel = np.zeros(self.nsys)
        st = lib.lair_solve_batched(self._h, _ptr(b), _ptr(x), tol, cycle, max_iter, its.ctypes.data, rel.ctypes.data)
        self._check(st, (LAIR_OK,) if raise_on_nc else (LAIR_OK, 7))
        return x, its, rel, st

    @classmethod
    def from_system(cls, sys_, device=False, **kw):
        if device:
            import torch
            rp = torch.from_numpy(np.ascontiguousarray(sys_.row_ptr, np.int64)).cuda()
            col = torch.from_numpy(np.ascontiguousarray(sys_.col, np.int32)).cuda()
            val = torch.from_numpy(np.ascontiguousarray(sys_.val, np.float64)).cuda()
            return cls(rp, col, val, **kw)
        return cls(np.ascontiguousarray(sys_.row_ptr, np.int64), np.ascontiguousarray(sys_.col, np.int32),
                   np.ascontiguousarray(sys_.val, np.float64), **kw)

    # -- helpers -------------------------------------------------------------------
    def last_error(self):
        return lib.lair_last_error(self._h).decode() if self._h else ""

    def _check(self, st, ok=(LAIR_OK,)):
        if st not in ok:
            raise LairError(st, self.last_error())
        return st

    def close(self):
        if self._h:
            lib.lair_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def launches(self) -> int:
        return int(lib.lair_kernel_launches(self._h))

    # -- calls ---------------------------------------------------------------------
    def _run(self, fn, b, x, tol, cycle, max_iter, hist_cap, raise_on_nc):
        rep = lair_report()
        hist = np.zeros(hist_cap)
        rep.hist = hist.ctypes.data
        rep.hist_cap = hist_cap
        st = fn(self._h, _ptr(b), _ptr(x), tol, cycle, max_iter, C.byref(rep))
        ok = (LAIR_OK,) if raise_on_nc else (LAIR_OK, 7)
        self._check(st, ok)
        return Report(st, rep.iters, rep.final_rel, rep.setup_ms, rep.solve_ms, rep.nlevels, rep.singular_R,
                      rep.singular_P, rep.op_complexity, rep.cycle_complexity, hist[:rep.hist_len].copy())

    def refresh(self, val):
        """New values (numpy or torch float64, nnz entries in the set-up's CSR order) on the set-up's
        pattern: every value of the hierarchy is recomputed, its structure is kept."""
        if isinstance(val, np.ndarray):
            if val.dtype != np.float64 or not val.flags.c_contiguous or val.shape != (self.nnz,):
                raise ValueError("val must be contiguous float64 with nnz entries")
        else:
            import torch
            if val.dtype != torch.float64 or not val.is_contiguous() or val.numel() != self.nnz:
                raise ValueError("val must be contiguous float64 with nnz entries")
        self._check(lib.lair_refresh(self._h, _ptr(val)))

    def solve(self, b, x=None, tol=1e-8, cycle=FGMRES, max_iter=500, hist_cap=4096, raise_on_nc=False):
        """Solve in place into x (numpy or torch, float64); returns (x, Report)."""
        b = _vec(b, self.n)
        if x is None:
            x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.new_zeros(self.n)
        x = _vec(x, self.n)
        rep = self._run(lib.lair_solve, b, x, tol, cycle, max_iter, hist_cap, raise_on_nc)
        return x, rep

    def adjoint(self, g, lam=None, tol=1e-8, cycle=FGMRES, max_iter=500, hist_cap=4096, raise_on_nc=False):
        g = _vec(g, self.n)
        if lam is None:
            lam = np.zeros(self.n) if isinstance(g, np.ndarray) else g.new_zeros(self.n)
        lam = _vec(lam, self.n)
        rep = self._run(lib.lair_adjoint, g, lam, tol, cycle, max_iter, hist_cap, raise_on_nc)
        return lam, rep

    def precond(self, b, x=None):
        b = _vec(b, self.n)
        if x is None:
            x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.new_zeros(self.n)
        self._check(lib.lair_precond_apply(self._h, _ptr(b), _ptr(x)))
        return x

    def grad_A(self, lam, x, out=None):
        if out is None:
            out = np.zeros(self.nnz) if isinstance(lam, np.ndarray) else lam.new_zeros(self.nnz)
        self._check(lib.lair_grad_A(self._h, _ptr(lam), _ptr(x), _ptr(out)))
        return out

    def timers(self):
        """{name: (launches, total_ms, bytes_per_launch)} of the kernels timed with options(timing=1)."""
        cnt = C.c_int(0)
        arr = (lair_kernel_timer * 64)()
        self._check(lib.lair_kernel_timers(self._h, arr, 64, C.byref(cnt)))
        return {arr[i].name.decode(): (int(arr[i].launches), float(arr[i].total_ms), float(arr[i].bytes_per_launch))
                for i in range(min(cnt.value, 64))}

    def info(self):
        nl = C.c_int(0)
        arr = (lair_level_info * 64)()
        self._check(lib.lair_hierarchy_info(self._h, arr, 64, C.byref(nl)))
        return [dict(n=arr[l].n, nnz=arr[l].nnz, nc=arr[l].nc, nnz_R=arr[l].nnz_R, nnz_P=arr[l].nnz_P,
                     coarsest=bool(arr[l].is_coarsest)) for l in range(nl.value)]

    def export_csr(self, level, which):
        inf = self.info()[level]
        if which == 0:
            nr, nnz = inf["n"], inf["nnz"]
        elif which == 1:
            nr, nnz = inf["nc"], inf["nnz_R"]
        else:
            nr, nnz = inf["n"], inf["nnz_P"]
        rp = np.zeros(nr + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz)
        self._check(lib.lair_export_csr(self._h, level, which, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rp, col, val

    def export_cf(self, level):
        inf = self.info()[level]
        cf = np.zeros(inf["n"], np.int8)
        strong = np.zeros(inf["nnz"], np.uint8)
        lsr = np.zeros(max(inf["nc"], 1), np.uint8)
        lsp = np.zeros(max(inf["nc"], 1), np.uint8)
        self._check(lib.lair_export_cf(self._h, level, cf.ctypes.data, strong.ctypes.data, lsr.ctypes.data,
                                       lsp.ctypes.data))
        return cf, strong, lsr[:inf["nc"]], lsp[:inf["nc"]]
