"""ctypes front end of the plain C oracle (``lair_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``. The product path never loads it.

The oracle is FP64 C compiled with ``-ffp-contract=off`` so that only the explicit
``fma()`` calls of the source fuse operations. Built with OpenMP where the compiler
has it: loops over independent rows, C points and index blocks may then use several
host threads (``set_threads``); every result is bit-identical for any thread count.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lair_oracle.c")
LIB = os.path.join(HERE, "liblair_oracle.so")

CF_F, CF_C = 0, 1
CF_RS, CF_PMIS, CF_USER, CF_AUTO = 0, 1, 2, 3
P_LAIP, P_ONEPOINT = 0, 1
R_LAIR, R_NEUMANN = 0, 1
RELAX_FFC, RELAX_FCF, RELAX_FF = 0, 1, 2
STATUS = {0: "OK", 1: "ARG", 5: "ZERO_DIAG", 6: "STALLED", 7: "NOT_CONVERGED", 8: "NAN", 9: "OOM"}


def build(force: bool = False) -> str:
    """Compile the oracle (portable flags only: the same source builds on x86_64 and aarch64;
    no -march=native, so the same code runs on both). OpenMP if gcc has it, else serial."""
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-o", LIB, SRC, "-lm"]
        r = subprocess.run(base[:1] + ["-fopenmp"] + base[1:], capture_output=True, text=True)
        if r.returncode != 0:
            subprocess.run(base, check=True)
    return LIB


def set_threads(t: int | None = None) -> int:
    """Host threads for the oracle's independent loops (None: every core); returns the count in use."""
    lib().ora_set_threads(0 if t is None else int(t))
    return threads()


def threads() -> int:
    return int(lib().ora_get_threads())


class Opts(C.Structure):
    _fields_ = [
        ("cf_mode", C.c_int), ("cf_user", C.c_void_p), ("distance", C.c_int),
        ("theta", C.c_double), ("theta_cf", C.c_double), ("strength_abs", C.c_int),
        ("interp", C.c_int), ("relax", C.c_int), ("lump_tol", C.c_double), ("lump_level0", C.c_int),
        ("prec", C.c_int), ("coarse_max", C.c_int), ("max_levels", C.c_int), ("block_size", C.c_int),
        ("rs_block", C.c_int), ("pmis_seed", C.c_uint64), ("seg", C.c_void_p), ("nseg", C.c_int),
        ("restriction", C.c_int), ("nodal", C.c_int),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(LIB)
        p = C.c_void_p
        L.ora_setup.restype = p
        L.ora_setup.argtypes = [C.c_int64, p, p, p, C.POINTER(Opts), C.POINTER(C.c_int)]
        L.ora_free.argtypes = [p]
        L.ora_opts_default.argtypes = [C.POINTER(Opts)]
        L.ora_nlevels.argtypes = [p]
        L.ora_singular_count.restype = C.c_int64
        L.ora_singular_count.argtypes = [p, C.c_int]
        L.ora_level_info.argtypes = [p, C.c_int, p]
        L.ora_export_csr.argtypes = [p, C.c_int, C.c_int, p, p, p]
        L.ora_export_cf.argtypes = [p, C.c_int, p, p, p, p]
        L.ora_solve.restype = C.c_int
        L.ora_solve.argtypes = [p, p, p, C.c_double, C.c_int, C.c_int, C.c_int,
                                C.POINTER(C.c_int), C.POINTER(C.c_double), p, C.c_int]
        L.ora_precond_apply.argtypes = [p, p, p]
        L.ora_strength.argtypes = [C.c_int64, p, p, p, C.c_double, C.c_int, p]
        L.ora_cf_split.argtypes = [C.c_int64, p, p, p, C.c_int, C.c_uint64, p]
        L.ora_local_solve.restype = C.c_int
        L.ora_local_solve.argtypes = [C.c_int64, p, p, p]
        L.ora_local_solve_f32.restype = C.c_int
        L.ora_local_solve_f32.argtypes = [C.c_int64, p, p, p]
        L.ora_pmis_weight.restype = C.c_double
        L.ora_pmis_weight.argtypes = [C.c_int64, C.c_int64, C.c_uint64]
        L.ora_block_scale_nnz.restype = C.c_int64
        L.ora_block_scale_nnz.argtypes = [C.c_int64, p, p, C.c_int64]
        L.ora_block_scale.restype = C.c_int
        L.ora_block_scale.argtypes = [C.c_int64, p, p, p, C.c_int64, p, p, p, p]
        L.ora_solve_batched.restype = C.c_int
        L.ora_solve_batched.argtypes = [p, p, p, C.c_double, C.c_int, p, p]
        L.ora_export_seg.argtypes = [p, C.c_int, p]
        L.ora_solve_batched_fgmres.restype = C.c_int
        L.ora_solve_batched_fgmres.argtypes = [p, p, p, C.c_double, C.c_int, C.c_int, p, p]
        L.ora_transpose.restype = C.c_int64
        L.ora_refresh.restype = C.c_int
        L.ora_refresh.argtypes = [p, C.c_int64, p, p, p]
        L.ora_transpose.argtypes = [C.c_int64, p, p, p, p, p, p]
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_get_threads.restype = C.c_int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _csr_arrays(A):
    rp = np.ascontiguousarray(A.row_ptr, np.int64)
    col = np.ascontiguousarray(A.col, np.int32)
    val = np.ascontiguousarray(A.val, np.float64)
    return rp, col, val


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().ora_opts_default(C.byref(o))
    for k, v in kw.items():
        if k == "cf_user":
            continue
        setattr(o, k, v)
    return o


@dataclass
class Level:
    n: int
    A: tuple               # (rp, col, val)
    cf: np.ndarray | None
    strong: np.ndarray | None
    R: tuple | None
    P: tuple | None
    ls_R: np.ndarray | None
    ls_P: np.ndarray | None

    @property
    def nc(self):
        return None if self.R is None else len(self.R[0]) - 1


class Hierarchy:
    """An oracle hierarchy: ``Hierarchy(A, **opts)``; ``levels`` holds host copies."""

    def __init__(self, A, cf_user=None, seg=None, **kw):
        L = lib()
        self.opts = default_opts(**kw)
        self._keep = []
        if seg is not None:
            sg = np.ascontiguousarray(seg, np.int64)
            self._keep.append(sg)
            self.opts.seg = sg.ctypes.data
            self.opts.nseg = len(sg) - 1
        if cf_user is not None:
            cfu = np.ascontiguousarray(cf_user, np.int8)
            self._keep.append(cfu)
            self.opts.cf_user = cfu.ctypes.data
            self.opts.cf_mode = CF_USER
        rp, col, val = _csr_arrays(A)
        st = C.c_int(0)
        self.h = L.ora_setup(A.n, _ptr(rp), _ptr(col), _ptr(val), C.byref(self.opts), C.byref(st))
        self.status = st.value
        self.n = A.n
        self.levels = []
        if self.status == 0:
            self._export()

    def _export(self):
        L = lib()
        nl = L.ora_nlevels(self.h)
        for l in range(nl):
            info = np.zeros(8, np.int64)
            L.ora_level_info(self.h, l, _ptr(info))
            n, nnz, nc, nr_, np_, has_cf = (int(v) for v in info[:6])
            A = (np.zeros(n + 1, np.int64), np.zeros(nnz, np.int32), np.zeros(nnz))
            L.ora_export_csr(self.h, l, 0, *(_ptr(a) for a in A))
            cf = strong = lsr = lsp = R = P = None
            if has_cf:
                cf = np.zeros(n, np.int8)
                strong = np.zeros(nnz, np.uint8)
                if nc > 0 and nr_ > 0:
                    lsr = np.zeros(nc, np.uint8)
                    lsp = np.zeros(nc, np.uint8)
                L.ora_export_cf(self.h, l, _ptr(cf), _ptr(strong), _ptr(lsr), _ptr(lsp))
                if nr_ > 0:
                    R = (np.zeros(nc + 1, np.int64), np.zeros(nr_, np.int32), np.zeros(nr_))
                    P = (np.zeros(n + 1, np.int64), np.zeros(np_, np.int32), np.zeros(np_))
                    L.ora_export_csr(self.h, l, 1, *(_ptr(a) for a in R))
                    L.ora_export_csr(self.h, l, 2, *(_ptr(a) for a in P))
            self.levels.append(Level(n, A, cf, strong, R, P, lsr, lsp))

    def refresh(self, A):
        """New values of the set-up matrix's pattern: every value of the hierarchy is recomputed with
        the splittings, neighbourhoods and patterns kept. Returns the oracle status."""
        rp, col, val = _csr_arrays(A)
        self.status = lib().ora_refresh(self.h, A.n, _ptr(rp), _ptr(col), _ptr(val))
        self.levels = []
        if self.status == 0:
            self._export()
        return self.status

    def singular_count(self, which=0):
        return int(lib().ora_singular_count(self.h, which))

    def precond(self, b):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b)
        lib().ora_precond_apply(self.h, _ptr(b), _ptr(x))
        return x

    def solve(self, b, x0=None, tol=1e-8, cycle=1, max_iter=500, restart=30, hist_cap=2048):
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b) if x0 is None else np.array(x0, np.float64, copy=True)
        it = C.c_int(0)
        rel = C.c_double(0)
        hist = np.zeros(hist_cap)
        st = lib().ora_solve(self.h, _ptr(b), _ptr(x), tol, cycle, max_iter, restart,
                             C.byref(it), C.byref(rel), _ptr(hist), hist_cap)
        nh = min(hist_cap, it.value + 1 if cycle == 0 else hist_cap)
        return x, dict(status=st, iters=it.value, rel=rel.value, hist=hist[:nh])

    def solve_batched(self, b, tol=1e-8, max_iter=500, cycle=0, restart=30):
        """Per-system solves of a batch (systems given by seg at set-up): stationary refinement
        (cycle 0) or FGMRES per system (cycle 1)."""
        b = np.ascontiguousarray(b, np.float64)
        x = np.zeros_like(b)
        nseg = self.opts.nseg
        its = np.zeros(nseg, np.int32)
        rel = np.zeros(nseg)
        if cycle == 0:
            st = lib().ora_solve_batched(self.h, _ptr(b), _ptr(x), tol, max_iter, _ptr(its), _ptr(rel))
        else:
            st = lib().ora_solve_batched_fgmres(self.h, _ptr(b), _ptr(x), tol, max_iter, restart, _ptr(its), _ptr(rel))
        return x, dict(status=st, iters=its, rel=rel)

    def seg(self, level):
        out = np.zeros(self.opts.nseg + 1, np.int64)
        lib().ora_export_seg(self.h, level, _ptr(out))
        return out

    def close(self):
        if getattr(self, "h", None):
            lib().ora_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------------
# stand-alone steps (pins)
# ---------------------------------------------------------------------------------

def strength(A, theta, absmode=False):
    rp, col, val = _csr_arrays(A)
    out = np.zeros(len(col), np.uint8)
    lib().ora_strength(A.n, _ptr(rp), _ptr(col), _ptr(val), theta, int(absmode), _ptr(out))
    return out


def cf_split(A, mask, mode=CF_RS, seed=0x5EED):
    """mode CF_RS, CF_PMIS (seed = hash seed) or CF_AUTO (blocked first pass, seed = block size)."""
    rp, col, _ = _csr_arrays(A)
    mask = np.ascontiguousarray(mask, np.uint8)
    cf = np.zeros(A.n, np.int8)
    lib().ora_cf_split(A.n, _ptr(rp), _ptr(col), _ptr(mask), mode, seed, _ptr(cf))
    return cf


def local_solve(M, rhs, f32=False):
    s = len(rhs)
    if f32:
        Mc = np.array(M, np.float32, order="C", copy=True)
        r = np.array(rhs, np.float32, copy=True)
        z = np.zeros(s, np.float32)
        ls = lib().ora_local_solve_f32(s, _ptr(Mc), _ptr(r), _ptr(z))
    else:
        Mc = np.array(M, np.float64, order="C", copy=True)
        r = np.array(rhs, np.float64, copy=True)
        z = np.zeros(s)
        ls = lib().ora_local_solve(s, _ptr(Mc), _ptr(r), _ptr(z))
    return z, bool(ls)


def pmis_weight(lam, i, seed):
    return lib().ora_pmis_weight(lam, i, seed)


def block_scale(A, bs):
    rp, col, val = _csr_arrays(A)
    nnz = lib().ora_block_scale_nnz(A.n, _ptr(rp), _ptr(col), bs)
    orp = np.zeros(A.n + 1, np.int64)
    ocol = np.zeros(nnz, np.int32)
    oval = np.zeros(nnz)
    dinv = np.zeros(A.n * bs)
    st = lib().ora_block_scale(A.n, _ptr(rp), _ptr(col), _ptr(val), bs, _ptr(orp), _ptr(ocol), _ptr(oval), _ptr(dinv))
    return st, (orp, ocol, oval), dinv.reshape(A.n // bs, bs, bs)


def transpose(A):
    rp, col, val = _csr_arrays(A)
    trp = np.zeros(A.n + 1, np.int64)
    tcol = np.zeros(len(col), np.int32)
    tval = np.zeros(len(col))
    lib().ora_transpose(A.n, _ptr(rp), _ptr(col), _ptr(val), _ptr(trp), _ptr(tcol), _ptr(tval))
    return trp, tcol, tval
