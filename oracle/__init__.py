"""Oracle for the supernodal right-looking Cholesky (arXiv 2409.13090): TEST INFRASTRUCTURE.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of `bench.py`
may import this package. The product path (the CUDA library and its binding)
never loads it, and the oracle shares no code with it.

The arithmetic lives in `oracle.c` (plain C, FP64). This module only compiles
it (`build()`) and marshals numpy arrays in and out through ctypes, except for
the general-graph orderings (`ordering.py`: `nd_graph`, `nd_graph_ml`), which
are plain Python on sets and dicts (small cases only).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/_build/liboracle.so (portable C, no arch flags)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        P = C.c_void_p
        i64, i32, dbl = C.c_int64, C.c_int32, C.c_double
        L.or_nd_grid.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P]
        L.or_analyze.argtypes = [i64, P, P, P, C.c_int, C.c_double, C.POINTER(P)]
        L.or_free.argtypes = [P]
        L.or_factor.argtypes = [P, P]
        L.or_factor.restype = i64
        L.or_solve.argtypes = [P, i64, P, i64, P, i64]
        L.or_backward_error.argtypes = [i64, P, P, P, i64, P, i64, P, i64, P]
        for name in ("or_n", "or_nsuper", "or_nnzL", "or_nblocks", "or_npairs", "or_glbind_len",
                     "or_relind_len", "or_relindB_len"):
            getattr(L, name).argtypes = [P]
            getattr(L, name).restype = i64
        L.or_flops.argtypes = [P]
        L.or_flops.restype = dbl
        L.or_export.argtypes = [P] + [P] * 17
        L.or_export_columns.argtypes = [P, P, P]
        L.or_export_L_supernodal.argtypes = [P, P]
        L.or_export_L_columns.argtypes = [P, P]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


from .ordering import nd_graph, nd_graph_ml  # noqa: E402,F401  (plain Python; no library code)


def nd_grid(nx: int, ny: int, nz: int, leaf: int = 8) -> np.ndarray:
    """Geometric nested-dissection ordering of an nx*ny*nz grid: perm[new] = old."""
    perm = np.empty(nx * ny * nz, dtype=np.int32)
    rc = lib().or_nd_grid(nx, ny, nz, leaf, _p(perm))
    if rc != 0:
        raise RuntimeError(f"or_nd_grid failed: {rc}")
    return perm


@dataclass
class Symbolic:
    n: int
    nsuper: int
    perm: np.ndarray
    sup_ptr: np.ndarray
    sup_parent: np.ndarray
    gl_ptr: np.ndarray
    glbind: np.ndarray
    ri_ptr: np.ndarray
    relind: np.ndarray
    blk_ptr: np.ndarray
    blk_first: np.ndarray
    blk_size: np.ndarray
    blk_owner: np.ndarray
    rb_pair_ptr: np.ndarray
    rb_pair_P: np.ndarray
    rb_val_ptr: np.ndarray
    rb_val: np.ndarray
    level: np.ndarray
    cparent: np.ndarray
    nnzL: int
    flops: float


class Oracle:
    """Handle around the C oracle: analyze (own symbolic pass), factor (Alg. 1), solve, eta."""

    def __init__(self, A, perm0: np.ndarray | None = None, pr: bool = True, merge: float = 0.0):
        self.A = A
        L = lib()
        h = C.c_void_p()
        p0 = None if perm0 is None else np.ascontiguousarray(perm0, dtype=np.int32)
        self._colptr = np.ascontiguousarray(A.colptr, dtype=np.int64)
        self._rowind = np.ascontiguousarray(A.rowind, dtype=np.int32)
        rc = L.or_analyze(A.n, _p(self._colptr), _p(self._rowind), None if p0 is None else _p(p0),
                          1 if pr else 0, float(merge), C.byref(h))
        if rc != 0:
            raise RuntimeError(f"or_analyze failed: {rc}")
        self._h = h
        self.factored = False

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().or_free(self._h)
                self._h = None
        except Exception:
            pass

    def symbolic(self) -> Symbolic:
        L, h = lib(), self._h
        n, ns = L.or_n(h), L.or_nsuper(h)
        nb, npairs = L.or_nblocks(h), L.or_npairs(h)
        a = dict(
            perm=np.empty(n, np.int32), sup_ptr=np.empty(ns + 1, np.int32), sup_parent=np.empty(ns, np.int32),
            gl_ptr=np.empty(ns + 1, np.int64), glbind=np.empty(L.or_glbind_len(h), np.int32),
            ri_ptr=np.empty(ns + 1, np.int64), relind=np.empty(L.or_relind_len(h), np.int32),
            blk_ptr=np.empty(ns + 1, np.int64), blk_first=np.empty(nb, np.int32), blk_size=np.empty(nb, np.int32),
            blk_owner=np.empty(nb, np.int32), rb_pair_ptr=np.empty(ns + 1, np.int64),
            rb_pair_P=np.empty(npairs, np.int32), rb_val_ptr=np.empty(npairs + 1, np.int64),
            rb_val=np.empty(L.or_relindB_len(h), np.int32), level=np.empty(ns, np.int32),
            cparent=np.empty(n, np.int32))
        order = ["perm", "sup_ptr", "sup_parent", "gl_ptr", "glbind", "ri_ptr", "relind", "blk_ptr",
                 "blk_first", "blk_size", "blk_owner", "rb_pair_ptr", "rb_pair_P", "rb_val_ptr", "rb_val",
                 "level", "cparent"]
        L.or_export(h, *[_p(a[k]) for k in order])
        return Symbolic(n=n, nsuper=ns, nnzL=L.or_nnzL(h), flops=L.or_flops(h), **a)

    def columns(self):
        """Column structure of L (final ordering): (colptr int64[n+1], rows int32[nnzL])."""
        L, h = lib(), self._h
        n = L.or_n(h)
        cp = np.empty(n + 1, np.int64)
        rows = np.empty(L.or_nnzL(h), np.int32)
        L.or_export_columns(h, _p(cp), _p(rows))
        return cp, rows

    def factor(self, values: np.ndarray | None = None) -> int:
        v = np.ascontiguousarray(self.A.values if values is None else values, dtype=np.float64)
        info = lib().or_factor(self._h, _p(v))
        self.factored = info == 0
        return int(info)

    def L_columns(self) -> np.ndarray:
        out = np.empty(lib().or_nnzL(self._h), np.float64)
        if lib().or_export_L_columns(self._h, _p(out)) != 0:
            raise RuntimeError("not factored")
        return out

    def L_supernodal(self) -> np.ndarray:
        s = self.symbolic()
        total = int(sum((s.gl_ptr[J + 1] - s.gl_ptr[J]) * (s.sup_ptr[J + 1] - s.sup_ptr[J]) for J in range(s.nsuper)))
        out = np.empty(total, np.float64)
        if lib().or_export_L_supernodal(self._h, _p(out)) != 0:
            raise RuntimeError("not factored")
        return out

    def solve(self, B: np.ndarray) -> np.ndarray:
        B = np.asfortranarray(B, dtype=np.float64)
        if B.ndim == 1:
            B = B.reshape(-1, 1, order="F")
        X = np.zeros_like(B, order="F")
        rc = lib().or_solve(self._h, B.shape[1], _p(B), B.shape[0], _p(X), X.shape[0])
        if rc != 0:
            raise RuntimeError("not factored")
        return X


def backward_error(A, B: np.ndarray, X: np.ndarray) -> np.ndarray:
    """eta_r = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) per right-hand side."""
    B = np.asfortranarray(B, dtype=np.float64)
    X = np.asfortranarray(X, dtype=np.float64)
    if B.ndim == 1:
        B = B.reshape(-1, 1, order="F")
        X = X.reshape(-1, 1, order="F")
    eta = np.empty(B.shape[1], np.float64)
    colptr = np.ascontiguousarray(A.colptr, dtype=np.int64)
    rowind = np.ascontiguousarray(A.rowind, dtype=np.int32)
    values = np.ascontiguousarray(A.values, dtype=np.float64)
    lib().or_backward_error(A.n, _p(colptr), _p(rowind), _p(values), B.shape[1], _p(B), B.shape[0],
                            _p(X), X.shape[0], _p(eta))
    return eta
