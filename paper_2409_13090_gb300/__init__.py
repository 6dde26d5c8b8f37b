"""GB300 supernodal sparse Cholesky (right-looking RL / RLB of arXiv 2409.13090).

Thin Python binding over the C ABI of libsc (include/sc.h): argument
marshalling only. Every step of the numeric path runs in the CUDA library;
there is no Python or CPU fallback -- using the binding without the built
library raises.

    sym = Symbolic(A, ordering="grid_nd")          # sc_analyze  (host)
    num = sym.factor(precision="fp64")              # sc_factor   (GPU)
    X, info = num.solve(B)                          # sc_solve    (GPU)

Inputs may be numpy arrays (host) or torch CUDA tensors (device); torch is
used only for device memory and the current stream.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["Symbolic", "Numeric", "build", "lib", "SCError", "sc_options_default", "sc_analyze",
           "sc_analyze_batch", "sc_symbolic_export", "sc_factor", "sc_refactor", "sc_solve",
           "sc_numeric_export_L", "sc_numeric_free", "sc_symbolic_free", "sc_strerror", "sc_relind_compose"]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "_build", "libsc.so")
_lib = None

SC_OK = 0
SC_ERR_CUDA, SC_ERR_TIMEOUT, SC_ERR_NOT_CONVERGED, SC_ERR_OOM = -101, -102, -103, -104
SC_ERR_IN_USE, SC_ERR_INTERNAL, SC_ERR_UNSUPPORTED, SC_ERR_IO = -105, -106, -107, -108
ORDERING = {"natural": 0, "grid_nd": 1, "user": 2, "graph_nd": 3, "graph_ml": 4}
VARIANT = {"rlb": 0, "rl": 1}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "tf32x3": 3}


class Options(C.Structure):
    _fields_ = [("ordering", C.c_int32), ("grid", C.c_int32 * 3), ("nd_leaf", C.c_int32),
                ("user_perm", C.c_void_p), ("pr", C.c_int32), ("variant", C.c_int32),
                ("precision", C.c_int32), ("chunk", C.c_int32), ("ir_tol", C.c_double),
                ("ir_maxit", C.c_int32), ("pivot_tau", C.c_double), ("spin_limit", C.c_int64),
                ("use_graph", C.c_int32), ("merge_frac", C.c_double), ("tune", C.c_void_p),
                ("deterministic", C.c_int32), ("threads", C.c_int32), ("reserved", C.c_int32 * 2)]


TUNE_FIELDS = ["tile_min_entries", "tile_min_k", "loop_budget", "lookahead", "tc_min_k", "tc_wide_n", "thin_dim",
               "defer_width", "fused", "tc_wide256", "solve_group", "tc_multicast"]


class TuneTable(C.Structure):
    """sc_tune_table: launch-plan settings (0 = library default)."""
    _fields_ = [(f, C.c_int32) for f in TUNE_FIELDS] + [("reserved", C.c_int32 * 2), ("factor_ms", C.c_double)]

    def to_dict(self) -> dict:
        d = {f: getattr(self, f) for f in TUNE_FIELDS}
        d["factor_ms"] = self.factor_ms
        return d

    @classmethod
    def from_dict(cls, d: dict) -> "TuneTable":
        t = cls()
        for f in TUNE_FIELDS:
            setattr(t, f, int(d.get(f, 0)))
        return t


class SymbolicView(C.Structure):
    _fields_ = [("n", C.c_int64), ("nsuper", C.c_int64), ("nnzL", C.c_int64), ("nblocks", C.c_int64),
                ("npairs", C.c_int64), ("flops", C.c_double)] + [
        (name, C.c_void_p) for name in ("perm", "sup_ptr", "sup_parent", "gl_ptr", "glbind", "ri_ptr", "relind",
                                        "blk_ptr", "blk_first", "blk_size", "blk_owner", "rb_pair_ptr",
                                        "rb_pair_P", "rb_val_ptr", "rb_val", "level", "cparent")]


class FactorInfo(C.Structure):
    _fields_ = [("failed_col", C.c_int64), ("precision", C.c_int32), ("pivot_fallbacks", C.c_int32),
                ("flops", C.c_double), ("factor_ms", C.c_double), ("device_bytes", C.c_int64),
                ("kernel_launches", C.c_int32), ("reserved", C.c_int32 * 5)]


class FactorView(C.Structure):
    _fields_ = [("lnz", C.c_void_p), ("elt", C.c_int32), ("precision", C.c_int32), ("size", C.c_int64),
                ("nsuper", C.c_int64), ("panel_off", C.c_void_p), ("panel_ld", C.c_void_p)]


class SolveInfo(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("converged", C.c_int32), ("eta_max", C.c_double),
                ("solve_ms", C.c_double), ("eta", C.c_void_p), ("refine", C.c_int32),
                ("kernel_launches", C.c_int32), ("method", C.c_int32), ("max_iterations", C.c_int32),
                ("copy_in_ms", C.c_float), ("copy_out_ms", C.c_float)]


class SCError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        super().__init__(f"{what}: {sc_strerror(code)} (code {code})" if what else f"{sc_strerror(code)} ({code})")


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def lib():
    """Loads libsc.so (built in-tree by build()); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"libsc is not built ({_LIB_PATH} missing): run paper_2409_13090_gb300.build()")
        L = C.CDLL(_LIB_PATH)
        P, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
        sig = {
            "sc_options_default": ([P], C.c_int),
            "sc_analyze": ([i64, P, P, P, C.POINTER(P)], C.c_int),
            "sc_analyze_batch": ([C.c_int, P, C.POINTER(P)], C.c_int),
            "sc_symbolic_export": ([P, P], C.c_int),
            "sc_relind_compose": ([P, i64, P, i64, P], C.c_int),
            "sc_symbolic_free": ([P], C.c_int),
            "sc_factor": ([P, P, C.c_int, C.c_int, P, C.POINTER(P), P], C.c_int),
            "sc_refactor": ([P, P, C.c_int, P, P], C.c_int),
            "sc_solve": ([P, i64, P, i64, P, i64, C.c_int, P, P], C.c_int),
            "sc_numeric_export_L": ([P, P], C.c_int),
            "sc_numeric_view": ([P, P], C.c_int),
            "sc_numeric_free": ([P], None),
            "sc_factor_profile": ([P, P, C.c_int, P, P, P, P], C.c_int),
            "sc_probe_fma_peak": ([C.c_int, P, P], C.c_int),
            "sc_plan_stats": ([P, C.c_int, P, C.c_int], C.c_int),
            "sc_test_stall_solve": ([P, i64], C.c_int),
            "sc_test_stall_factor": ([P, i64], C.c_int),
            "sc_factor_batch": ([C.c_int, P, P, C.c_int, C.c_int, P, C.POINTER(P), C.POINTER(P), P], C.c_int),
            "sc_tune": ([P, P, C.c_int, C.c_int, C.c_int, P, P, P], C.c_int),
            "sc_check_schedule": ([P, P, C.c_int], C.c_int),
            "sc_symbolic_save": ([P, C.c_char_p], C.c_int),
            "sc_symbolic_load": ([C.c_char_p, C.POINTER(P)], C.c_int),
            "sc_test_perturb_schedule": ([P, C.c_int], C.c_int),
            "sc_strerror": ([C.c_int], C.c_char_p),
            "sc_build_info": ([], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _ptr(a) -> int:
    return a.ctypes.data if isinstance(a, np.ndarray) else int(a.data_ptr())


def _is_device(a) -> bool:
    return not isinstance(a, np.ndarray) and getattr(a, "is_cuda", False)


def _stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:
        pass
    return C.c_void_p(0)


# ------------------------------------------------------------------ raw C ABI names
def sc_options_default() -> Options:
    o = Options()
    lib().sc_options_default(C.byref(o))
    return o


def sc_strerror(code: int) -> str:
    try:
        return lib().sc_strerror(code).decode()
    except Exception:
        return f"error {code}"


def sc_analyze(n, colptr, rowind, opts):
    h = C.c_void_p()
    rc = lib().sc_analyze(n, _ptr(colptr), _ptr(rowind), C.byref(opts), C.byref(h))
    return rc, h


def sc_analyze_batch(handles):
    arr = (C.c_void_p * len(handles))(*[h.value for h in handles])
    h = C.c_void_p()
    rc = lib().sc_analyze_batch(len(handles), arr, C.byref(h))
    return rc, h


def sc_symbolic_export(h):
    v = SymbolicView()
    rc = lib().sc_symbolic_export(h, C.byref(v))
    return rc, v


def sc_relind_compose(rJC, rCP):
    rJC = np.ascontiguousarray(rJC, np.int32)
    rCP = np.ascontiguousarray(rCP, np.int32)
    out = np.empty_like(rJC)
    rc = lib().sc_relind_compose(_ptr(rJC), len(rJC), _ptr(rCP), len(rCP), _ptr(out))
    if rc:
        raise SCError(rc, "sc_relind_compose")
    return out


def sc_symbolic_free(h) -> int:
    return lib().sc_symbolic_free(h)


def sc_factor(sym_h, values, on_device, precision, stream):
    h = C.c_void_p()
    info = FactorInfo()
    rc = lib().sc_factor(sym_h, _ptr(values), int(on_device), precision, stream, C.byref(h), C.byref(info))
    return rc, h, info


def sc_refactor(num_h, values, on_device, stream):
    info = FactorInfo()
    rc = lib().sc_refactor(num_h, _ptr(values), int(on_device), stream, C.byref(info))
    return rc, info


def sc_solve(num_h, nrhs, B, ldb, X, ldx, on_device, stream, info):
    return lib().sc_solve(num_h, nrhs, _ptr(B), ldb, _ptr(X), ldx, int(on_device), stream, C.byref(info))


def sc_numeric_export_L(num_h, out):
    return lib().sc_numeric_export_L(num_h, _ptr(out))


def sc_numeric_free(num_h):
    lib().sc_numeric_free(num_h)


def sc_probe_fma_peak(kind: int, stream=None) -> float:
    """Measured FMA FLOP/s of the current GPU: kind 0 = FP64, 1 = FP32."""
    out = C.c_double()
    rc = lib().sc_probe_fma_peak(kind, _stream(stream), C.byref(out))
    if rc:
        raise SCError(rc, "sc_probe_fma_peak")
    return out.value


# ------------------------------------------------------------------ handles
_VIEW_ARRAYS = [("perm", np.int32, "n"), ("sup_ptr", np.int32, "ns1"), ("sup_parent", np.int32, "ns"),
                ("gl_ptr", np.int64, "ns1"), ("glbind", np.int32, "gl"), ("ri_ptr", np.int64, "ns1"),
                ("relind", np.int32, "ri"), ("blk_ptr", np.int64, "ns1"), ("blk_first", np.int32, "nb"),
                ("blk_size", np.int32, "nb"), ("blk_owner", np.int32, "nb"), ("rb_pair_ptr", np.int64, "ns1"),
                ("rb_pair_P", np.int32, "np"), ("rb_val_ptr", np.int64, "np1"), ("rb_val", np.int32, "rv"),
                ("level", np.int32, "ns"), ("cparent", np.int32, "n")]


def _view_array(addr, dtype, count):
    if count == 0:
        return np.zeros(0, dtype)
    buf = (C.c_byte * (count * np.dtype(dtype).itemsize)).from_address(addr)
    return np.frombuffer(buf, dtype=dtype, count=count).copy()


class Symbolic:
    """Symbolic analysis handle (sc_analyze): ordering, supernodes, PR, blocks, relind(B)."""

    def __init__(self, A=None, *, ordering="natural", grid=None, nd_leaf=8, user_perm=None, pr=True,
                 variant="rlb", precision="fp64", chunk=64, ir_tol=1e-14, ir_maxit=30, use_graph=True,
                 merge=0.0, spin_limit=None, pivot_tau=None, tune=None, deterministic=False, threads=0,
                 _handle=None, _parts=None):
        self._parts = _parts
        if _handle is not None:
            self._h = _handle
            self.n = sc_symbolic_export(_handle)[1].n
            return
        o = sc_options_default()
        o.ordering = ORDERING[ordering]
        g = grid if grid is not None else getattr(A, "grid", (0, 0, 0))
        for i in range(3):
            o.grid[i] = int(g[i]) if g else 0
        o.nd_leaf = nd_leaf
        self._perm_keep = None
        if user_perm is not None:
            self._perm_keep = np.ascontiguousarray(user_perm, np.int32)
            o.user_perm = self._perm_keep.ctypes.data
        o.pr = 1 if pr else 0
        o.variant = VARIANT[variant]
        o.precision = PRECISION[precision]
        o.chunk = chunk
        o.ir_tol = ir_tol
        o.ir_maxit = ir_maxit
        o.use_graph = 1 if use_graph else 0
        o.merge_frac = float(merge)
        o.deterministic = 1 if deterministic else 0
        o.threads = int(threads)
        if spin_limit is not None:
            o.spin_limit = int(spin_limit)
        if pivot_tau is not None:
            o.pivot_tau = float(pivot_tau)
        self._tune_keep = None
        if tune is not None:
            self._tune_keep = TuneTable.from_dict(tune)
            o.tune = C.addressof(self._tune_keep)
        colptr = np.ascontiguousarray(A.colptr, np.int64)
        rowind = np.ascontiguousarray(A.rowind, np.int32)
        rc, h = sc_analyze(A.n, colptr, rowind, o)
        if rc != 0:
            raise SCError(rc, "sc_analyze")
        self._h = h
        self.n = A.n
        self.precision = precision

    @staticmethod
    def factor_batch(syms, values_list, precision="fp64", stream=None):
        """sc_factor_batch: one factorization of many matrices; returns (batch
        Symbolic, Numeric). values_list: one FP64 array per matrix (all numpy,
        or all CUDA tensors)."""
        count = len(syms)
        dev = not isinstance(values_list[0], np.ndarray)
        keep = [v if dev else np.ascontiguousarray(v, np.float64) for v in values_list]
        hs = (C.c_void_p * count)(*[s._h for s in syms])
        vs = (C.c_void_p * count)(*[_ptr(v) for v in keep])
        bsym, h = C.c_void_p(), C.c_void_p()
        info = FactorInfo()
        rc = lib().sc_factor_batch(count, hs, vs, int(dev), PRECISION[precision], _stream(stream), C.byref(bsym),
                                   C.byref(h), C.byref(info))
        if rc < 0:
            raise SCError(rc, "sc_factor_batch")
        b = Symbolic(_handle=bsym, _parts=list(syms))
        num = Numeric.__new__(Numeric)
        num.sym, num._h, num.info, num.rc, num._vals_keep = b, h, info, rc, keep
        return b, num

    @classmethod
    def batch(cls, syms):
        rc, h = sc_analyze_batch([s._h for s in syms])
        if rc != 0:
            raise SCError(rc, "sc_analyze_batch")
        return cls(_handle=h, _parts=list(syms))

    def view(self) -> dict:
        rc, v = sc_symbolic_export(self._h)
        if rc:
            raise SCError(rc, "sc_symbolic_export")
        sizes = {"n": v.n, "ns": v.nsuper, "ns1": v.nsuper + 1, "nb": v.nblocks, "np": v.npairs,
                 "np1": v.npairs + 1}
        out = {"n": v.n, "nsuper": v.nsuper, "nnzL": v.nnzL, "flops": v.flops}
        for name, dt, key in _VIEW_ARRAYS:
            if key in ("gl", "ri", "rv"):
                continue
            out[name] = _view_array(getattr(v, name), dt, sizes[key])
        out["glbind"] = _view_array(v.glbind, np.int32, int(out["gl_ptr"][-1]))
        out["relind"] = _view_array(v.relind, np.int32, int(out["ri_ptr"][-1]))
        out["rb_val"] = _view_array(v.rb_val, np.int32, int(out["rb_val_ptr"][-1]))
        return out

    PLAN_KEYS = ["levels", "chunks", "tasks", "warp_tasks", "tiled_tasks", "simt_tiles", "tc_tiles", "trsm_tiles",
                 "rl_pairs", "loop_items", "thin_units", "split_tiles", "rl_slabs", "tc256_tiles"]

    CHECK_KINDS = {0: "ok", 1: "source range", 2: "target range", 3: "trapezoid", 4: "not an ancestor",
                   5: "level order", 6: "critical flag", 7: "run mapping", 8: "RL pool", 9: "RL relind",
                   10: "plain write outside the own panel", 11: "entry mapping",
                   12: "tensor-core K range", 13: "deterministic plan"}

    def save(self, path) -> None:
        """sc_symbolic_save: the analysis on disk (factor later without analysing again)."""
        rc = lib().sc_symbolic_save(self._h, os.fsencode(path))
        if rc:
            raise SCError(rc, "sc_symbolic_save")

    @classmethod
    def load(cls, path) -> "Symbolic":
        """sc_symbolic_load: a handle from a file written by save()."""
        h = C.c_void_p()
        rc = lib().sc_symbolic_load(os.fsencode(path), C.byref(h))
        if rc:
            raise SCError(rc, "sc_symbolic_load")
        return cls(_handle=h)

    def check_schedule(self) -> dict:
        """sc_check_schedule: host-side bounds / order check of the device schedule."""
        out = np.zeros(5, np.int64)
        rc = lib().sc_check_schedule(self._h, _ptr(out), len(out))
        if rc not in (0, SC_ERR_INTERNAL):
            raise SCError(rc, "sc_check_schedule")
        return {"ok": rc == 0, "tasks": int(out[0]), "loop_products": int(out[1]), "rl_entries": int(out[2]),
                "bad_level": int(out[3]), "kind": self.CHECK_KINDS.get(int(out[4]), str(out[4]))}

    def _perturb_schedule(self, kind: int) -> int:
        return lib().sc_test_perturb_schedule(self._h, int(kind))

    def tune(self, values, precision=None, reps=3, stream=None) -> dict:
        """sc_tune: time candidate launch-plan settings on this matrix and keep
        the fastest in the handle. Returns the table (fields of TUNE_FIELDS,
        factor_ms) and the number of settings timed ("tried")."""
        dev = not isinstance(values, np.ndarray)
        vals = values if dev else np.ascontiguousarray(values, np.float64)
        best = TuneTable()
        tried = C.c_int32(0)
        prec = -1 if precision is None else PRECISION[precision]
        rc = lib().sc_tune(self._h, _ptr(vals), int(dev), prec, int(reps), _stream(stream), C.byref(best),
                           C.byref(tried))
        if rc != 0:
            raise SCError(rc, "sc_tune")
        d = best.to_dict()
        d["tried"] = tried.value
        return d

    def plan_stats(self, precision="fp64") -> dict:
        out = np.zeros(len(self.PLAN_KEYS), np.int64)
        rc = lib().sc_plan_stats(self._h, PRECISION[precision], _ptr(out), len(out))
        if rc:
            raise SCError(rc, "sc_plan_stats")
        return dict(zip(self.PLAN_KEYS, out.tolist()))

    def factor(self, values=None, precision=None, stream=None, A=None) -> "Numeric":
        return Numeric(self, values if values is not None else A.values, precision, stream)

    def free(self):
        if getattr(self, "_h", None):
            rc = sc_symbolic_free(self._h)
            if rc:
                raise SCError(rc, "sc_symbolic_free")
            self._h = None

    def __del__(self):
        try:
            if getattr(self, "_h", None):
                lib().sc_symbolic_free(self._h)
        except Exception:
            pass


class Numeric:
    """Numeric factor on the GPU (sc_factor); solve with sc_solve."""

    def __init__(self, sym: Symbolic, values, precision=None, stream=None):
        self.sym = sym
        prec = -1 if precision is None else PRECISION[precision]
        if isinstance(values, np.ndarray):
            values = np.ascontiguousarray(values, np.float64)
        self._vals_keep = values
        rc, h, info = sc_factor(sym._h, values, _is_device(values), prec, _stream(stream))
        self._h = h if h.value else None
        self.info = info
        self.rc = rc
        if rc < 0:
            raise SCError(rc, "sc_factor")

    @property
    def failed_col(self) -> int:
        return int(self.info.failed_col)

    def refactor(self, values, stream=None) -> FactorInfo:
        if isinstance(values, np.ndarray):
            values = np.ascontiguousarray(values, np.float64)
        rc, info = sc_refactor(self._h, values, _is_device(values), _stream(stream))
        self.info = info
        self.rc = rc
        if rc < 0:
            raise SCError(rc, "sc_refactor")
        return info

    def solve(self, B, X=None, refine=None, stream=None, method="ir", max_iterations=0):
        """Solves A X = B.

        B as a numpy array: n x nrhs (host, column-major). B as a torch tensor
        (CUDA, or pinned/host CPU): shape (nrhs, n) contiguous, i.e. column-major
        n x nrhs; X likewise (allocated when None). method "ir": classical
        refinement; "cg": conjugate gradients preconditioned by the factor.
        max_iterations caps the iterations of this solve (0: the options' cap).
        Returns (X, info); info holds the iterations, convergence, eta per
        right-hand side, the device time of the solve and of its B / X copies
        (solve_ms, copy_in_ms, copy_out_ms) and the kernel launches."""
        if isinstance(B, np.ndarray):
            dev = False
            B = np.asfortranarray(B, np.float64)
            if B.ndim == 1:
                B = B.reshape(-1, 1, order="F")
            nrhs, ldb = B.shape[1], B.shape[0]
            if X is None:
                X = np.zeros_like(B, order="F")
            ldx = X.shape[0]
        else:
            dev = bool(B.is_cuda)
            if B.dim() == 1:
                B = B.reshape(1, -1)
            nrhs, ldb = B.shape[0], B.shape[1]
            if X is None:
                import torch
                X = torch.zeros_like(B)
            ldx = X.shape[1]
        info = SolveInfo()
        eta = np.zeros(nrhs)
        info.eta = eta.ctypes.data
        info.refine = -1 if refine is None else int(bool(refine))
        info.method = {"ir": 0, "cg": 1}[method]
        info.max_iterations = int(max_iterations)
        rc = sc_solve(self._h, nrhs, B, ldb, X, ldx, dev, _stream(stream), info)
        if rc not in (0, SC_ERR_NOT_CONVERGED):
            raise SCError(rc, "sc_solve")
        return X, {"iterations": info.iterations, "converged": bool(info.converged), "eta_max": info.eta_max,
                   "eta": eta, "solve_ms": info.solve_ms, "rc": rc, "kernel_launches": info.kernel_launches,
                "copy_in_ms": info.copy_in_ms, "copy_out_ms": info.copy_out_ms}

    def stall_next_factor(self, chunk: int):
        """Test hook (sc_test_stall_factor): the next refactor's units that read
        `chunk` wait for one completion too many; their bounded waits give up."""
        rc = lib().sc_test_stall_factor(self._h, int(chunk))
        if rc:
            raise SCError(rc, "sc_test_stall_factor")

    def stall_next_solve(self, chunk: int):
        """Test hook (sc_test_stall_solve): the next solve's forward sweep waits at
        `chunk` for an arrival that never comes; its bounded waits give up and the
        solve raises SCError(SC_ERR_TIMEOUT)."""
        rc = lib().sc_test_stall_solve(self._h, int(chunk))
        if rc:
            raise SCError(rc, "sc_test_stall_solve")

    PROFILE_CLASSES = ["value_load", "potrf", "trsm", "gemm_simt", "gemm_tc", "gemm_warp", "rl_update", "rl_assemble",
                       "rlb_loop"]

    def profile(self, values, stream=None) -> dict:
        """One factorization with CUDA events around every launch (sc_factor_profile)."""
        if isinstance(values, np.ndarray):
            values = np.ascontiguousarray(values, np.float64)
        nc = len(self.PROFILE_CLASSES)
        ms, fl = np.zeros(nc), np.zeros(nc)
        ln = np.zeros(nc, np.int32)
        rc = lib().sc_factor_profile(self._h, _ptr(values), _is_device(values), _stream(stream), _ptr(ms),
                                     _ptr(fl), _ptr(ln))
        if rc < 0:
            raise SCError(rc, "sc_factor_profile")
        return {k: {"ms": float(ms[i]), "flops": float(fl[i]), "launches": int(ln[i])}
                for i, k in enumerate(self.PROFILE_CLASSES)}

    def device_view(self) -> dict:
        """sc_numeric_view: the factor storage where it lives. Returns the panel
        offsets and leading dimensions (numpy) and `lnz`, a torch tensor over
        the library's device memory (no copy; valid until the handle is
        refactored or freed). torch takes no read-only flag for foreign device
        memory: the tensor must not be written."""
        import torch
        v = FactorView()
        rc = lib().sc_numeric_view(self._h, C.byref(v))
        if rc:
            raise SCError(rc, "sc_numeric_view")

        class _Mem:  # __cuda_array_interface__ (version 2) over the library's buffer
            __cuda_array_interface__ = {"shape": (int(v.size),), "typestr": "<f8" if v.elt == 8 else "<f4",
                                        "data": (int(v.lnz), False), "version": 2, "strides": None}

        return {"lnz": torch.as_tensor(_Mem(), device="cuda"), "elt": v.elt,
                "panel_off": _view_array(v.panel_off, np.int64, int(v.nsuper)),
                "panel_ld": _view_array(v.panel_ld, np.int32, int(v.nsuper))}

    def export_L(self) -> np.ndarray:
        v = self.sym.view()
        gl, sp = v["gl_ptr"], v["sup_ptr"]
        total = int(np.sum((gl[1:] - gl[:-1]) * (sp[1:] - sp[:-1])))
        out = np.empty(total, np.float64)
        rc = sc_numeric_export_L(self._h, out)
        if rc:
            raise SCError(rc, "sc_numeric_export_L")
        return out

    def free(self):
        if getattr(self, "_h", None):
            sc_numeric_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass
