"""Thin Python binding of ``libopm_bsr.so`` (C ABI in ``include/opm_bsr.h``).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  Functions keep the C names (``opm_bsr_create``,
``opm_ilu0_factor``, ``opm_bicgstab_solve`` ...).  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); PyTorch supplies device memory
and streams only.  If the compiled library is missing, loading raises
``ImportError``: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libopm_bsr.so")

OPM_OK = 0
OPM_NOT_CONVERGED = 1
OPM_ERR_ARG = -1
OPM_ERR_PATTERN = -2
OPM_ERR_NO_DIAG = -3
OPM_ERR_ZERO_PIVOT = -4
OPM_ERR_BREAKDOWN = -5
OPM_ERR_NONFINITE = -6
OPM_ERR_OOM = -7
OPM_ERR_TIMEOUT = -8
OPM_ERR_CUDA = -9
OPM_MAX_ROWS = 2147479551  # largest nb a handle or an analysis accepts

SCHEDULES = {"auto": 0, "natural": 1, "level": 2, "colour": 3, "colour_sl": 4, "colour_kempe": 5}
SWEEPS = {"auto": 0, "per_phase": 1, "cooperative": 2}
PRECISIONS = {"fp64": 0, "fp32": 1}

# every symbol include/opm_bsr.h declares
EXPORTS = ["opm_options_default", "opm_bsr_create", "opm_ilu0_factor", "opm_bicgstab_solve",
           "opm_spmv", "opm_ilu_apply", "opm_destroy", "opm_status_str", "opm_last_error_row",
           "opm_get_info", "opm_get_permutation", "opm_get_factors", "opm_get_timing",
           "opm_reset_timing", "opm_bsr_residual_noalloc", "opm_solve_launch", "opm_solve_ready",
           "opm_solve_wait", "opm_batch_create", "opm_batch_factor", "opm_batch_solve", "opm_batch_launch",
           "opm_batch_ready", "opm_batch_wait", "opm_batch_destroy", "opm_autotune", "opm_autotune_batch",
           "opm_bsr_create_jacobi", "opm_set_wells", "opm_gmres_solve", "opm_bsr_analyse",
           "opm_analysis_create", "opm_bsr_create_from_analysis", "opm_analysis_get_info",
           "opm_analysis_destroy"]


class opm_options(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("precision", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("chunk", ctypes.c_int32), ("spin_limit_us", ctypes.c_int32),
                ("debug_skip_item", ctypes.c_int32), ("profile_kernels", ctypes.c_int32),
                ("sweep_launch", ctypes.c_int32), ("small_phase_slices", ctypes.c_int32),
                ("cp_sweeps", ctypes.c_int32), ("tri_sweeps", ctypes.c_int32), ("product_reuse", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


OPM_TUNE_MAX = 24


class opm_tune_entry(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("sweep_launch", ctypes.c_int32), ("chunk", ctypes.c_int32),
                ("small_phase_slices", ctypes.c_int32), ("status", ctypes.c_int32), ("iters", ctypes.c_int32),
                ("ms", ctypes.c_double)]


class opm_tune_report(ctypes.Structure):
    _fields_ = [("ncand", ctypes.c_int32), ("best", ctypes.c_int32), ("cand", opm_tune_entry * OPM_TUNE_MAX)]


class opm_info(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int32), ("schedule", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("nsets", ctypes.c_int32), ("nnzb", ctypes.c_int64), ("nnzb_lower", ctypes.c_int64),
                ("nnzb_upper", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("nphases", ctypes.c_int32), ("rows_identity", ctypes.c_int32), ("nupdates", ctypes.c_int64),
                ("nnzb_product", ctypes.c_int64), ("rows_reuse", ctypes.c_int32), ("reserved2", ctypes.c_int32)]


class opm_analysis_info(ctypes.Structure):
    _fields_ = [("schedule", ctypes.c_int32), ("nsets", ctypes.c_int32), ("nphases", ctypes.c_int32),
                ("rows_identity", ctypes.c_int32), ("nnzb_kept", ctypes.c_int64), ("nnzb_lower", ctypes.c_int64),
                ("nnzb_upper", ctypes.c_int64), ("nupdates", ctypes.c_int64), ("nnzb_product", ctypes.c_int64),
                ("rows_reuse", ctypes.c_int32), ("reserved2", ctypes.c_int32)]


KERNELS = ["factor", "apply", "spmv", "update", "setup", "finish"]


class opm_timing(ctypes.Structure):
    _fields_ = [("setup_ms", ctypes.c_float), ("iterate_ms", ctypes.c_float),
                ("finish_ms", ctypes.c_float), ("factor_ms", ctypes.c_float),
                ("launches", ctypes.c_int64), ("kernel_ms", ctypes.c_double * 6),
                ("kernel_count", ctypes.c_int64 * 6)]

    def kernels(self):
        return {k: (self.kernel_ms[q], self.kernel_count[q]) for q, k in enumerate(KERNELS)}


_lib = None


def lib() -> ctypes.CDLL:
    """Load the compiled library; raise ImportError when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run paper_2309_11488_gb300/build.py (no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
        L.opm_options_default.argtypes = [ctypes.POINTER(opm_options)]
        L.opm_options_default.restype = None
        L.opm_bsr_create.argtypes = [i32, vp, vp, vp, ctypes.POINTER(opm_options), ctypes.POINTER(vp)]
        L.opm_bsr_create_jacobi.argtypes = [i32, vp, vp, vp, vp, ctypes.POINTER(opm_options), ctypes.POINTER(vp)]
        L.opm_bsr_create_jacobi.restype = i32
        L.opm_bsr_analyse.argtypes = [i32, vp, vp, vp, i32, vp, ctypes.POINTER(opm_analysis_info)]
        L.opm_bsr_analyse.restype = i32
        L.opm_analysis_create.argtypes = [i32, vp, vp, vp, i32, ctypes.POINTER(vp)]
        L.opm_analysis_create.restype = i32
        L.opm_bsr_create_from_analysis.argtypes = [vp, vp, ctypes.POINTER(opm_options), ctypes.POINTER(vp)]
        L.opm_bsr_create_from_analysis.restype = i32
        L.opm_analysis_get_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i64), vp,
                                            ctypes.POINTER(opm_analysis_info)]
        L.opm_analysis_get_info.restype = i32
        L.opm_analysis_destroy.argtypes = [vp]
        L.opm_analysis_destroy.restype = None
        L.opm_set_wells.argtypes = [vp, i32, vp, vp, vp, vp, vp]
        L.opm_set_wells.restype = i32
        L.opm_gmres_solve.argtypes = [vp, vp, vp, f64, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(f64)]
        L.opm_gmres_solve.restype = i32
        L.opm_bsr_create.restype = i32
        L.opm_ilu0_factor.argtypes = [vp, vp]
        L.opm_ilu0_factor.restype = i32
        L.opm_bicgstab_solve.argtypes = [vp, vp, vp, f64, i32, ctypes.POINTER(i32), ctypes.POINTER(f64)]
        L.opm_bicgstab_solve.restype = i32
        L.opm_spmv.argtypes = [vp, vp, vp]
        L.opm_spmv.restype = i32
        L.opm_ilu_apply.argtypes = [vp, vp, vp]
        L.opm_ilu_apply.restype = i32
        L.opm_destroy.argtypes = [vp]
        L.opm_destroy.restype = None
        L.opm_status_str.argtypes = [i32]
        L.opm_status_str.restype = ctypes.c_char_p
        L.opm_last_error_row.argtypes = [vp]
        L.opm_last_error_row.restype = i32
        L.opm_get_info.argtypes = [vp, ctypes.POINTER(opm_info)]
        L.opm_get_info.restype = i32
        L.opm_get_permutation.argtypes = [vp, vp]
        L.opm_get_permutation.restype = i32
        L.opm_get_factors.argtypes = [vp, vp, vp]
        L.opm_get_factors.restype = i32
        L.opm_get_timing.argtypes = [vp, ctypes.POINTER(opm_timing)]
        L.opm_get_timing.restype = i32
        L.opm_reset_timing.argtypes = [vp]
        L.opm_reset_timing.restype = i32
        L.opm_bsr_residual_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.opm_bsr_residual_noalloc.restype = i32
        L.opm_solve_launch.argtypes = [vp, vp, vp, vp, f64, i32]
        L.opm_solve_launch.restype = i32
        L.opm_solve_ready.argtypes = [vp]
        L.opm_solve_ready.restype = i32
        L.opm_solve_wait.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(f64)]
        L.opm_solve_wait.restype = i32
        L.opm_batch_create.argtypes = [i32, vp, ctypes.POINTER(opm_options), ctypes.POINTER(vp)]
        L.opm_batch_create.restype = i32
        L.opm_batch_factor.argtypes = [vp, vp, vp]
        L.opm_batch_factor.restype = i32
        L.opm_batch_solve.argtypes = [vp, vp, vp, vp, i32, vp, vp, vp]
        L.opm_batch_solve.restype = i32
        L.opm_batch_launch.argtypes = [vp, vp, vp, vp, vp, i32]
        L.opm_batch_launch.restype = i32
        L.opm_batch_ready.argtypes = [vp]
        L.opm_batch_ready.restype = i32
        L.opm_batch_wait.argtypes = [vp, vp, vp, vp]
        L.opm_batch_wait.restype = i32
        L.opm_batch_destroy.argtypes = [vp]
        L.opm_batch_destroy.restype = None
        L.opm_autotune.argtypes = [i32, vp, vp, vp, vp, f64, i32, i32, ctypes.POINTER(opm_options),
                                   ctypes.POINTER(opm_options), ctypes.POINTER(opm_tune_report)]
        L.opm_autotune.restype = i32
        L.opm_autotune_batch.argtypes = [i32, vp, vp, vp, vp, vp, vp, i32, i32, ctypes.POINTER(opm_options),
                                         ctypes.POINTER(opm_options), ctypes.POINTER(opm_tune_report)]
        L.opm_autotune_batch.restype = i32
        _lib = L
    return _lib


class OpmError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = status
        super().__init__(f"{what}: {opm_status_str(status)} ({status})")


def opm_status_str(status: int) -> str:
    return lib().opm_status_str(status).decode()


def _ptr(a, dtype):
    """Address of a contiguous numpy array or torch tensor of the given dtype."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype) or not a.flags["C_CONTIGUOUS"]:
            raise TypeError(f"expected a C-contiguous {np.dtype(dtype)} array")
        return a.ctypes.data
    # torch tensor
    import torch
    want = {np.float64: torch.float64, np.int32: torch.int32}[np.dtype(dtype).type]
    if a.dtype != want or not a.is_contiguous():
        raise TypeError(f"expected a contiguous {want} tensor")
    return a.data_ptr()


@dataclass
class Handle:
    ptr: int
    nb: int
    nnzb: int

    def __bool__(self):
        return bool(self.ptr)


def opm_options_default(**kw) -> opm_options:
    o = opm_options()
    lib().opm_options_default(ctypes.byref(o))
    for k, v in kw.items():
        if k == "schedule" and isinstance(v, str):
            v = SCHEDULES[v]
        if k == "precision" and isinstance(v, str):
            v = PRECISIONS[v]
        if k == "sweep_launch" and isinstance(v, str):
            v = SWEEPS[v]
        setattr(o, k, v)
    return o


def opm_bsr_create(nb, rowptr, colidx, vals, options: opm_options | None = None, check=True, part=None):
    """Returns (status, Handle or None); with part, opm_bsr_create_jacobi."""
    out = ctypes.c_void_p()
    opt = ctypes.byref(options) if options is not None else None
    if part is None:
        st = lib().opm_bsr_create(int(nb), _ptr(rowptr, np.int32), _ptr(colidx, np.int32), _ptr(vals, np.float64),
                                  opt, ctypes.byref(out))
    else:
        st = lib().opm_bsr_create_jacobi(int(nb), _ptr(rowptr, np.int32), _ptr(colidx, np.int32),
                                         _ptr(vals, np.float64), _ptr(part, np.int32), opt, ctypes.byref(out))
    nnzb = int(rowptr[-1]) if nb >= 0 and len(rowptr) else 0
    h = Handle(out.value or 0, int(nb), nnzb) if out.value else None
    if check and st != OPM_OK:
        if h:
            opm_destroy(h)
        raise OpmError(st, "opm_bsr_create")
    return st, h


def opm_bsr_analyse(nb, rowptr, colidx, schedule="auto", part=None):
    """Host-only symbolic analysis: returns (status, perm, opm_analysis_info)."""
    if isinstance(schedule, str):
        schedule = SCHEDULES[schedule]
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int32)
    colidx = np.ascontiguousarray(colidx, dtype=np.int32)
    pt = None if part is None else np.ascontiguousarray(part, dtype=np.int32)
    perm = np.empty(int(nb) if 0 <= int(nb) <= OPM_MAX_ROWS else 0, dtype=np.int32)
    info = opm_analysis_info()
    st = lib().opm_bsr_analyse(int(nb), rowptr.ctypes.data, colidx.ctypes.data if colidx.size else None,
                               pt.ctypes.data if pt is not None and pt.size else None, int(schedule),
                               perm.ctypes.data if perm.size else None, ctypes.byref(info))
    return st, perm, info


class Analysis:
    """A kept symbolic analysis (opm_analysis_create): handles of its pattern
    are made from it by Solver.from_analysis without analysing again."""

    def __init__(self, nb, rowptr, colidx, schedule="auto", part=None):
        if isinstance(schedule, str):
            schedule = SCHEDULES[schedule]
        out = ctypes.c_void_p()
        self.status = lib().opm_analysis_create(int(nb), _ptr(rowptr, np.int32), _ptr(colidx, np.int32),
                                                _ptr(part, np.int32), int(schedule), ctypes.byref(out))
        self.ptr = out.value or 0
        if self.status != OPM_OK:
            raise OpmError(self.status, "opm_analysis_create")
        nbv, nnzb = ctypes.c_int32(), ctypes.c_int64()
        self.info = opm_analysis_info()
        lib().opm_analysis_get_info(self.ptr, ctypes.byref(nbv), ctypes.byref(nnzb), None, ctypes.byref(self.info))
        self.nb, self.nnzb = nbv.value, nnzb.value

    def permutation(self) -> np.ndarray:
        perm = np.empty(self.nb, dtype=np.int32)
        lib().opm_analysis_get_info(self.ptr, None, None, perm.ctypes.data if self.nb else None, None)
        return perm

    def close(self):
        if self.ptr:
            lib().opm_analysis_destroy(self.ptr)
            self.ptr = 0

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def opm_bsr_create_from_analysis(an: Analysis, vals, options: opm_options | None = None, check=True):
    """Returns (status, Handle or None): a handle of the analysed pattern."""
    out = ctypes.c_void_p()
    opt = ctypes.byref(options) if options is not None else None
    st = lib().opm_bsr_create_from_analysis(an.ptr, _ptr(vals, np.float64), opt, ctypes.byref(out))
    h = Handle(out.value or 0, an.nb, an.nnzb) if out.value else None
    if check and st != OPM_OK:
        if h:
            opm_destroy(h)
        raise OpmError(st, "opm_bsr_create_from_analysis")
    return st, h


def opm_ilu0_factor(h: Handle, vals=None) -> int:
    return lib().opm_ilu0_factor(h.ptr, _ptr(vals, np.float64))


def opm_bicgstab_solve(h: Handle, b, x, rtol=1e-2, maxit=200):
    """Returns (status, iters, relres); x is filled in place."""
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = lib().opm_bicgstab_solve(h.ptr, _ptr(b, np.float64), _ptr(x, np.float64), float(rtol), int(maxit),
                                  ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def opm_spmv(h: Handle, x, y) -> int:
    return lib().opm_spmv(h.ptr, _ptr(x, np.float64), _ptr(y, np.float64))


def opm_ilu_apply(h: Handle, r, z) -> int:
    return lib().opm_ilu_apply(h.ptr, _ptr(r, np.float64), _ptr(z, np.float64))


def opm_destroy(h: Handle | None) -> None:
    if h and h.ptr:
        lib().opm_destroy(h.ptr)
        h.ptr = 0


def opm_last_error_row(h: Handle | None) -> int:
    return lib().opm_last_error_row(h.ptr if h else None)


def opm_get_info(h: Handle) -> opm_info:
    info = opm_info()
    st = lib().opm_get_info(h.ptr, ctypes.byref(info))
    if st != OPM_OK:
        raise OpmError(st, "opm_get_info")
    return info


def opm_get_permutation(h: Handle) -> np.ndarray:
    perm = np.empty(h.nb, dtype=np.int32)
    st = lib().opm_get_permutation(h.ptr, perm.ctypes.data if h.nb else None)
    if st != OPM_OK:
        raise OpmError(st, "opm_get_permutation")
    return perm


def opm_get_factors(h: Handle):
    """(lu (nnzb, 9), dinv (nb, 9)) in the schedule's CSR order."""
    lu = np.empty((h.nnzb, 9))
    dinv = np.empty((h.nb, 9))
    st = lib().opm_get_factors(h.ptr, lu.ctypes.data, dinv.ctypes.data)
    if st != OPM_OK:
        raise OpmError(st, "opm_get_factors")
    return lu, dinv


def opm_get_timing(h: Handle) -> opm_timing:
    t = opm_timing()
    lib().opm_get_timing(h.ptr, ctypes.byref(t))
    return t


def opm_reset_timing(h: Handle) -> int:
    return lib().opm_reset_timing(h.ptr)


def opm_bsr_residual_noalloc(nb, rowptr, colidx, vals, x, b, r, norms, stream=None) -> int:
    """r = b - A x and norms = (||b - A x||, ||b||) on device arrays, without
    allocating (see include/opm_bsr.h)."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    return lib().opm_bsr_residual_noalloc(int(nb), _ptr(rowptr, np.int32), _ptr(colidx, np.int32),
                                          _ptr(vals, np.float64), _ptr(x, np.float64), _ptr(b, np.float64),
                                          _ptr(r, np.float64), _ptr(norms, np.float64), stream)


def opm_solve_launch(h: Handle, vals, b, x, rtol=1e-2, maxit=200) -> int:
    """Enqueue an optional refactorisation and a solve without waiting
    (device arrays only; keep them alive until opm_solve_wait)."""
    return lib().opm_solve_launch(h.ptr, _ptr(vals, np.float64), _ptr(b, np.float64), _ptr(x, np.float64),
                                  float(rtol), int(maxit))


def opm_solve_ready(h: Handle) -> bool:
    return bool(lib().opm_solve_ready(h.ptr))


def opm_solve_wait(h: Handle):
    """Returns (status, iters, relres) of the pending launch."""
    it = ctypes.c_int32(0)
    rr = ctypes.c_double(0.0)
    st = lib().opm_solve_wait(h.ptr, ctypes.byref(it), ctypes.byref(rr))
    return st, it.value, rr.value


def _ptr_array(arrays, dtype):
    if arrays is None:
        return None, None
    addrs = (ctypes.c_void_p * len(arrays))(*[_ptr(a, dtype) for a in arrays])
    return addrs, arrays


class Batch:
    """A set of handles factorised and solved together (see include/opm_bsr.h)."""

    def __init__(self, handles, stream=None, chunk=0, sweep_launch="auto", small_phase_slices=0, cp_sweeps=0,
                 tri_sweeps=0, product_reuse=0):
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        self.handles = list(handles)
        hs = (ctypes.c_void_p * len(self.handles))(*[h.ptr for h in self.handles])
        o = opm_options_default(stream=stream, chunk=chunk, sweep_launch=sweep_launch,
                                small_phase_slices=small_phase_slices, cp_sweeps=cp_sweeps, tri_sweeps=tri_sweeps,
                                product_reuse=product_reuse)
        out = ctypes.c_void_p()
        st = lib().opm_batch_create(len(self.handles), hs, ctypes.byref(o), ctypes.byref(out))
        if st != OPM_OK:
            raise OpmError(st, "opm_batch_create")
        self.ptr = out.value
        self._keep = None

    def __len__(self):
        return len(self.handles)

    def factor(self, vals=None):
        n = len(self)
        va, keep = _ptr_array(vals, np.float64)
        st = (ctypes.c_int32 * n)()
        s = lib().opm_batch_factor(self.ptr, va, st)
        return s, list(st)

    def solve(self, bs, xs, rtol=1e-2, maxit=200):
        n = len(self)
        ba, kb = _ptr_array(bs, np.float64)
        xa, kx = _ptr_array(xs, np.float64)
        rt = (ctypes.c_double * n)(*([rtol] * n if np.isscalar(rtol) else list(rtol)))
        it = (ctypes.c_int32 * n)()
        rr = (ctypes.c_double * n)()
        st = (ctypes.c_int32 * n)()
        s = lib().opm_batch_solve(self.ptr, ba, xa, rt, int(maxit), it, rr, st)
        return s, list(st), list(it), list(rr)

    def launch(self, vals, bs, xs, rtol=1e-2, maxit=200):
        n = len(self)
        va, kv = _ptr_array(vals, np.float64)
        ba, kb = _ptr_array(bs, np.float64)
        xa, kx = _ptr_array(xs, np.float64)
        rt = (ctypes.c_double * n)(*([rtol] * n if np.isscalar(rtol) else list(rtol)))
        self._keep = (va, ba, xa, rt, kv, kb, kx)
        return lib().opm_batch_launch(self.ptr, va, ba, xa, rt, int(maxit))

    def ready(self) -> bool:
        return bool(lib().opm_batch_ready(self.ptr))

    def wait(self):
        n = len(self)
        it = (ctypes.c_int32 * n)()
        rr = (ctypes.c_double * n)()
        st = (ctypes.c_int32 * n)()
        s = lib().opm_batch_wait(self.ptr, it, rr, st)
        self._keep = None
        return s, list(st), list(it), list(rr)

    def close(self):
        if self.ptr:
            lib().opm_batch_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Convenience owner of one handle (context manager)."""

    def __init__(self, nb, rowptr, colidx, vals, schedule="auto", precision="fp64", stream=None, chunk=0,
                 spin_limit_us=0, debug_skip_item=-1, profile_kernels=False, sweep_launch="auto",
                 small_phase_slices=0, part=None, cp_sweeps=0, tri_sweeps=0, product_reuse=0):
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        self.options = opm_options_default(schedule=schedule, precision=precision, stream=stream, chunk=chunk,
                                           spin_limit_us=spin_limit_us, debug_skip_item=debug_skip_item,
                                           profile_kernels=int(bool(profile_kernels)), sweep_launch=sweep_launch,
                                           small_phase_slices=small_phase_slices, cp_sweeps=cp_sweeps,
                                           tri_sweeps=tri_sweeps, product_reuse=product_reuse)
        self.status, self.h = opm_bsr_create(nb, rowptr, colidx, vals, self.options, part=part)
        self.nb = nb

    @classmethod
    def from_analysis(cls, an: Analysis, vals, precision="fp64", stream=None, **kw):
        """A handle of an analysed pattern (opm_bsr_create_from_analysis)."""
        self = cls.__new__(cls)
        if stream is not None and not isinstance(stream, int):
            stream = stream.cuda_stream
        self.options = opm_options_default(precision=precision, stream=stream, **kw)
        self.status, self.h = opm_bsr_create_from_analysis(an, vals, self.options)
        self.nb = an.nb
        return self

    def factor(self, vals=None) -> int:
        return opm_ilu0_factor(self.h, vals)

    def gmres(self, b, x=None, rtol=1e-2, maxit=200, restart=30):
        """opm_gmres_solve; returns (x, status, iters, relres)."""
        if x is None:
            x = np.empty(3 * self.nb) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
        it = ctypes.c_int32()
        rr = ctypes.c_double()
        st = lib().opm_gmres_solve(self.h.ptr, _ptr(b, np.float64), _ptr(x, np.float64), float(rtol), int(maxit),
                                   int(restart), ctypes.byref(it), ctypes.byref(rr))
        return x, st, it.value, rr.value

    def set_wells(self, wells=None) -> int:
        """opm_set_wells from an object with ptr, cells, B, C, Dinv (numpy or
        torch); None removes the wells."""
        if wells is None:
            return lib().opm_set_wells(self.h.ptr, 0, None, None, None, None, None)
        nw = int(wells.ptr.shape[0] - 1)
        return lib().opm_set_wells(self.h.ptr, nw, _ptr(wells.ptr, np.int32), _ptr(wells.cells, np.int32),
                                   _ptr(wells.B, np.float64), _ptr(wells.C, np.float64),
                                   _ptr(wells.Dinv, np.float64))

    def solve(self, b, x=None, rtol=1e-2, maxit=200):
        if x is None:
            x = np.empty(3 * self.nb) if isinstance(b, np.ndarray) else b.new_empty(b.shape)
        st, it, rr = opm_bicgstab_solve(self.h, b, x, rtol, maxit)
        return x, st, it, rr

    def spmv(self, x, y=None):
        if y is None:
            y = np.empty(3 * self.nb) if isinstance(x, np.ndarray) else x.new_empty(x.shape)
        st = opm_spmv(self.h, x, y)
        if st != OPM_OK:
            raise OpmError(st, "opm_spmv")
        return y

    def ilu_apply(self, r, z=None):
        if z is None:
            z = np.empty(3 * self.nb) if isinstance(r, np.ndarray) else r.new_empty(r.shape)
        st = opm_ilu_apply(self.h, r, z)
        if st != OPM_OK:
            raise OpmError(st, "opm_ilu_apply")
        return z

    def info(self):
        return opm_get_info(self.h)

    def permutation(self):
        return opm_get_permutation(self.h)

    def factors(self):
        return opm_get_factors(self.h)

    def timing(self):
        return opm_get_timing(self.h)

    def reset_timing(self):
        return opm_reset_timing(self.h)

    def launch(self, vals, b, x, rtol=1e-2, maxit=200):
        st = opm_solve_launch(self.h, vals, b, x, rtol, maxit)
        if st != OPM_OK:
            raise OpmError(st, "opm_solve_launch")

    def ready(self) -> bool:
        return opm_solve_ready(self.h)

    def wait(self):
        return opm_solve_wait(self.h)

    def close(self):
        opm_destroy(self.h)

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ autotuner

def _tune_result(st, best, rep):
    names = {v: k for k, v in SCHEDULES.items()}
    sweeps = {v: k for k, v in SWEEPS.items()}
    cands = [{"schedule": names[e.schedule], "sweep_launch": sweeps[e.sweep_launch], "chunk": e.chunk,
              "small_phase_slices": e.small_phase_slices, "status": e.status, "iters": e.iters, "ms": e.ms}
             for e in rep.cand[:rep.ncand]]
    kw = {"schedule": names[best.schedule], "sweep_launch": sweeps[best.sweep_launch], "chunk": best.chunk,
          "small_phase_slices": best.small_phase_slices}
    return st, kw, cands, rep.best


def autotune(nb, rowptr, colidx, vals, b, rtol=1e-2, maxit=200, repeats=3, precision="fp64", stream=None):
    """opm_autotune: returns (status, best keyword options for Solver,
    candidates tried, index of the chosen candidate)."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    base = opm_options_default(precision=precision, stream=stream)
    best = opm_options()
    rep = opm_tune_report()
    st = lib().opm_autotune(int(nb), _ptr(rowptr, np.int32), _ptr(colidx, np.int32), _ptr(vals, np.float64),
                            _ptr(b, np.float64), float(rtol), int(maxit), int(repeats), ctypes.byref(base),
                            ctypes.byref(best), ctypes.byref(rep))
    return _tune_result(st, best, rep)


def autotune_batch(systems, rtol=None, maxit=200, repeats=3, precision="fp64", stream=None):
    """opm_autotune_batch over systems = [(nb, rowptr, colidx, vals, b), ...];
    returns (status, best keyword options (schedule for the members' Solver,
    the rest for Batch), candidates tried, index of the chosen candidate)."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    n = len(systems)
    nbs = (ctypes.c_int32 * n)(*[int(s[0]) for s in systems])
    rp, k1 = _ptr_array([s[1] for s in systems], np.int32)
    ci, k2 = _ptr_array([s[2] for s in systems], np.int32)
    va, k3 = _ptr_array([s[3] for s in systems], np.float64)
    bv, k4 = _ptr_array([s[4] for s in systems], np.float64)
    rt = (ctypes.c_double * n)(*rtol) if rtol is not None else None
    base = opm_options_default(precision=precision, stream=stream)
    best = opm_options()
    rep = opm_tune_report()
    st = lib().opm_autotune_batch(n, nbs, rp, ci, va, bv, rt, int(maxit), int(repeats), ctypes.byref(base),
                                  ctypes.byref(best), ctypes.byref(rep))
    return _tune_result(st, best, rep)
