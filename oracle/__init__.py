"""Plain FP64 CPU oracle for ILU0-preconditioned BiCGStab on 3x3 BSR matrices.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()`` and
the benchmark's CPU-baseline leg import this package; the GPU library and its
Python binding never do, and this package imports nothing from them.

The arithmetic lives in ``oracle.c`` (single-threaded C, ``-O2
-ffp-contract=off``); this module only marshals numpy arrays through ctypes and
assembles dense matrices for brute-force checks.

Section references are to arXiv 2309.11488:
  * SpMV                       -- Section 4.3
  * ILU0 decomposition          -- Section 2.2, Algorithm 2 (block reading:
                                   right product with the inverse pivot block)
  * ILU0 application            -- Section 2.2, Algorithm 1, equations 3-4
  * BiCGStab and stopping rule  -- Section 4.2 (method: van der Vorst 1992,
                                   right preconditioning, x0 = 0)
  * block-Jacobi ILU0           -- Section 4.5 (partition-internal blocks
                                   only; copy by an index vector)
  * standard wells, separate    -- Section 4.6 (y -= C^T inv(D) B x)
  * iterative ILU0, Jacobi      -- Section 3's "Chow Patel ILU0" (Chow & Patel
    triangular solves              2015; Anzt, Chow & Dongarra 2015)
  * restarted GMRES             -- Section 2 names it as OPM's other solver
                                   (method: Saad & Schultz 1986, right
                                   preconditioning, CGS2 Arnoldi)
  * level scheduling / colouring-- Section 4.4 (greedy colouring in natural or
                                   smallest-last order)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")

_i32p = ctypes.POINTER(ctypes.c_int32)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library beside it (plain gcc)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
                               "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = build()
        L = ctypes.CDLL(path)
        L.orc_inv3.argtypes = [_f64p, _f64p]
        L.orc_spmv.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.orc_spmv.restype = None
        L.orc_ilu0.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p]
        L.orc_ilu0_f32.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f32p, _f32p]
        L.orc_ilu_apply.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p]
        L.orc_ilu_apply.restype = None
        L.orc_ilu_apply_f32.argtypes = [ctypes.c_int32, _i32p, _i32p, _f32p, _f32p, _f64p, _f64p]
        L.orc_ilu_apply_f32.restype = None
        L.orc_bicgstab.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f32p, _f32p,
                                   _f64p, _f64p, ctypes.c_double, ctypes.c_int32, _i32p, _f64p, _f64p]
        L.orc_dense_solve.argtypes = [ctypes.c_int32, _f64p, _f64p]
        L.orc_levels.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        L.orc_levels.restype = ctypes.c_int32
        L.orc_colours.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        L.orc_colours.restype = ctypes.c_int32
        L.orc_order_by_key.argtypes = [ctypes.c_int32, _i32p, ctypes.c_int32, _i32p]
        L.orc_order_by_key.restype = None
        L.orc_colours_kempe.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        L.orc_colours_kempe.restype = ctypes.c_int32
        L.orc_ilu0_cp.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, ctypes.c_int32, _f64p, _f64p]
        L.orc_ilu0_cp.restype = ctypes.c_int32
        L.orc_ilu_apply_jacobi.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, ctypes.c_int32]
        L.orc_ilu_apply_jacobi.restype = None
        L.orc_bicgstab_x.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p, _f64p, _f32p,
                                     _f32p, ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, ctypes.c_int32,
                                     _f64p, _f64p, ctypes.c_double, ctypes.c_int32, _i32p, _f64p, _f64p]
        L.orc_bicgstab_x.restype = ctypes.c_int
        L.orc_gmres.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p, ctypes.c_double,
                                ctypes.c_int32, ctypes.c_int32, _i32p, _f64p, _f64p]
        L.orc_gmres.restype = ctypes.c_int
        L.orc_apply_wells.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p]
        L.orc_apply_wells.restype = None
        L.orc_bicgstab_w.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p, _f64p, _f32p,
                                     _f32p, ctypes.c_int32, _i32p, _i32p, _f64p, _f64p, _f64p, _f64p, _f64p,
                                     ctypes.c_double, ctypes.c_int32, _i32p, _f64p, _f64p]
        L.orc_bicgstab_w.restype = ctypes.c_int
        L.orc_bicgstab_pc.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _f64p, _f64p, _f32p,
                                      _f32p, _f64p, _f64p, ctypes.c_double, ctypes.c_int32, _i32p, _f64p, _f64p]
        L.orc_bicgstab_pc.restype = ctypes.c_int
        L.orc_colours_sl.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p]
        L.orc_colours_sl.restype = ctypes.c_int32
        L.orc_closed_first_key.argtypes = [ctypes.c_int32, _i32p, _i32p, _i32p, _i32p]
        L.orc_closed_first_key.restype = None
        L.orc_permute.argtypes = [ctypes.c_int32, _i32p, _i32p, _f64p, _i32p, _i32p, _i32p, _f64p]
        L.orc_permute.restype = None
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t) if a is not None else None


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# ---------------------------------------------------------------------------

def inv3(a):
    a = _f64(a).reshape(9)
    out = np.empty(9)
    st = lib().orc_inv3(_p(a, _f64p), _p(out, _f64p))
    return out.reshape(3, 3), st


def spmv(nb, rowptr, colidx, vals, x):
    rowptr, colidx, vals, x = _i32(rowptr), _i32(colidx), _f64(vals), _f64(x)
    y = np.empty(3 * nb)
    lib().orc_spmv(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(vals, _f64p), _p(x, _f64p), _p(y, _f64p))
    return y


@dataclass
class Factors:
    lu: np.ndarray    # same pattern as A, (nnzb, 9)
    dinv: np.ndarray  # (nb, 9)
    status: int       # 0, or -(1+i) singular pivot at row i, -(1+nb+i) no diagonal in row i
    f32: bool = False


def ilu0(nb, rowptr, colidx, vals, f32=False, cp_sweeps=0) -> Factors:
    """ILU0 factors (Algorithm 2); with cp_sweeps > 0 the fine-grained
    iterative ILU0 of Chow & Patel after that many synchronous sweeps."""
    rowptr, colidx, vals = _i32(rowptr), _i32(colidx), _f64(vals)
    nnzb = int(rowptr[nb])
    if cp_sweeps > 0:
        if f32:
            raise ValueError("the iterative ILU0 is FP64 only")
        lu = np.empty((nnzb, 9))
        dinv = np.empty((nb, 9))
        st = lib().orc_ilu0_cp(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(vals, _f64p), int(cp_sweeps),
                               _p(lu, _f64p), _p(dinv, _f64p))
        return Factors(lu, dinv, int(st), False)
    if f32:
        lu = np.empty((nnzb, 9), dtype=np.float32)
        dinv = np.empty((nb, 9), dtype=np.float32)
        st = lib().orc_ilu0_f32(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(vals, _f64p),
                                _p(lu, _f32p), _p(dinv, _f32p))
    else:
        lu = np.empty((nnzb, 9))
        dinv = np.empty((nb, 9))
        st = lib().orc_ilu0(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(vals, _f64p),
                            _p(lu, _f64p), _p(dinv, _f64p))
    return Factors(lu, dinv, int(st), f32)


def ilu_apply(nb, rowptr, colidx, fac: Factors, r, tri_sweeps=0):
    """z = inv(U) inv(L) r (Algorithm 1); with tri_sweeps > 0 by that many
    Jacobi sweeps per triangle (Anzt, Chow & Dongarra)."""
    rowptr, colidx, r = _i32(rowptr), _i32(colidx), _f64(r)
    z = np.empty(3 * nb)
    if tri_sweeps > 0:
        lib().orc_ilu_apply_jacobi(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(fac.lu, _f64p),
                                   _p(fac.dinv, _f64p), _p(r, _f64p), _p(z, _f64p), int(tri_sweeps))
        return z
    if fac.f32:
        lib().orc_ilu_apply_f32(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(fac.lu, _f32p),
                                _p(fac.dinv, _f32p), _p(r, _f64p), _p(z, _f64p))
    else:
        lib().orc_ilu_apply(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(fac.lu, _f64p),
                            _p(fac.dinv, _f64p), _p(r, _f64p), _p(z, _f64p))
    return z


@dataclass
class SolveResult:
    x: np.ndarray
    status: int      # 0 converged, 1 not converged, -5 breakdown, -6 non-finite rhs
    iters: int
    relres: float    # true ||b - A x|| / ||b||
    res_hist: np.ndarray


def apply_wells(wells, x, y):
    """y -= sum over wells of C^T inv(D) B x (Section 4.6, in place); wells
    is an object with ptr, cells, B, C, Dinv (cells in the numbering of x)."""
    y = _f64(y)
    lib().orc_apply_wells(int(wells.ptr.shape[0] - 1), _p(_i32(wells.ptr), _i32p), _p(_i32(wells.cells), _i32p),
                          _p(_f64(wells.B), _f64p), _p(_f64(wells.C), _f64p), _p(_f64(wells.Dinv), _f64p),
                          _p(_f64(x), _f64p), _p(y, _f64p))
    return y


def spmv_wells(nb, rowptr, colidx, vals, wells, x):
    """y = A x - sum over wells of C^T inv(D) B x."""
    return apply_wells(wells, x, spmv(nb, rowptr, colidx, vals, x))


def bicgstab(nb, rowptr, colidx, vals, fac: Factors, b, rtol=1e-2, maxit=200, mpattern=None,
             wells=None, tri_sweeps=0) -> SolveResult:
    """Right-preconditioned BiCGStab (Section 4.2); the factors live on
    mpattern = (rowptr, colidx) when given (block-Jacobi, Section 4.5), else
    on the matrix's own pattern; with wells (Section 4.6) every product with
    the system operator subtracts their contributions."""
    rowptr, colidx, vals, b = _i32(rowptr), _i32(colidx), _f64(vals), _f64(b)
    mrp, mci = (rowptr, colidx) if mpattern is None else (_i32(mpattern[0]), _i32(mpattern[1]))
    if wells is None:
        nw, wp, wc, wb, wcc, wd = 0, None, None, None, None, None
    else:
        nw = int(wells.ptr.shape[0] - 1)
        wp, wc, wb, wcc, wd = (_i32(wells.ptr), _i32(wells.cells), _f64(wells.B), _f64(wells.C),
                               _f64(wells.Dinv))
    x = np.empty(3 * nb)
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    hist = np.full(2 * maxit + 1, np.nan)
    lu64 = fac.lu if not fac.f32 else None
    d64 = fac.dinv if not fac.f32 else None
    lu32 = fac.lu if fac.f32 else None
    d32 = fac.dinv if fac.f32 else None
    st = lib().orc_bicgstab_x(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(vals, _f64p),
                              _p(mrp, _i32p), _p(mci, _i32p),
                              _p(lu64, _f64p), _p(d64, _f64p), _p(lu32, _f32p), _p(d32, _f32p),
                              nw, _p(wp, _i32p), _p(wc, _i32p), _p(wb, _f64p), _p(wcc, _f64p), _p(wd, _f64p),
                              int(tri_sweeps), _p(b, _f64p), _p(x, _f64p), rtol, maxit, _p(it, _i32p),
                              _p(rr, _f64p), _p(hist, _f64p))
    return SolveResult(x, int(st), int(it[0]), float(rr[0]), hist)


def dense_solve(a, b):
    a = np.array(a, dtype=np.float64, order="C", copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    st = lib().orc_dense_solve(a.shape[0], _p(a, _f64p), _p(b, _f64p))
    return b, st


def levels(nb, rowptr, colidx):
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    lev = np.empty(nb, dtype=np.int32)
    n = lib().orc_levels(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(lev, _i32p))
    return lev, int(n)


def colours(nb, rowptr, colidx):
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    col = np.empty(nb, dtype=np.int32)
    n = lib().orc_colours(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(col, _i32p))
    return col, int(n)


def colours_sl(nb, rowptr, colidx):
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    col = np.empty(nb, dtype=np.int32)
    n = lib().orc_colours_sl(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(col, _i32p))
    return col, int(n)


def colours_kempe(nb, rowptr, colidx):
    """Smallest-last colouring, then the highest colour classes emptied by
    Kempe-chain exchanges while possible (orc_colours_kempe)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    col = np.empty(nb, dtype=np.int32)
    n = lib().orc_colours_kempe(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(col, _i32p))
    return col, int(n)


def order_by_key(key, nkeys):
    key = _i32(key)
    perm = np.empty(key.shape[0], dtype=np.int32)
    lib().orc_order_by_key(key.shape[0], _p(key, _i32p), nkeys, _p(perm, _i32p))
    return perm


def schedule_perm(nb, rowptr, colidx, schedule):
    """perm[new] = old for 'natural', 'level', 'colour', 'colour_sl' or
    'colour_kempe' (Section 4.4):
    set-major; inside a set the closed rows (no neighbour in a later set)
    first; inside each of these groups the rows longer than the most common
    row length last; natural order inside each part.  Returns (perm, number
    of sets)."""
    if schedule == "natural":
        return np.arange(nb, dtype=np.int32), 1
    if schedule == "level":
        key, n = levels(nb, rowptr, colidx)
    elif schedule == "colour":
        key, n = colours(nb, rowptr, colidx)
    elif schedule == "colour_sl":
        key, n = colours_sl(nb, rowptr, colidx)
    elif schedule == "colour_kempe":
        key, n = colours_kempe(nb, rowptr, colidx)
    else:
        raise ValueError(schedule)
    # inside each set: rows without a neighbour in a later set first; inside
    # each of these two groups, rows with more blocks than the most common
    # count (ties to the smaller count) last
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    key2 = np.empty(nb, dtype=np.int32)
    lib().orc_closed_first_key(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(_i32(key), _i32p), _p(key2, _i32p))
    lens = np.diff(rowptr)
    common = int(np.argmax(np.bincount(lens))) if nb else 0
    key3 = 2 * key2 + (lens > common).astype(np.int32)
    return order_by_key(key3, 4 * n), n


def permute(nb, rowptr, colidx, vals, perm):
    rowptr, colidx, vals, perm = _i32(rowptr), _i32(colidx), _f64(vals), _i32(perm)
    nnzb = int(rowptr[nb])
    prow = np.empty(nb + 1, dtype=np.int32)
    pcol = np.empty(nnzb, dtype=np.int32)
    pval = np.empty((nnzb, 9))
    lib().orc_permute(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(vals, _f64p), _p(perm, _i32p),
                      _p(prow, _i32p), _p(pcol, _i32p), _p(pval, _f64p))
    return prow, pcol, pval


def to_dense(nb, rowptr, colidx, vals):
    """Assemble the 3nb x 3nb dense matrix (brute-force checks only)."""
    a = np.zeros((3 * nb, 3 * nb))
    vals = np.asarray(vals).reshape(-1, 3, 3)
    for i in range(nb):
        for m in range(rowptr[i], rowptr[i + 1]):
            j = colidx[m]
            a[3 * i:3 * i + 3, 3 * j:3 * j + 3] = vals[m]
    return a


def gmres(nb, rowptr, colidx, vals, fac: Factors, b, rtol=1e-2, maxit=200, restart=30) -> SolveResult:
    """Restarted GMRES(m), right-preconditioned by the ILU0 factors (see
    orc_gmres: CGS2 Arnoldi, Givens rotations, restart from the true
    residual); res_hist holds ||r_0|| and the estimate after each step."""
    rowptr, colidx, vals, b = _i32(rowptr), _i32(colidx), _f64(vals), _f64(b)
    x = np.empty(3 * nb)
    it = np.zeros(1, dtype=np.int32)
    rr = np.zeros(1)
    hist = np.full(maxit + 1, np.nan)
    st = lib().orc_gmres(nb, _p(rowptr, _i32p), _p(colidx, _i32p), _p(vals, _f64p), _p(fac.lu, _f64p),
                         _p(fac.dinv, _f64p), _p(b, _f64p), _p(x, _f64p), rtol, maxit, restart, _p(it, _i32p),
                         _p(rr, _f64p), _p(hist, _f64p))
    return SolveResult(x, int(st), int(it[0]), float(rr[0]), hist)


def solve_system_gmres(nb, rowptr, colidx, vals, b, rtol=1e-2, maxit=200, restart=30, schedule="natural"):
    """Same-ordering reference for GMRES: ILU0 of P A P^T, GMRES on P A P^T;
    returns (x in natural order, SolveResult, perm)."""
    perm, _ = schedule_perm(nb, rowptr, colidx, schedule)
    prow, pcol, pval = permute(nb, rowptr, colidx, vals, perm)
    fac = ilu0(nb, prow, pcol, pval)
    if fac.status != 0:
        raise ArithmeticError(f"oracle ILU0 failed with status {fac.status}")
    res = gmres(nb, prow, pcol, pval, fac, np.asarray(b).reshape(nb, 3)[perm].ravel(), rtol, maxit, restart)
    x = np.empty(3 * nb)
    x.reshape(nb, 3)[perm] = res.x.reshape(nb, 3)
    return x, res, perm


def jacobi_pattern(nb, rowptr, colidx, vals, part):
    """Block-Jacobi matrix of Section 4.5: the blocks of A that join two rows
    of the same partition (part[i] == part[j]), same rows; its values are
    gathered from A's by an index vector (the paper's copy-indexes loop:
    jvals[k] = vals[indices[k]]).  Returns (rowptr, colidx, vals, indices)."""
    rowptr, colidx = _i32(rowptr), _i32(colidx)
    part = np.asarray(part)
    rows = np.repeat(np.arange(nb), np.diff(rowptr))
    keep = part[rows] == part[colidx]
    indices = np.flatnonzero(keep)
    jrowptr = np.zeros(nb + 1, dtype=np.int32)
    jrowptr[1:] = np.cumsum(np.bincount(rows[keep], minlength=nb))
    jvals = np.asarray(vals).reshape(-1, 9)[indices]
    return jrowptr, colidx[indices].copy(), jvals, indices


def solve_system(nb, rowptr, colidx, vals, b, rtol=1e-2, maxit=200, schedule="natural", f32=False, part=None,
                 wells=None, cp_sweeps=0, tri_sweeps=0):
    """Same-ordering reference: ILU0 + BiCGStab on P A P^T with the oracle's
    own schedule permutation; with part, the preconditioner is the
    block-Jacobi ILU0 (Section 4.5): the schedule and the factors come from
    the partition-internal blocks, the SpMV uses all of A.  Returns (x in
    natural order, SolveResult, perm, nsets).  With wells (Section 4.6) the
    system operator is A - sum C^T inv(D) B, preconditioned by ILU0 of A."""
    if part is None:
        mrp, mci, mvals = rowptr, colidx, vals
    else:
        mrp, mci, mvals, _ = jacobi_pattern(nb, rowptr, colidx, vals, part)
    perm, nsets = schedule_perm(nb, mrp, mci, schedule)
    prow, pcol, pval = permute(nb, rowptr, colidx, vals, perm)
    mprow, mpcol, mpval = permute(nb, mrp, mci, mvals, perm)
    pb = np.asarray(b).reshape(nb, 3)[perm].ravel()
    fac = ilu0(nb, mprow, mpcol, mpval, f32=f32, cp_sweeps=cp_sweeps)
    if fac.status != 0:
        raise ArithmeticError(f"oracle ILU0 failed with status {fac.status}")
    pw = None
    if wells is not None:
        iperm = np.empty(nb, dtype=np.int64)
        iperm[perm] = np.arange(nb)
        pw = type(wells)(**{**wells.__dict__, "cells": iperm[np.asarray(wells.cells)].astype(np.int32)})
    res = bicgstab(nb, prow, pcol, pval, fac, pb, rtol, maxit, mpattern=(mprow, mpcol), wells=pw,
                   tri_sweeps=tri_sweeps)
    x = np.empty(3 * nb)
    x.reshape(nb, 3)[perm] = res.x.reshape(nb, 3)
    return x, res, perm, nsets
