"""Iterative FP64 solve of the oracle's linearised system, for meshes where
the sparse direct LU of ``Oracle.solve_linear`` runs out of memory.

TEST INFRASTRUCTURE ONLY (see oracle/fem.py).  The arithmetic is the plain C
of ``oracle/krylov.c``: scalar ILU(0) in the pattern of the matrix and
restarted GMRES(m) with modified Gram-Schmidt, right preconditioned.  Around
it this module applies the same exact change of rows and unknowns as the
direct solve (row then column max-abs equilibration, because the Newton
matrix mixes force rows ~E h, identity rows and scaled flux rows), and
iterative refinement on the true residual of the equilibrated system.  No
blocking, coarse level or other structure of the CUDA library's solver is
used: this is an independent route to the solution of the linear system of
Sec. 3 (the Newton system after Eq. fully-coupled-fully-discrete).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np
import scipy.sparse as sp

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "krylov.c")
LIB = os.path.join(HERE, "_build", "libhforacle.so")

_lib = None


def build(force=False):
    """Compiles krylov.c with the host C compiler (plain C, no target-specific
    flags, so the same source builds on x86-64 and Arm)."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        i64, dp, i64p, i32p = C.c_int64, C.POINTER(C.c_double), C.POINTER(C.c_int64), C.POINTER(C.c_int32)
        lib.oracle_ilu0.argtypes = [i64, i64p, i32p, dp, dp, i64p]
        lib.oracle_ilu0.restype = i64
        lib.oracle_ilu0_solve.argtypes = [i64, i64p, i32p, dp, i64p, dp, dp]
        lib.oracle_csr_matvec.argtypes = [i64, i64p, i32p, dp, dp, dp]
        lib.oracle_gmres.argtypes = [i64, i64p, i32p, dp, dp, i64p, dp, dp, i64, i64, C.c_double, dp]
        lib.oracle_gmres.restype = i64
        _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(C.POINTER(t))


class CSR:
    """A CSR matrix in the layout krylov.c reads: int64 row pointers, int32
    sorted column indices, FP64 values."""

    def __init__(self, A):
        A = sp.csr_matrix(A)
        A.sum_duplicates()
        A.sort_indices()
        self.n = A.shape[0]
        self.ptr = np.ascontiguousarray(A.indptr, dtype=np.int64)
        self.col = np.ascontiguousarray(A.indices, dtype=np.int32)
        self.val = np.ascontiguousarray(A.data, dtype=np.float64)

    def matvec(self, x):
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n)
        _load().oracle_csr_matvec(self.n, _p(self.ptr, C.c_int64), _p(self.col, C.c_int32), _p(self.val, C.c_double),
                                  _p(x, C.c_double), _p(y, C.c_double))
        return y


class ILU0:
    """Scalar ILU(0) factors of a CSR matrix (the pattern of A, no fill)."""

    def __init__(self, A: CSR):
        self.A = A
        self.lu = np.empty_like(A.val)
        self.diag = np.empty(A.n, dtype=np.int64)
        st = _load().oracle_ilu0(A.n, _p(A.ptr, C.c_int64), _p(A.col, C.c_int32), _p(A.val, C.c_double),
                                 _p(self.lu, C.c_double), _p(self.diag, C.c_int64))
        if st != 0:
            raise ArithmeticError(f"ILU(0): row {-st - 1} has no diagonal entry or a zero pivot")

    def solve(self, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        z = np.empty(self.A.n)
        A = self.A
        _load().oracle_ilu0_solve(A.n, _p(A.ptr, C.c_int64), _p(A.col, C.c_int32), _p(self.lu, C.c_double),
                                  _p(self.diag, C.c_int64), _p(r, C.c_double), _p(z, C.c_double))
        return z


def gmres(A: CSR, M: ILU0, b, x0=None, restart=100, maxit=20000, tol_abs=0.0):
    """Restarted right-preconditioned GMRES(restart) from x0 (zeros by
    default).  Returns (x, Arnoldi steps, last residual norm)."""
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(A.n) if x0 is None else np.array(x0, dtype=np.float64)
    out = np.zeros(2)
    st = _load().oracle_gmres(A.n, _p(A.ptr, C.c_int64), _p(A.col, C.c_int32), _p(A.val, C.c_double),
                              _p(M.lu, C.c_double), _p(M.diag, C.c_int64), _p(b, C.c_double), _p(x, C.c_double),
                              int(restart), int(maxit), float(tol_abs), _p(out, C.c_double))
    if st != 0:
        raise MemoryError("GMRES workspace")
    return x, int(out[0]), float(out[1])


def solve_linear_iterative(J, b, rtol=1e-13, restart=100, maxit=20000, refinements=6, info=None):
    """Solution of J d = b by ILU(0)-preconditioned GMRES on the row- then
    column-equilibrated matrix A = D_r J D_c (max-abs scaling, as in the
    direct solve), with iterative refinement: each pass solves A e = s - A y
    for the true residual of the current iterate and adds e, until that
    residual is at most rtol ||s|| (s = D_r b), it stops shrinking, or
    `refinements` passes are done.  Returns d = D_c y."""
    J = sp.csr_matrix(J)
    r = 1.0 / abs(J).max(axis=1).toarray().ravel()
    J1 = sp.diags(r) @ J
    c = 1.0 / abs(J1).max(axis=0).toarray().ravel()
    A = CSR(J1 @ sp.diags(c))
    A_nz = sp.csr_matrix((A.val, A.col, A.ptr), shape=(A.n, A.n))
    A_nz.eliminate_zeros()
    Ap = CSR(A_nz)
    M = ILU0(Ap)
    s = r * np.asarray(b, dtype=np.float64)
    snorm = np.linalg.norm(s)
    y = np.zeros(A.n)
    hist, its = [], 0
    if snorm == 0.0:
        return np.zeros(A.n)
    res = snorm
    for _ in range(refinements):
        e, k, _ = gmres(Ap, M, s - Ap.matvec(y), restart=restart, maxit=maxit, tol_abs=0.1 * rtol * snorm)
        its += k
        y = y + e
        new = np.linalg.norm(s - Ap.matvec(y))
        hist.append(new / snorm)
        if new <= rtol * snorm or new >= 0.5 * res:
            res = new
            break
        res = new
    if info is not None:
        info.update(iters=its, rel_res=res / snorm, history=hist, nnz=int(Ap.ptr[-1]))
    return c * y
