"""FP64 CPU oracle for the generalized eigenproblem A y = lambda B y.

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check and by
the CPU-baseline leg of the benchmark, never by the solver package.  It shares
no code with the GPU path.  The arithmetic lives in ``gep_oracle.c`` (plain
C, FP64, no BLAS/LAPACK); this module compiles it with gcc and exposes each
routine on numpy arrays.

Every routine follows section 3.1 of Imachi & Hoshi (Eq. 2-6) or a textbook
algorithm named in its C header comment.  Parity pins live in
``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gep_oracle.c")
_LIB = os.path.join(_HERE, "_gep_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int


def build(force: bool = False) -> str:
    """Compile gep_oracle.c into _gep_oracle.so (gcc, OpenMP, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", "-std=c11",
           "-Wall", "-Wno-unused-function", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.oc_cholesky.argtypes = [_I, _D, _I]
            lib.oc_cholesky.restype = _I
            lib.oc_two_sided.argtypes = [_I, _D, _I, _D, _I]
            lib.oc_tridiag.argtypes = [_I, _D, _I, _D, _D, _D, _I]
            lib.oc_tql.argtypes = [_I, _D, _D, _D, _I]
            lib.oc_tql.restype = _I
            lib.oc_sturm_count.argtypes = [_I, _D, _D, ctypes.c_double]
            lib.oc_sturm_count.restype = _I
            lib.oc_bisect.argtypes = [_I, _D, _D, _D]
            lib.oc_backsub.argtypes = [_I, _I, _D, _I, _D, _I]
            lib.oc_gep_solve.argtypes = [_I, _D, _I, _D, _I, _D, _D, _I, _I]
            lib.oc_gep_solve.restype = _I
            lib.oc_gep_solve_eigenexa.argtypes = [_I, _D, _I, _D, _I, _D, _D, _I, _I]
            lib.oc_gep_solve_eigenexa.restype = _I
            lib.oc_gep_solve_partial.argtypes = [_I, _D, _I, _D, _I, _I, _D, _D, _I]
            lib.oc_gep_solve_partial.restype = _I
            lib.oc_jacobi.argtypes = [_I, _D, _I, _D, _D, _I]
            lib.oc_jacobi.restype = _I
            lib.oc_inertia.argtypes = [_I, _D, _I, _D, _I, ctypes.c_double,
                                       ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_I)]
            lib.oc_adjoint.argtypes = [_I, _I, _D, _D, _I, _D, _D, _I, _D, _D, _I]
            _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(_D)


def _colmajor(a):
    """Copy of a 2-D array as a Fortran-ordered float64 array (column-major)."""
    return np.array(a, dtype=np.float64, order="F", copy=True)


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (must be called before the first call)."""
    os.environ["OMP_NUM_THREADS"] = str(int(n))


# ----------------------------------------------------------------- stages

def cholesky(B):
    """Eq. 4: returns (L, info); L lower with B = L L^T (upper part zero)."""
    L = _colmajor(B)
    M = L.shape[0]
    info = _load().oc_cholesky(M, _p(L), max(M, 1))
    return L, int(info)


def two_sided(A, L):
    """Eq. 5: C = L^-1 A L^-T (full symmetric)."""
    C = _colmajor(A)
    Lf = _colmajor(L)
    M = C.shape[0]
    _load().oc_two_sided(M, _p(C), max(M, 1), _p(Lf), max(M, 1))
    return C


def tridiag(C, want_q=True):
    """Householder tridiagonalisation C = Q T Q^T; returns (d, e, Q or None)."""
    S = _colmajor(C)
    M = S.shape[0]
    d = np.zeros(M)
    e = np.zeros(max(M - 1, 1))
    Q = np.zeros((M, M), order="F") if want_q else None
    _load().oc_tridiag(M, _p(S), max(M, 1), _p(d), _p(e), _p(Q), max(M, 1))
    return d, e[: max(M - 1, 0)], Q


def tql(d, e, Z=None):
    """Implicit QL on (d, e); returns (eigenvalues unsorted, Z G, status)."""
    d = np.array(d, dtype=np.float64, copy=True)
    M = d.shape[0]
    ee = np.zeros(max(M, 1))
    ee[: M - 1] = e[: M - 1]
    Zf = None if Z is None else _colmajor(Z)
    st = _load().oc_tql(M, _p(d), _p(ee), _p(Zf), max(M, 1))
    return d, Zf, int(st)


def sturm_count(d, e, sigma):
    d = np.ascontiguousarray(d, dtype=np.float64)
    M = d.shape[0]
    ee = np.zeros(max(M, 1))
    ee[: M - 1] = e[: M - 1]
    return int(_load().oc_sturm_count(M, _p(d), _p(ee), float(sigma)))


def bisect(d, e):
    """All eigenvalues of the tridiagonal (d, e), ascending, by Sturm bisection."""
    d = np.ascontiguousarray(d, dtype=np.float64)
    M = d.shape[0]
    ee = np.zeros(max(M, 1))
    ee[: M - 1] = e[: M - 1]
    w = np.zeros(M)
    _load().oc_bisect(M, _p(d), _p(ee), _p(w))
    return w


def backsub(L, Z):
    """Eq. 6: Y = L^-T Z."""
    Lf = _colmajor(L)
    Y = _colmajor(Z)
    M, n = Y.shape
    _load().oc_backsub(M, n, _p(Lf), max(M, 1), _p(Y), max(M, 1))
    return Y


def gep_solve(A, B, want_vectors=True):
    """Eq. 2: (w ascending, Y B-orthonormal or None, info)."""
    Af = _colmajor(A)
    Bf = _colmajor(B)
    M = Af.shape[0]
    w = np.zeros(M)
    Y = np.zeros((M, M), order="F") if want_vectors else None
    info = _load().oc_gep_solve(M, _p(Af), max(M, 1), _p(Bf), max(M, 1), _p(w), _p(Y), max(M, 1),
                                1 if want_vectors else 0)
    return w, Y, int(info)


def gep_solve_eigenexa(A, B, want_vectors=True):
    """Eq. 7-9 (Cholesky-free reducer): (w ascending, Y B-orthonormal or None, info)."""
    Af = _colmajor(A)
    Bf = _colmajor(B)
    M = Af.shape[0]
    w = np.zeros(M)
    Y = np.zeros((M, M), order="F") if want_vectors else None
    info = _load().oc_gep_solve_eigenexa(M, _p(Af), max(M, 1), _p(Bf), max(M, 1), _p(w), _p(Y), max(M, 1),
                                         1 if want_vectors else 0)
    return w, Y, int(info)


def gep_solve_partial(A, B, n_want):
    """The n_want lowest eigenpairs (bisection + inverse iteration): (w, Y M x n_want, info)."""
    Af = _colmajor(A)
    Bf = _colmajor(B)
    M = Af.shape[0]
    n = max(0, min(int(n_want), M))
    w = np.zeros(max(n, 1))
    Y = np.zeros((M, max(n, 1)), order="F")
    info = _load().oc_gep_solve_partial(M, _p(Af), max(M, 1), _p(Bf), max(M, 1), n, _p(w), _p(Y), max(M, 1))
    return w[:n], Y[:, :n], int(info)


def jacobi(S, want_v=True):
    """Cyclic Jacobi: (eigenvalues ascending, V with matching column order, sweeps)."""
    Sf = _colmajor(S)
    M = Sf.shape[0]
    w = np.zeros(M)
    V = np.zeros((M, M), order="F") if want_v else None
    sweeps = _load().oc_jacobi(M, _p(Sf), max(M, 1), _p(w), _p(V), max(M, 1))
    order = np.argsort(w, kind="stable")
    return w[order], (V[:, order] if V is not None else None), int(sweeps)


def inertia(A, B, sigma):
    """(n_neg, n_zero, n_pos) of A - sigma B (Bunch-Parlett LDL^T)."""
    Af = _colmajor(A)
    Bf = _colmajor(B)
    M = Af.shape[0]
    n, z, p = _I(), _I(), _I()
    _load().oc_inertia(M, _p(Af), max(M, 1), _p(Bf), max(M, 1), float(sigma),
                       ctypes.byref(n), ctypes.byref(z), ctypes.byref(p))
    return n.value, z.value, p.value


def adjoint(w, Y, n_occ, lbar, W=None):
    """Reverse-mode (Abar, Bbar) of sum_k lbar_k lambda_k + <W, Y_o Y_o^T>."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    Yf = _colmajor(Y)
    M = Yf.shape[0]
    lb = np.ascontiguousarray(lbar, dtype=np.float64)
    Wf = None if W is None else _colmajor(W)
    Ab = np.zeros((M, M), order="F")
    Bb = np.zeros((M, M), order="F")
    _load().oc_adjoint(M, int(n_occ), _p(w), _p(Yf), max(M, 1), _p(lb), _p(Wf), max(M, 1),
                       _p(Ab), _p(Bb), max(M, 1))
    return Ab, Bb
