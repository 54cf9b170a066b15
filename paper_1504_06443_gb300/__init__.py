"""Python binding of libgep (include/gep.h): a one-GPU dense solver for the
generalized eigenproblem A y = lambda B y (Imachi & Hoshi, Eq. 1-6).

Argument marshalling only: every step of the solve runs in the library's CUDA
kernels.  PyTorch provides device memory (the workspace is a torch tensor) and
the stream.  If the compiled library is missing the import of a solver function
raises; there is no CPU fallback.

Matrices cross the boundary column-major.  Helpers accept any strided float64
CUDA tensor: symmetric inputs may be passed row-major (their transpose is
themselves); outputs come back as column-major views with the logical indices
of the mathematics (Y[i, k] is component i of eigenvector k).
"""
from __future__ import annotations

import ctypes
import os
import threading

__all__ = ["load", "solve", "solve_host", "cholesky", "reduce", "tridiag_1stage", "tridiag_eig",
           "sep_backtransform", "tridiag_2stage", "sep_backtransform_2stage", "gep_backtransform", "dgemm", "Handle", "default_handle",
           "RED_TWOSIDED", "RED_EXPLICIT_INV", "RED_EIGENEXA", "SEP_1STAGE", "SEP_JACOBI", "SEP_2STAGE", "PREC_FP64",
           "PREC_FP64_EMULATED", "PREC_MIXED_REFINED", "GepError", "shard_batch"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgep.so")

RED_TWOSIDED, RED_EXPLICIT_INV, RED_EIGENEXA = 0, 1, 2
SEP_1STAGE, SEP_2STAGE, SEP_JACOBI = 0, 1, 2
PREC_FP64, PREC_FP64_EMULATED, PREC_MIXED_REFINED = 0, 1, 2
# return codes of include/gep.h
ERR_CUDA, ERR_ALLOC, ERR_NONFINITE, ERR_TIMEOUT, ERR_HANDLE, ERR_UNSUPPORTED, ERR_TOO_LARGE = (
    -100, -101, -102, -103, -104, -105, -106)

_REDUCERS = {"twosided": RED_TWOSIDED, "explicit_inv": RED_EXPLICIT_INV, "eigenexa": RED_EIGENEXA}
_SEPS = {"1stage": SEP_1STAGE, "2stage": SEP_2STAGE, "jacobi": SEP_JACOBI}
_PRECS = {"fp64": PREC_FP64, "fp64_emulated": PREC_FP64_EMULATED, "mixed_refined": PREC_MIXED_REFINED}


class GepError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        msg = _lib_or_none().gep_status_string(code).decode() if _lib_or_none() else str(code)
        super().__init__(f"{where} returned {code}: {msg}")


class GepOptions(ctypes.Structure):
    _fields_ = [("reducer", ctypes.c_int), ("sep", ctypes.c_int), ("bandwidth", ctypes.c_int),
                ("precision", ctypes.c_int), ("want_vectors", ctypes.c_int), ("overwrite", ctypes.c_int),
                ("timers", ctypes.c_int), ("refine_iters", ctypes.c_int), ("n_want", ctypes.c_int),
                ("batch_small", ctypes.c_int)]


_lib = None
_lock = threading.Lock()
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t


def _lib_or_none():
    return _lib


def load():
    """Loads the compiled library; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libgep.so not built ({LIB_PATH}); run paper_1504_06443_gb300.build.build() "
                               "or __graft_entry__.build() first")
        lib = ctypes.CDLL(LIB_PATH)
        sig = {
            "gep_default_options": (None, [ctypes.POINTER(GepOptions)]),
            "gep_create": (_I, [ctypes.POINTER(_P), _P]),
            "gep_destroy": (_I, [_P]),
            "gep_set_stream": (_I, [_P, _P]),
            "gep_workspace_size": (_I, [_P, _I, ctypes.POINTER(GepOptions), ctypes.POINTER(_SZ)]),
            "gep_workspace_size_host": (_I, [_P, _I, ctypes.POINTER(GepOptions), ctypes.POINTER(_SZ)]),
            "gep_set_workspace": (_I, [_P, _P, _SZ]),
            "gep_cholesky": (_I, [_P, _I, _P, _I]),
            "gep_reduce": (_I, [_P, _I, _P, _I, _P, _I, _I]),
            "gep_backtransform": (_I, [_P, _I, _I, _P, _I, _P, _I, _I]),
            "sep_tridiag_1stage": (_I, [_P, _I, _P, _I, _P, _P, _P]),
            "sep_tridiag_eig": (_I, [_P, _I, _P, _P, _P, _P, _I, _I]),
            "sep_backtransform": (_I, [_P, _I, _I, _P, _I, _P, _P, _I]),
            "sep_q2_elems": (_SZ, [_I, _I]),
            "sep_tridiag_2stage": (_I, [_P, _I, _P, _I, _I, _P, _P, _P, _P]),
            "sep_backtransform_2stage": (_I, [_P, _I, _I, _I, _P, _I, _P, _P, _P, _I]),
            "gep_solve": (_I, [_P, _I, _P, _I, _P, _I, _P, _P, _I, ctypes.POINTER(GepOptions)]),
            "gep_solve_host": (_I, [_P, _I, _P, _I, _P, _I, _P, _P, _I, ctypes.POINTER(GepOptions)]),
            "gep_get_info": (_I, [_P, ctypes.POINTER(_I)]),
            "gep_reset_info": (_I, [_P]),
            "gep_set_wait_fault": (_I, [_P, _I, _D]),
            "gep_set_panel_qr": (_I, [_P, _I]),
            "gep_get_stage_times": (_I, [_P, ctypes.POINTER(_D)]),
            "gep_launch_count": (ctypes.c_longlong, [_P, _I]),
            "gep_refine_steps": (_I, [_P]),
            "gep_stage_workspace_size": (_I, [_P, _I, _I, ctypes.POINTER(_SZ)]),
            "gep_profile_entry": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)]),
            "gep_get_band_times": (_I, [_P, ctypes.POINTER(_D)]),
            "gep_profile_enable": (_I, [_P, _I]),
            "gep_profile_read": (_I, [_P, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D),
                                      ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong), _I]),
            "gep_status_string": (ctypes.c_char_p, [_I]),
            "gep_adjoint_workspace_size": (_I, [_P, _I, _I, ctypes.POINTER(_SZ)]),
            "gep_adjoint": (_I, [_P, _I, _I, _P, _P, _I, _P, _P, _I, _P, _P, _I]),
            "gep_solve_batched_workspace_size": (_I, [_P, _I, _P, ctypes.POINTER(GepOptions), _P, _I,
                                                     ctypes.POINTER(_SZ)]),
            "gep_solve_batched": (_I, [_P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(GepOptions), _P, _I]),
            "gep_solve_batched_opts_workspace_size": (_I, [_P, _I, _P, ctypes.POINTER(GepOptions), _I,
                                                          ctypes.POINTER(_SZ)]),
            "gep_solve_batched_opts": (_I, [_P, _I, _P, _P, _P, _P, _P, ctypes.POINTER(GepOptions), _I]),
            "gep_batched_info": (_I, [_P, ctypes.POINTER(_I)]),
            "gep_set_band_group": (_I, [_P, _I]),
            "gep_dgemm": (_I, [_P, ctypes.c_char, ctypes.c_char, ctypes.c_char, _I, _I, _I, _D, _P, _I, _P, _I,
                               _D, _P, _I, _I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _check(rc, where):
    if rc != 0:
        raise GepError(rc, where)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _torch():
    import torch
    return torch


def colmajor(t):
    """A float64 CUDA tensor with the same logical values, stored column-major (strides (1, m))."""
    torch = _torch()
    t = t.to(dtype=torch.float64)
    if t.dim() == 2 and t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.t().contiguous().t()


def _ld(t):
    return max(1, t.stride(1)) if t.dim() == 2 else max(1, t.shape[0])


def _sym_ptr_ld(t):
    """Pointer + leading dimension for a symmetric matrix argument (any 2-D memory order)."""
    if t.stride(0) == 1:
        return _ptr(t), max(1, t.stride(1))
    if t.stride(1) == 1:
        return _ptr(t), max(1, t.stride(0))  # row-major buffer = transpose = itself
    raise ValueError("symmetric matrix argument must have a unit stride in one dimension")


def _need_cuda(t, name):
    if not t.is_cuda:
        raise ValueError(f"{name}: expected a CUDA tensor (the library has no CPU path), got {t.device}")


def _need_matrix(t, name, rows=None, cols=None, square=False, f64=False, cuda=True):
    """Host-side check of a matrix argument before any pointer reaches the device: a 2-D CUDA
    tensor of the stated size (float64 where the library reads the caller's buffer in place)."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if t.dim() != 2:
        raise ValueError(f"{name}: expected a 2-D tensor, got shape {tuple(t.shape)}")
    if square and t.shape[0] != t.shape[1]:
        raise ValueError(f"{name}: expected a square matrix, got shape {tuple(t.shape)}")
    if rows is not None and t.shape[0] != rows:
        raise ValueError(f"{name}: expected {rows} rows, got shape {tuple(t.shape)}")
    if cols is not None and t.shape[1] != cols:
        raise ValueError(f"{name}: expected {cols} columns, got shape {tuple(t.shape)}")
    if f64 and t.dtype != torch.float64:
        raise TypeError(f"{name}: expected float64, got {t.dtype}")
    if cuda:
        _need_cuda(t, name)


def _need_vector(t, name, min_len, f64=False, cuda=True):
    """Host-side check of a vector argument: a CUDA tensor with at least min_len elements."""
    torch = _torch()
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor, got {type(t).__name__}")
    if t.numel() < min_len:
        raise ValueError(f"{name}: expected at least {min_len} elements, got {t.numel()}")
    if f64 and t.dtype != torch.float64:
        raise TypeError(f"{name}: expected float64, got {t.dtype}")
    if cuda:
        _need_cuda(t, name)


def _need_on_device(*named):
    """Device check of already shape-checked arguments (pairs name, tensor; None skipped)."""
    for name, t in zip(named[0::2], named[1::2]):
        if t is not None:
            _need_cuda(t, name)


def _same_device(h, *ts):
    for t in ts:
        if t is not None and t.device != h.device:
            raise ValueError(f"tensor on {t.device} but the handle is bound to {h.device}")


class Handle:
    """A libgep handle bound to one CUDA stream, with a torch-allocated workspace."""

    def __init__(self, stream=None, device=None):
        torch = _torch()
        self.lib = load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(self.lib.gep_create(ctypes.byref(h), ctypes.c_void_p(self.stream.cuda_stream)), "gep_create")
        self.h = h
        self.ws = None

    def close(self):
        if self.h:
            self.lib.gep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ensure_workspace(self, nbytes):
        torch = _torch()
        if self.ws is None or self.ws.numel() < nbytes:
            self.ws = None
            self.ws = torch.empty(max(int(nbytes), 256) + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        aligned = (base + 255) & ~255
        _check(self.lib.gep_set_workspace(self.h, ctypes.c_void_p(aligned), self.ws.numel() - (aligned - base)),
               "gep_set_workspace")

    def info(self):
        v = _I()
        _check(self.lib.gep_get_info(self.h, ctypes.byref(v)), "gep_get_info")
        return v.value

    def reset_info(self):
        _check(self.lib.gep_reset_info(self.h), "gep_reset_info")

    def set_wait_fault(self, drop_sweep=-1, wait_limit_s=4.0):
        """Failure-detection hook: bounded device waits give up after wait_limit_s seconds
        (at most 4) with GEP_ERR_TIMEOUT; drop_sweep >= 0 stops that bulge-chasing sweep from
        publishing progress, so the wait behind it runs out (-1: no injection)."""
        _check(self.lib.gep_set_wait_fault(self.h, int(drop_sweep), float(wait_limit_s)), "gep_set_wait_fault")

    def set_panel_qr(self, rows=0):
        """Test hook: force the panel-QR CTA height of the full -> band reduction (64, 128 or
        256 rows per CTA), the per-column-step kernel (-1), or the automatic choice (0)."""
        _check(self.lib.gep_set_panel_qr(self.h, int(rows)), "gep_set_panel_qr")

    def set_band_group(self, min_order=-1):
        """Test hook: the trailing order from which the full -> band reduction groups panels in
        fours (0: always, -1: the library default)."""
        _check(self.lib.gep_set_band_group(self.h, int(min_order)), "gep_set_band_group")

    def stage_times(self):
        t = (_D * 7)()
        _check(self.lib.gep_get_stage_times(self.h, t), "gep_get_stage_times")
        return list(t)

    def launches(self, reset=False):
        return int(self.lib.gep_launch_count(self.h, 1 if reset else 0))

    def profile_entries(self, count):
        """[(m, n, k, ms)] of the first `count` recorded product launches."""
        out = []
        mnk = (_I * 3)()
        ms = _D()
        for i in range(int(count)):
            _check(self.lib.gep_profile_entry(self.h, i, mnk, ctypes.byref(ms)), "gep_profile_entry")
            out.append((mnk[0], mnk[1], mnk[2], ms.value))
        return out

    def band_times(self):
        """(full->band ms, bulge-chasing ms) of the last two-stage solve with timers."""
        t = (_D * 2)()
        _check(self.lib.gep_get_band_times(self.h, t), "gep_get_band_times")
        return [t[0], t[1]]

    def refine_steps(self):
        """FP64 refinement steps the last mixed-precision solve on this handle took."""
        return int(self.lib.gep_refine_steps(self.h))

    def profile_enable(self, cap):
        _check(self.lib.gep_profile_enable(self.h, int(cap)), "gep_profile_enable")

    def profile_read(self, reset=True):
        ms, f, f64 = _D(), _D(), _D()
        n, sk = ctypes.c_longlong(), ctypes.c_longlong()
        _check(self.lib.gep_profile_read(self.h, ctypes.byref(ms), ctypes.byref(f), ctypes.byref(f64), ctypes.byref(n),
                                         ctypes.byref(sk), 1 if reset else 0), "gep_profile_read")
        return dict(ms=ms.value, tensor_flops=f.value, fp64_flops=f64.value, launches=n.value, skipped=sk.value)


_handles = {}


def default_handle():
    torch = _torch()
    key = (torch.cuda.current_device(), torch.cuda.current_stream().cuda_stream)
    h = _handles.get(key)
    if h is None:
        h = Handle()
        _handles[key] = h
    return h


def make_options(reducer="twosided", sep="1stage", precision="fp64", want_vectors=True, overwrite=False,
                 timers=False, bandwidth=0, refine_iters=0, n_want=0, batch_small=0):
    o = GepOptions()
    load().gep_default_options(ctypes.byref(o))
    o.reducer = _REDUCERS[reducer] if isinstance(reducer, str) else int(reducer)
    o.sep = _SEPS[sep] if isinstance(sep, str) else int(sep)
    o.precision = _PRECS[precision] if isinstance(precision, str) else int(precision)
    o.want_vectors = 1 if want_vectors else 0
    o.overwrite = 1 if overwrite else 0
    o.timers = 1 if timers else 0
    o.bandwidth = int(bandwidth)
    o.refine_iters = int(refine_iters)
    o.n_want = int(n_want)
    o.batch_small = int(batch_small)
    return o


def workspace_bytes(M, handle=None, **opts):
    h = handle or default_handle()
    o = make_options(**opts)
    n = _SZ()
    _check(h.lib.gep_workspace_size(h.h, int(M), ctypes.byref(o), ctypes.byref(n)), "gep_workspace_size")
    return n.value


def solve(A, B, reducer="twosided", sep="1stage", precision="fp64", want_vectors=True, overwrite=False,
          timers=False, bandwidth=0, handle=None, out=None, refine_iters=0, n_want=0):
    """All eigenpairs of A y = lambda B y (A, B symmetric float64 CUDA tensors, B SPD), or
    only the n_want lowest (0 = all).

    Returns (w, Y, info): w ascending (n entries), Y (M x n column-major view) B-orthonormal
    or None.  info != 0 reports a numerical failure (k: B's leading minor k not positive
    definite)."""
    torch = _torch()
    _need_matrix(A, "A", square=True, f64=True, cuda=False)
    M = int(A.shape[0])
    _need_matrix(B, "B", rows=M, cols=M, f64=True, cuda=False)
    if not 0 <= int(n_want) <= M:
        raise ValueError(f"n_want must lie in [0, {M}]")
    n = int(n_want) if n_want else M
    if out is not None:
        _need_vector(out[0], "out[0] (w)", n, f64=True)
        if want_vectors:
            _need_matrix(out[1], "out[1] (Y^T)", rows=n, cols=M, f64=True)
            if not out[1].is_contiguous():
                raise ValueError("out[1] (Y^T) must be contiguous")
    _need_on_device("A", A, "B", B)
    h = handle or default_handle()
    _same_device(h, A, B)
    o = make_options(reducer, sep, precision, want_vectors, overwrite, timers, bandwidth, refine_iters, n_want)
    nb = _SZ()
    _check(h.lib.gep_workspace_size(h.h, M, ctypes.byref(o), ctypes.byref(nb)), "gep_workspace_size")
    h.ensure_workspace(nb.value)
    pa, lda = _sym_ptr_ld(A)
    pb, ldb = _sym_ptr_ld(B)
    if out is not None:
        w, Yt = out
    else:
        w = torch.empty(n, dtype=torch.float64, device=A.device)
        Yt = torch.empty((n, M), dtype=torch.float64, device=A.device) if want_vectors else None
    _check(h.lib.gep_solve(h.h, M, pa, lda, pb, ldb, _ptr(w), _ptr(Yt), max(1, M), ctypes.byref(o)), "gep_solve")
    info = h.info()
    return w, (Yt.t() if Yt is not None else None), info


def solve_async(A, B, w, Yt, opts, handle):
    """Enqueue-only variant used by the benchmark: no synchronisation, no allocation."""
    _need_matrix(A, "A", square=True, f64=True, cuda=False)
    _need_matrix(B, "B", rows=A.shape[0], cols=A.shape[0], f64=True, cuda=False)
    n = int(opts.n_want) if opts.n_want else int(A.shape[0])  # w: n entries, Yt: n x M (Y^T)
    _need_vector(w, "w", n, f64=True, cuda=False)
    if Yt is not None:
        _need_matrix(Yt, "Yt", rows=n, cols=A.shape[0], f64=True, cuda=False)
        if not Yt.is_contiguous():
            raise ValueError("Yt must be contiguous")
    _need_on_device("A", A, "B", B, "w", w, "Yt", Yt)
    pa, lda = _sym_ptr_ld(A)
    pb, ldb = _sym_ptr_ld(B)
    _check(handle.lib.gep_solve(handle.h, int(A.shape[0]), pa, lda, pb, ldb, _ptr(w), _ptr(Yt), max(1, A.shape[0]),
                                ctypes.byref(opts)), "gep_solve")


def solve_host(A_np, B_np, want_vectors=True, handle=None, **opts):
    """Host numpy arrays in and out (copies inside the library).  Returns (w, Y, info)."""
    import numpy as np
    h = handle or default_handle()
    M = int(A_np.shape[0])
    o = make_options(want_vectors=want_vectors, **opts)
    nk = o.n_want if o.n_want else M
    nb = _SZ()
    _check(h.lib.gep_workspace_size_host(h.h, M, ctypes.byref(o), ctypes.byref(nb)), "gep_workspace_size_host")
    h.ensure_workspace(nb.value)
    A = np.ascontiguousarray(A_np, dtype=np.float64)
    B = np.ascontiguousarray(B_np, dtype=np.float64)
    w = np.empty(nk)
    Y = np.empty((M, nk), order="F") if want_vectors else None
    _check(h.lib.gep_solve_host(h.h, M, A.ctypes.data_as(_P), max(1, M), B.ctypes.data_as(_P), max(1, M),
                                w.ctypes.data_as(_P), Y.ctypes.data_as(_P) if Y is not None else None,
                                max(1, M), ctypes.byref(o)), "gep_solve_host")
    return w, Y, h.info()


# ------------------------------------------------------------------ stages

def cholesky(B, handle=None):
    """Eq. 4: returns (L column-major, info)."""
    _need_matrix(B, "B", square=True)
    h = handle or default_handle()
    L = colmajor(B.clone())
    M = L.shape[0]
    h.ensure_workspace(_stage_ws(M, handle=h))
    h.reset_info()
    _check(h.lib.gep_cholesky(h.h, M, _ptr(L), _ld(L)), "gep_cholesky")
    return L, h.info()


def _stage_ws(M, ncol=None, handle=None):
    """Workspace bytes the stage entry points need (asked from the library)."""
    h = handle or default_handle()
    n = _SZ()
    _check(h.lib.gep_stage_workspace_size(h.h, int(M), int(M if ncol is None else ncol), ctypes.byref(n)),
           "gep_stage_workspace_size")
    return n.value


def reduce(A, L, variant="twosided", handle=None):
    """Eq. 5: (C, L_or_R).  For 'explicit_inv' the returned second matrix is R = L^-1.
    For 'eigenexa' (Eq. 7-8, no Cholesky factor) pass B itself as L: the result is
    (A' = X^T A X, X = W D^-1/2) with B W = W D."""
    _need_matrix(A, "A", square=True, cuda=False)
    _need_matrix(L, "L", rows=A.shape[0], cols=A.shape[0], cuda=False)
    _need_on_device("A", A, "L", L)
    h = handle or default_handle()
    C = colmajor(A.clone())
    Lc = colmajor(L.clone())
    M = C.shape[0]
    h.ensure_workspace(_stage_ws(M, handle=h))
    _check(h.lib.gep_reduce(h.h, M, _ptr(C), _ld(C), _ptr(Lc), _ld(Lc), _REDUCERS[variant]), "gep_reduce")
    return C, Lc


def gep_backtransform(LR, Z, variant="twosided", handle=None):
    """Eq. 6: Y = L^-T Z (twosided) or Y = R^T Z (explicit_inv); Eq. 9: Y = X Z (eigenexa)."""
    _need_matrix(LR, "LR", square=True, cuda=False)
    _need_matrix(Z, "Z", rows=LR.shape[0], cuda=False)
    _need_on_device("LR", LR, "Z", Z)
    h = handle or default_handle()
    Y = colmajor(Z.clone())
    Lc = colmajor(LR)
    M, ncol = Y.shape
    h.ensure_workspace(_stage_ws(M, ncol, handle=h))
    _check(h.lib.gep_backtransform(h.h, M, ncol, _ptr(Lc), _ld(Lc), _ptr(Y), _ld(Y), _REDUCERS[variant]),
           "gep_backtransform")
    return Y


def tridiag_1stage(C, handle=None):
    """Householder tridiagonalisation: (d, e, tau, C_with_reflectors)."""
    torch = _torch()
    _need_matrix(C, "C", square=True)
    h = handle or default_handle()
    Cc = colmajor(C.clone())
    M = Cc.shape[0]
    d = torch.empty(M, dtype=torch.float64, device=C.device)
    e = torch.zeros(max(M, 1), dtype=torch.float64, device=C.device)
    tau = torch.zeros(max(M, 1), dtype=torch.float64, device=C.device)
    h.ensure_workspace(_stage_ws(M, handle=h))
    _check(h.lib.sep_tridiag_1stage(h.h, M, _ptr(Cc), _ld(Cc), _ptr(d), _ptr(e), _ptr(tau)), "sep_tridiag_1stage")
    return d, e[: max(M - 1, 0)], tau[: max(M - 1, 0)], Cc


def tridiag_eig(d, e, want_vectors=True, handle=None):
    """Divide and conquer (or bisection when want_vectors=False): (w ascending, Z or None, info)."""
    torch = _torch()
    _need_vector(d, "d", 0, cuda=False)
    M = int(d.shape[0])
    _need_vector(e, "e", max(M - 1, 0), cuda=False)
    _need_on_device("d", d, "e", e)
    h = handle or default_handle()
    dd = d.to(torch.float64).contiguous()
    ee = torch.zeros(max(M, 1), dtype=torch.float64, device=d.device)
    if M > 1:
        ee[: M - 1] = e[: M - 1]
    w = torch.empty(M, dtype=torch.float64, device=d.device)
    Zt = torch.empty((M, M), dtype=torch.float64, device=d.device) if want_vectors else None
    h.ensure_workspace(_stage_ws(M, handle=h))
    h.reset_info()
    _check(h.lib.sep_tridiag_eig(h.h, M, _ptr(dd), _ptr(ee), _ptr(w), _ptr(Zt), max(1, M), 1 if want_vectors else 0),
           "sep_tridiag_eig")
    return w, (Zt.t() if Zt is not None else None), h.info()


def sep_backtransform(C_refl, tau, Z, handle=None):
    """Z <- Q Z with the reflectors of tridiag_1stage."""
    torch = _torch()
    _need_matrix(C_refl, "C_refl", square=True, cuda=False)
    _need_matrix(Z, "Z", rows=C_refl.shape[0], cuda=False)
    _need_vector(tau, "tau", max(C_refl.shape[0] - 1, 0), cuda=False)
    _need_on_device("C_refl", C_refl, "Z", Z, "tau", tau)
    h = handle or default_handle()
    Y = colmajor(Z.clone())
    Cc = colmajor(C_refl)
    M, ncol = Y.shape
    tt = torch.zeros(max(M, 1), dtype=torch.float64, device=Z.device)
    if M > 1:
        tt[: M - 1] = tau[: M - 1]
    h.ensure_workspace(_stage_ws(M, ncol, handle=h))
    _check(h.lib.sep_backtransform(h.h, M, ncol, _ptr(Cc), _ld(Cc), _ptr(tt), _ptr(Y), _ld(Y)), "sep_backtransform")
    return Y


def _two_stage_ws(h, M, b):
    o = make_options(sep="2stage", bandwidth=b)
    n = _SZ()
    _check(h.lib.gep_workspace_size(h.h, M, ctypes.byref(o), ctypes.byref(n)), "gep_workspace_size")
    return n.value


def tridiag_2stage(C, b=64, want_q2=True, handle=None):
    """Two-stage reduction (full -> band of width b -> tridiagonal):
    (d, e, tau1, q2 or None, C with the band and the panel reflectors)."""
    torch = _torch()
    _need_matrix(C, "C", square=True)
    h = handle or default_handle()
    Cc = colmajor(C.clone())
    M = Cc.shape[0]
    d = torch.empty(max(M, 1), dtype=torch.float64, device=C.device)
    e = torch.zeros(max(M, 1), dtype=torch.float64, device=C.device)
    tau1 = torch.zeros(max(M, 1), dtype=torch.float64, device=C.device)
    nq = int(h.lib.sep_q2_elems(M, int(b)))
    q2 = torch.empty(max(nq, 1), dtype=torch.float64, device=C.device) if want_q2 else None
    h.ensure_workspace(_two_stage_ws(h, M, b))
    _check(h.lib.sep_tridiag_2stage(h.h, M, _ptr(Cc), _ld(Cc), int(b), _ptr(d), _ptr(e), _ptr(tau1), _ptr(q2)),
           "sep_tridiag_2stage")
    return d[:M], e[: max(M - 1, 0)], tau1[:M], q2, Cc


def sep_backtransform_2stage(C_refl, tau1, q2, b, Z, handle=None):
    """Z <- Q1 (Q2 Z) with the output of tridiag_2stage."""
    _need_matrix(C_refl, "C_refl", square=True, cuda=False)
    M = int(C_refl.shape[0])
    _need_matrix(Z, "Z", rows=M, cuda=False)
    _need_vector(tau1, "tau1", M, f64=True, cuda=False)
    if M > 2:
        _need_vector(q2, "q2", int(load().sep_q2_elems(M, int(b))), f64=True, cuda=False)
    _need_on_device("C_refl", C_refl, "Z", Z, "tau1", tau1, "q2", q2)
    h = handle or default_handle()
    Y = colmajor(Z.clone())
    Cc = colmajor(C_refl)
    M, ncol = Y.shape
    h.ensure_workspace(max(_two_stage_ws(h, M, b), _stage_ws(M, ncol, handle=h)))
    _check(h.lib.sep_backtransform_2stage(h.h, M, ncol, int(b), _ptr(Cc), _ld(Cc), _ptr(tau1.contiguous()),
                                          _ptr(q2), _ptr(Y), _ld(Y)), "sep_backtransform_2stage")
    return Y


def dgemm(A, B, transa="N", transb="N", alpha=1.0, beta=0.0, C=None, uplo="F", engine="fp64", handle=None):
    """C = alpha op(A) op(B) + beta C on the library's GEMM engine (column-major views).
    transa 'S': A symmetric with only its lower triangle read (op(A) = A)."""
    torch = _torch()
    if transa not in ("N", "T", "S") or transb not in ("N", "T") or uplo not in ("F", "L"):
        raise ValueError("transa in N/T/S, transb in N/T, uplo in F/L")
    _need_matrix(A, "A", square=(transa == "S"), cuda=False)
    _need_matrix(B, "B", cuda=False)
    m = A.shape[1] if transa == "T" else A.shape[0]
    k = A.shape[0] if transa == "T" else A.shape[1]
    kb = B.shape[1] if transb == "T" else B.shape[0]
    n = B.shape[0] if transb == "T" else B.shape[1]
    if kb != k:
        raise ValueError(f"inner dimensions differ: op(A) is {m} x {k}, op(B) is {kb} x {n}")
    if C is not None:
        _need_matrix(C, "C", rows=m, cols=n)
    _need_cuda(A, "A")
    _need_cuda(B, "B")
    h = handle or default_handle()
    Ac, Bc = colmajor(A), colmajor(B)
    Cc = colmajor(C.clone()) if C is not None else torch.zeros((n, m), dtype=torch.float64, device=A.device).t()
    kp = min(max(k, 1), 4096)
    h.ensure_workspace(8 * (m + n) * (kp + 32) * 2 + 4 * (m + n) + 8192)
    _check(h.lib.gep_dgemm(h.h, transa.encode(), transb.encode(), uplo.encode(), m, n, k, float(alpha), _ptr(Ac),
                           _ld(Ac), _ptr(Bc), _ld(Bc), float(beta), _ptr(Cc), _ld(Cc), _PRECS[engine]), "gep_dgemm")
    return Cc


# ------------------------------------------------------------------ adjoint

def adjoint(w, Y, n_occ, lbar=None, W=None, handle=None):
    """(Abar, Bbar) of loss = sum_k lbar_k lambda_k + <W, Y_o Y_o^T> (gep_adjoint).

    w: eigenvalues ascending, Y: B-orthonormal eigenvectors (both from solve);
    lbar: M weights (None = 1 on the n_occ occupied, 0 elsewhere); W: M x M or None (both
    triangles are read; the library uses its symmetric part (W + W^T) / 2)."""
    torch = _torch()
    _need_vector(w, "w", 0, cuda=False)
    M = int(w.shape[0])
    _need_matrix(Y, "Y", rows=M, cols=M, cuda=False)
    if not 0 <= int(n_occ) <= M:
        raise ValueError(f"n_occ must lie in [0, {M}]")
    if lbar is not None:
        _need_vector(lbar, "lbar", M, cuda=False)
    if W is not None:
        _need_matrix(W, "W", rows=M, cols=M, cuda=False)
    _need_on_device("w", w, "Y", Y, "lbar", lbar, "W", W)
    h = handle or default_handle()
    Yc = colmajor(Y)
    ww = w.to(torch.float64).contiguous()
    lb = None if lbar is None else lbar.to(torch.float64).contiguous()
    Wc = None if W is None else colmajor(W)
    Ab = torch.empty((M, M), dtype=torch.float64, device=w.device).t()
    Bb = torch.empty((M, M), dtype=torch.float64, device=w.device).t()
    n = _SZ()
    _check(h.lib.gep_adjoint_workspace_size(h.h, M, int(n_occ), ctypes.byref(n)), "gep_adjoint_workspace_size")
    h.ensure_workspace(n.value)
    _check(h.lib.gep_adjoint(h.h, M, int(n_occ), _ptr(ww), _ptr(Yc), _ld(Yc), _ptr(lb), _ptr(Wc),
                             _ld(Wc) if Wc is not None else max(1, M), _ptr(Ab), _ptr(Bb), max(1, M)), "gep_adjoint")
    return Ab, Bb


def _autograd_function():
    torch = _torch()

    class GEPDensity(torch.autograd.Function):
        """(lambda, P) = eigenvalues and occupied density matrix P = Y_o Y_o^T of the pencil
        (A, B); backward by the hand-written adjoint (no eigenvectors of the perturbation
        are stored, only w and Y of the forward solve)."""

        @staticmethod
        def forward(ctx, A, B, n_occ, precision="fp64_emulated"):
            w, Y, info = solve(A.detach(), B.detach(), precision=precision)
            if info != 0:
                raise GepError(info, "gep_solve (forward)")
            Yc = colmajor(Y)
            Yo = Yc[:, :n_occ]
            P = dgemm(Yo, Yo, "N", "T", engine=precision if precision != "mixed_refined" else "fp64_emulated")
            ctx.save_for_backward(w, Yc)
            ctx.n_occ = int(n_occ)
            return w, P.contiguous()

        @staticmethod
        def backward(ctx, gw, gP):
            w, Yc = ctx.saved_tensors
            lbar = None if gw is None else gw.contiguous()
            if lbar is None:
                lbar = torch.zeros_like(w)
            # gep_adjoint reads both triangles of the cotangent and uses its symmetric part
            Ab, Bb = adjoint(w, Yc, ctx.n_occ, lbar, gP)
            return Ab.contiguous(), Bb.contiguous(), None, None

    return GEPDensity


_GEPDensity = None


def eigh_density(A, B, n_occ, precision="fp64_emulated"):
    """Differentiable (lambda, P = Y_o Y_o^T) of the pencil (A, B)."""
    global _GEPDensity
    if _GEPDensity is None:
        _GEPDensity = _autograd_function()
    return _GEPDensity.apply(A, B, n_occ, precision)


# ------------------------------------------------------------------ batched

SIZE_BUCKETS = (128, 256, 512, 1024, 2048, 4096)


def shard_batch(orders, world):
    """Longest-processing-time partition of independent pencils over `world` ranks:
    pencils in decreasing M^3 (ties: lower index first), each to the rank with the least
    assigned M^3 so far (ties: lower rank).  Returns one ascending index list per rank.
    The batched form needs no exchange between ranks: each solves its own pencils."""
    world = max(1, int(world))
    order = sorted(range(len(orders)), key=lambda i: (-float(orders[i]) ** 3, i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(orders[i]) ** 3
    return [sorted(p) for p in parts]


def _bucket(M):
    for b in SIZE_BUCKETS:
        if M <= b:
            return b
    return SIZE_BUCKETS[-1]


class Autotuner:
    """Per size bucket, the fastest route of one pencil of the bucket: the FP64-accurate
    product engine (FP64 FMA tiles or split-BF16 tensor-core tiles) and the SEP reduction
    (1-stage tridiagonalisation or full -> band -> tridiagonal); and, for the pencils of
    order <= 128, whether solving each whole in one CTA of one persistent launch
    (batch_small) beats the staged workflow on concurrent streams, timed on the batch."""

    def __init__(self):
        self.choice = {}      # bucket -> engine
        self.sep_choice = {}  # bucket -> SEP reduction
        self.batch_small = 0

    def tune_small(self, As, Bs, nstreams=16, reps=1, precision=None):
        """Times the whole batch both ways (pencils of order <= 128 in one persistent launch of
        one CTA each, or all of them on the streams, with the tuned routes, or with
        `precision` for every pencil when given) and keeps the faster: sets self.batch_small.
        The whole batch is timed because the two routes share the GPU with the larger
        pencils."""
        import time
        torch = _torch()
        if not any(int(a.shape[0]) <= 128 for a in As):
            self.batch_small = 0
            return self.batch_small
        best, best_t = 0, None
        for small in (128, 0):
            bs = BatchedSolver(As, Bs, nstreams=nstreams, batch_small=small,
                               precisions=[precision or self.precision_for(int(a.shape[0])) for a in As],
                               seps=[self.sep_for(int(a.shape[0])) for a in As])
            bs.run()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(reps):
                bs.run()
            torch.cuda.synchronize()
            t = (time.perf_counter() - t0) / reps
            if best_t is None or t < best_t:
                best, best_t = small, t
            bs.close()
        self.batch_small = best
        return best

    def tune(self, As, Bs, reps=2, seps=("1stage",), engines=("fp64", "fp64_emulated")):
        """Times every engine x SEP reduction (from `engines`, `seps`) on the first pencil of
        each size bucket and keeps the fastest; returns the engine per bucket (sep_for gives
        the reduction)."""
        import time
        torch = _torch()
        for A, B in zip(As, Bs):
            b = _bucket(int(A.shape[0]))
            if b in self.choice:
                continue
            best, best_t = None, None
            for sep in seps:
                for eng in engines:
                    solve(A, B, precision=eng, sep=sep)
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    for _ in range(reps):
                        solve(A, B, precision=eng, sep=sep)
                    torch.cuda.synchronize()
                    t = (time.perf_counter() - t0) / reps
                    if best_t is None or t < best_t:
                        best, best_t = (eng, sep), t
            self.choice[b], self.sep_choice[b] = best
        return self.choice

    def tune_routes(self, As, Bs, nstreams=16, thresholds=(None, 1024, 512, 0), precision=None):
        """Chooses, for the whole batch, the order above which pencils take the 2-stage route
        (None: none do): every candidate is captured into a graph and one replay is timed
        after a warm-up replay.  The 1-stage route launches six kernels per column, so its
        graphs are large; a candidate whose batch launches more kernels than one graph may
        hold (BatchedSolver.GRAPH_KERNEL_LIMIT) is skipped.  Sets sep_choice per bucket and
        returns the chosen threshold."""
        torch = _torch()
        best, best_t = None, None
        for T in thresholds:
            seps = ["2stage" if (T is not None and int(a.shape[0]) > T) else "1stage" for a in As]
            bs = BatchedSolver(As, Bs, nstreams=nstreams, batch_small=self.batch_small, seps=seps,
                               precisions=[precision or self.precision_for(int(a.shape[0])) for a in As])
            try:
                bs.capture()
            except ValueError:
                bs.close()
                continue
            bs.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            bs.replay()
            e1.record()
            torch.cuda.synchronize()
            t = e0.elapsed_time(e1)
            bs.close()
            if best_t is None or t < best_t:
                best, best_t = T, t
        self.sep_threshold = best
        for b in SIZE_BUCKETS:
            self.sep_choice[b] = "2stage" if (best is not None and b > best) else "1stage"
        return best

    def precision_for(self, M):
        return self.choice.get(_bucket(M), "fp64_emulated")

    def sep_for(self, M):
        if getattr(self, "sep_threshold", "unset") != "unset":
            T = self.sep_threshold
            return "2stage" if (T is not None and M > T) else "1stage"
        return self.sep_choice.get(_bucket(M), "1stage")


class BatchedSolver:
    """Many independent pencils (A_i, B_i) solved by gep_solve_batched_opts over `nstreams`
    concurrent streams, each pencil with its own route (precisions / seps per pencil, else
    precision / sep for all); capture() records the whole batch into one CUDA graph that
    replay() launches again (inputs are read from the same device buffers each time).
    batch_small > 0 (default 128): pencils of order <= batch_small (at most 128) are solved
    whole by one CTA each, all in one persistent launch; 0 puts every pencil on the streams.

    capture() refuses a batch whose eager run launched more than GRAPH_KERNEL_LIMIT kernels:
    graphs of about two million kernel nodes or more ended in a host crash inside the graph
    launch on this GPU's driver, with a GPU fault reported for the process.  Split such a
    batch, or give its larger pencils the 2-stage route (far fewer launches per pencil)."""

    GRAPH_KERNEL_LIMIT = 1_500_000

    def __init__(self, As, Bs, nstreams=8, precision="fp64_emulated", precisions=None, handle=None, batch_small=128,
                 sep="1stage", seps=None):
        torch = _torch()
        if len(As) != len(Bs) or len(As) == 0:
            raise ValueError("As and Bs must be non-empty lists of the same length")
        for i, (a, b) in enumerate(zip(As, Bs)):
            _need_matrix(a, f"As[{i}]", square=True, f64=True, cuda=False)
            _need_matrix(b, f"Bs[{i}]", rows=a.shape[0], cols=a.shape[0], f64=True, cuda=False)
            _need_on_device(f"As[{i}]", a, f"Bs[{i}]", b)
        n = len(As)
        if precisions is not None and len(precisions) != n:
            raise ValueError("precisions must give one entry per pencil")
        if seps is not None and len(seps) != n:
            raise ValueError("seps must give one entry per pencil")
        self._own_handle = handle is None
        self.h = handle or Handle()
        self.count = n
        self.As = [a.contiguous() for a in As]
        self.Bs = [b.contiguous() for b in Bs]
        self.M = [int(a.shape[0]) for a in self.As]
        dev = self.As[0].device
        self.w = [torch.empty(m, dtype=torch.float64, device=dev) for m in self.M]
        self.Yt = [torch.empty((m, m), dtype=torch.float64, device=dev) for m in self.M]
        self.nstreams = int(nstreams)
        self.opts = (GepOptions * n)()
        for i in range(n):
            self.opts[i] = make_options(precision=precisions[i] if precisions is not None else precision,
                                        sep=seps[i] if seps is not None else sep, batch_small=batch_small)
        self._M = (ctypes.c_int * n)(*self.M)
        self._A = (_P * n)(*[a.data_ptr() for a in self.As])
        self._B = (_P * n)(*[b.data_ptr() for b in self.Bs])
        self._w = (_P * n)(*[x.data_ptr() for x in self.w])
        self._Y = (_P * n)(*[y.data_ptr() for y in self.Yt])
        nb = _SZ()
        _check(self.h.lib.gep_solve_batched_opts_workspace_size(self.h.h, n, self._M, self.opts, self.nstreams,
                                                                 ctypes.byref(nb)),
               "gep_solve_batched_opts_workspace_size")
        self.h.ensure_workspace(nb.value)
        self.graph = None
        self.graph_kernels = 0
        self.eager_kernels = 0

    def run(self):
        _check(self.h.lib.gep_solve_batched_opts(self.h.h, self.count, self._M, self._A, self._B, self._w, self._Y,
                                                 self.opts, self.nstreams), "gep_solve_batched_opts")

    def capture(self):
        torch = _torch()
        self.h.launches(reset=True)
        self.run()  # eager first call creates the child streams outside the capture
        torch.cuda.synchronize()
        self.eager_kernels = self.h.launches(reset=True)
        if self.eager_kernels > self.GRAPH_KERNEL_LIMIT:
            raise ValueError(f"the batch launches {self.eager_kernels} kernels, more than one graph may hold "
                             f"({self.GRAPH_KERNEL_LIMIT}); split it or give its larger pencils the 2-stage route")
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        _check(self.h.lib.gep_set_stream(self.h.h, ctypes.c_void_p(s.cuda_stream)), "gep_set_stream")
        try:
            with torch.cuda.graph(g, stream=s):
                self.run()
            self.graph_kernels = self.h.launches(reset=True)  # kernel launches recorded in the graph
        finally:
            _check(self.h.lib.gep_set_stream(self.h.h, ctypes.c_void_p(self.h.stream.cuda_stream)),
                   "gep_set_stream")
        self.graph = g
        return g

    def close(self):
        """Releases the graph and, when this solver created it, the handle's workspace."""
        self.graph = None
        if self._own_handle:
            self.h.close()
            self.h.ws = None

    def replay(self):
        self.graph.replay()

    def info(self):
        v = _I()
        _check(self.h.lib.gep_batched_info(self.h.h, ctypes.byref(v)), "gep_batched_info")
        return v.value

    def results(self):
        return [(w, Yt.t()) for w, Yt in zip(self.w, self.Yt)]
