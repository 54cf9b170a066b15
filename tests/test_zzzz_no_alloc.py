"""The allocation-free product entry point, called through the C ABI.

gep_dgemm_emulated_noalloc serves callers that cannot call cudaMalloc (a framework
that owns all device memory through its own pool, a latency-critical loop that must
not let a library allocate mid-run): its scratch is a fixed device array inside the
library.  Its result must match the handle-based gep_dgemm with the same engine, and the
plain FP64 product alpha op(A) op(B) + beta C computed on the host, to the rounding bound
the engine tests use, on two calls in a row (the second call runs on the scratch the first
one left behind).  This file sorts after every other test file on purpose, so that a run
stopping at its first failure has already run the rest.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

GEP_ERR_TOO_LARGE = -106


@pytest.fixture(scope="module")
def lib():
    import torch
    assert torch.cuda.is_available()
    from paper_1504_06443_gb300 import build
    build.build()
    import paper_1504_06443_gb300 as g
    lib = g.load()
    f = lib.gep_dgemm_emulated_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_char, ctypes.c_char, ctypes.c_char, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                  ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_double,
                  ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]
    return g, f


def _noalloc(f, ta, tb, A, B, C, alpha, beta):
    import torch
    m = A.shape[1] if ta == b"T" else A.shape[0]
    k = A.shape[0] if ta == b"T" else A.shape[1]
    n = B.shape[0] if tb == b"T" else B.shape[1]
    stream = torch.cuda.current_stream().cuda_stream
    rc = f(ta, tb, b"F", m, n, k, alpha, ctypes.c_void_p(A.data_ptr()), A.stride(1),
           ctypes.c_void_p(B.data_ptr()), B.stride(1), beta, ctypes.c_void_p(C.data_ptr()), C.stride(1),
           ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("ta,tb,m,n,k", [(b"N", b"N", 300, 200, 500), (b"T", b"N", 257, 130, 5000),
                                         (b"N", b"T", 129, 65, 33)])
def test_noalloc_matches_handle_path_twice(lib, ta, tb, m, n, k):
    import torch
    g, f = lib
    for call in range(2):
        rng = np.random.default_rng(100 * call + m + k)
        Ah = rng.standard_normal((k, m) if ta == b"T" else (m, k))
        Bh = rng.standard_normal((n, k) if tb == b"T" else (k, n))
        Ch = rng.standard_normal((m, n))
        A = g.colmajor(torch.as_tensor(Ah, device="cuda"))
        B = g.colmajor(torch.as_tensor(Bh, device="cuda"))
        C = g.colmajor(torch.as_tensor(Ch, device="cuda"))
        ref = g.dgemm(A, B, ta.decode(), tb.decode(), alpha=1.25, beta=-0.5, C=C, engine="fp64_emulated")
        out = C.clone()
        assert _noalloc(f, ta, tb, A, B, out, 1.25, -0.5) == 0
        Ao = Ah.T if ta == b"T" else Ah
        Bo = Bh.T if tb == b"T" else Bh
        bound = 1e-14 * (1.25 * np.abs(Ao) @ np.abs(Bo) + 0.5 * np.abs(Ch))
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got)), call  # NaN would mean a device-side failure
        diff = np.abs(got - ref.cpu().numpy())
        assert np.all(diff <= bound), (call, float(diff.max()))
        exact = 1.25 * (Ao @ Bo) - 0.5 * Ch  # plain FP64 product on the host
        diff = np.abs(got - exact)
        assert np.all(diff <= bound), (call, float(diff.max()))


def test_noalloc_rejects_too_large(lib):
    g, f = lib
    rc = f(b"N", b"N", b"F", 100000, 100000, 64, 1.0, None, 100000, None, 64, 0.0, None, 100000, None)
    assert rc == GEP_ERR_TOO_LARGE
