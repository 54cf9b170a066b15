"""The lowest n eigenpairs (the occupied states of the paper's section 2) on the GPU, against
the oracle's bisection + inverse iteration (an algorithm that shares no step with the GPU's
divide and conquer with pruned back-transformations).

Eigenvalues compare element by element; eigenvectors element by element where isolated
(both sides apply the sign convention), and everywhere through the residual and
B-orthonormality of the M x n block.
"""
import numpy as np
import pytest

import gep_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gep():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1504_06443_gb300 import build
    build.build()
    import paper_1504_06443_gb300 as g
    g.load()
    return g


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


_REF = {}


def _ref(oracle_lib, M, n):
    key = (M, n)
    if key not in _REF:
        tb = gi.tight_binding(M, seed=M + 21)
        w, Y, info = oracle_lib.gep_solve_partial(tb["A"], tb["B"], n)
        assert info == 0
        wall, _, info = oracle_lib.gep_solve(tb["A"], tb["B"], want_vectors=False)
        assert info == 0
        _REF[key] = dict(A=tb["A"], B=tb["B"], w=w, Y=Y, wall=wall,
                         nA=float(np.max(np.abs(np.linalg.eigvalsh(tb["A"])))))
    return _REF[key]


def _check(p, wh, Yh, n):
    A, B, nA = p["A"], p["B"], p["nA"]
    M = A.shape[0]
    assert wh.shape == (n,)
    assert np.max(np.abs(wh - p["w"])) <= 1e-11 * nA
    if Yh is None:
        return
    assert Yh.shape == (M, n)
    res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Yh.T @ B @ Yh - np.eye(n)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth
    # isolation judged on the whole spectrum (the n-th eigenvalue's upper neighbour counts)
    wall = p["wall"]
    gaps = np.minimum(np.diff(wall, prepend=-np.inf), np.diff(wall, append=np.inf))[:n]
    iso = gaps > 1e-6 * nA
    if iso.any():
        assert np.max(np.abs(Yh[:, iso] - p["Y"][:, iso])) <= 1e-8


@pytest.mark.parametrize("M,n,sep,reducer,precision", [
    (516, 1, "2stage", "twosided", "fp64_emulated"),
    (516, 258, "2stage", "twosided", "fp64_emulated"),
    (516, 258, "1stage", "explicit_inv", "fp64"),
    (516, 516, "2stage", "twosided", "fp64_emulated"),
    (1280, 640, "2stage", "twosided", "fp64_emulated"),
    (1280, 77, "1stage", "twosided", "fp64_emulated"),
    (1280, 640, "2stage", "eigenexa", "fp64_emulated")])
def test_partial_spectrum_vs_oracle(gep, oracle_lib, M, n, sep, reducer, precision):
    p = _ref(oracle_lib, M, n)
    w, Y, info = gep.solve(dev(p["A"]), dev(p["B"]), n_want=n, sep=sep, reducer=reducer, precision=precision)
    assert info == 0
    _check(p, host(w), host(Y), n)


@pytest.mark.parametrize("sep", ["1stage", "2stage"])
def test_partial_values_only(gep, oracle_lib, sep):
    p = _ref(oracle_lib, 1280, 640)
    w, Y, info = gep.solve(dev(p["A"]), dev(p["B"]), n_want=640, want_vectors=False, sep=sep,
                           precision="fp64_emulated")
    assert info == 0 and Y is None
    _check(p, host(w), None, 640)


def test_partial_host_buffers(gep, oracle_lib):
    """gep_solve_host with n_want: the w[n] and M x n host outputs."""
    p = _ref(oracle_lib, 516, 258)
    w, Y, info = gep.solve_host(p["A"], p["B"], n_want=258, sep="2stage", precision="fp64_emulated")
    assert info == 0
    _check(p, w, Y, 258)


def test_partial_rejections(gep):
    import torch
    A = dev(np.eye(16))
    with pytest.raises(ValueError):
        gep.solve(A, A, n_want=17)
    with pytest.raises(gep.GepError):
        gep.solve(A, A, n_want=4, precision="mixed_refined")
    import ctypes
    h = gep.default_handle()
    o = gep.make_options(n_want=17)
    w = torch.empty(16, dtype=torch.float64, device="cuda")
    Y = torch.empty((16, 16), dtype=torch.float64, device="cuda")
    rc = h.lib.gep_solve(h.h, 16, ctypes.c_void_p(A.data_ptr()), 16, ctypes.c_void_p(A.data_ptr()), 16,
                         ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(Y.data_ptr()), 16, ctypes.byref(o))
    assert rc == -10
