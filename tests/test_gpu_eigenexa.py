"""The Cholesky-free ("EigenExa style") reducer of Eq. 7-9 on the GPU, against the FP64 oracle.

B W = W D is solved by the library's own SEP solver (Eq. 7), A' = D^-1/2 W^T A W D^-1/2 is
formed by two engine products (Eq. 8) and solved by the SEP solver again, and Y = W D^-1/2 Z
(Eq. 9).  The result must match both the oracle's Eq. 7-9 route and its Cholesky route at the
FP64 tolerances (the paper's workflows B and H of Table 1 solve the same pencil).
"""
import numpy as np
import pytest

import gep_inputs as gi

pytestmark = pytest.mark.gpu

EPS = 2.0 ** -52


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


def _pencil(oracle_lib, M):
    if M not in _REF:
        tb = gi.tight_binding(M, seed=M + 11) if M % 4 == 0 else gi.known_spectrum(M, seed=M)
        A, B = tb["A"], tb["B"]
        we, Ye, ie = oracle_lib.gep_solve_eigenexa(A, B)
        wc, Yc, ic = oracle_lib.gep_solve(A, B)
        assert ie == 0 and ic == 0
        _REF[M] = dict(A=A, B=B, we=we, Ye=Ye, wc=wc, nA=float(np.max(np.abs(np.linalg.eigvalsh(A)))))
    return _REF[M]


@pytest.mark.parametrize("M,sep,precision", [
    (129, "1stage", "fp64"), (129, "2stage", "fp64_emulated"),
    (516, "1stage", "fp64_emulated"), (516, "2stage", "fp64_emulated"), (516, "2stage", "mixed_refined"),
    (1280, "2stage", "fp64_emulated"), (1280, "1stage", "fp64")])
def test_eigenexa_solve_vs_oracle(gep, oracle_lib, M, sep, precision):
    p = _pencil(oracle_lib, M)
    A, B, nA = p["A"], p["B"], p["nA"]
    w, Y, info = gep.solve(dev(A), dev(B), reducer="eigenexa", sep=sep, precision=precision)
    assert info == 0
    wh, Yh = host(w), host(Y)
    assert np.max(np.abs(wh - p["we"])) <= 1e-11 * nA  # the oracle's Eq. 7-9 route
    assert np.max(np.abs(wh - p["wc"])) <= 1e-11 * nA  # and its Cholesky route
    res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Yh.T @ B @ Yh - np.eye(M)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth
    gaps = np.minimum(np.diff(p["we"], prepend=-np.inf), np.diff(p["we"], append=np.inf))
    iso = gaps > 1e-6 * nA
    assert np.max(np.abs(Yh[:, iso] - p["Ye"][:, iso])) <= 1e-8


def test_eigenexa_values_only_and_timers(gep, oracle_lib):
    p = _pencil(oracle_lib, 516)
    h = gep.Handle()
    w, Y, info = gep.solve(dev(p["A"]), dev(p["B"]), reducer="eigenexa", sep="2stage",
                           precision="fp64_emulated", want_vectors=False, timers=True, handle=h)
    assert info == 0 and Y is None
    assert np.max(np.abs(host(w) - p["we"])) <= 1e-11 * p["nA"]
    t = h.stage_times()
    assert t[0] > 0 and t[1] > 0 and t[2] > 0  # SEP of B, forming A', reduction of A'


def test_eigenexa_known_spectrum(gep):
    g = gi.known_spectrum(300, seed=8)
    w, Y, info = gep.solve(dev(g["A"]), dev(g["B"]), reducer="eigenexa", sep="2stage", precision="fp64_emulated")
    assert info == 0
    assert np.max(np.abs(host(w) - np.sort(g["lam"]))) <= 1e-11 * 20.0


def test_eigenexa_stage_entry_points(gep, oracle_lib):
    """gep_reduce(EIGENEXA) leaves X = W D^-1/2 (X^T B X = I) and A' = X^T A X, whose spectrum
    is the pencil's; gep_backtransform(EIGENEXA) maps eigenvectors of A' to Y = X Z."""
    p = _pencil(oracle_lib, 129)
    A, B, M = p["A"], p["B"], 129
    C, X = gep.reduce(dev(A), dev(B), variant="eigenexa")
    Ch, Xh = host(C), host(X)
    assert np.max(np.abs(Xh.T @ B @ Xh - np.eye(M))) <= 1e-12
    assert np.max(np.abs(Ch - Ch.T)) == 0.0
    assert np.max(np.abs(Ch - Xh.T @ A @ Xh)) <= 1e-12 * p["nA"]
    lam, Z, st = oracle_lib.tql(*_tridiag(oracle_lib, Ch))
    assert st == 0
    assert np.max(np.abs(np.sort(lam) - p["wc"])) <= 1e-11 * p["nA"]
    Y = host(gep.gep_backtransform(X, dev(Z), variant="eigenexa"))
    assert np.max(np.abs(Y - Xh @ Z)) <= 1e-13 * max(1.0, np.max(np.abs(Y)))


def _tridiag(oracle_lib, C):
    """(d, e, Q) of the oracle's Householder tridiagonalisation of C (then QL on T with Q)."""
    d, e, Q = oracle_lib.tridiag(C)
    return d, e, Q


def test_eigenexa_reports_indefinite_B(gep, oracle_lib):
    """B with two negative eigenvalues: the count of non-positive eigenvalues of B is the
    status, as in the oracle, and no NaN leaks out as a result."""
    rng = np.random.default_rng(22)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    dB = np.array([1.0, -0.5, 2.0, 3.0, -4.0, 1.5, 2.5, 0.7, 1.1, 1.9, 2.2, 3.3])
    B = (Q * dB[None, :]) @ Q.T
    B = 0.5 * (B + B.T)
    _, _, info_ref = oracle_lib.gep_solve_eigenexa(np.eye(12), B)
    assert info_ref == 2
    h = gep.Handle()
    _, _, info = gep.solve(dev(np.eye(12)), dev(B), reducer="eigenexa", handle=h)
    assert info == 2
