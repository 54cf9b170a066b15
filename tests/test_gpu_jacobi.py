"""The block-Jacobi SEP solver (GEP_SEP_JACOBI, the parallel block-Jacobi method the paper
names as future work in section 6) against the FP64 oracle: whole solves with every
reducer, eigenvalues only, the lowest-n option, a single block (M <= 32), ragged blocks,
and agreement with the tridiagonal routes."""
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


def _pencil(M):
    return gi.tight_binding(M, seed=M + 31) if M % 4 == 0 else gi.known_spectrum(M, seed=M)


@pytest.mark.parametrize("M,reducer", [(20, "twosided"), (64, "twosided"), (97, "explicit_inv"),
                                       (132, "twosided"), (300, "eigenexa"), (516, "twosided")])
def test_jacobi_solve_vs_oracle(gep, oracle_lib, M, reducer):
    p = _pencil(M)
    A, B = p["A"], p["B"]
    w_ref, Y_ref, info = oracle_lib.gep_solve(A, B)
    assert info == 0
    w, Y, info = gep.solve(dev(A), dev(B), sep="jacobi", reducer=reducer, precision="fp64_emulated")
    assert info == 0
    wh, Yh = host(w), host(Y)
    nA = float(np.max(np.abs(np.linalg.eigvalsh(A))))
    assert np.max(np.abs(wh - w_ref)) <= 1e-11 * nA
    res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Yh.T @ B @ Yh - np.eye(M)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth
    gaps = np.minimum(np.diff(w_ref, prepend=-np.inf), np.diff(w_ref, append=np.inf))
    iso = gaps > 1e-6 * nA
    assert np.max(np.abs(Yh[:, iso] - Y_ref[:, iso])) <= 1e-8


def test_jacobi_values_only_and_partial(gep, oracle_lib):
    M = 260
    p = _pencil(M)
    A, B = p["A"], p["B"]
    w_ref, _, info = oracle_lib.gep_solve(A, B, want_vectors=False)
    nA = float(np.max(np.abs(np.linalg.eigvalsh(A))))
    w, Y, info = gep.solve(dev(A), dev(B), sep="jacobi", want_vectors=False)
    assert info == 0 and Y is None
    assert np.max(np.abs(host(w) - w_ref)) <= 1e-11 * nA
    w, Y, info = gep.solve(dev(A), dev(B), sep="jacobi", n_want=100)
    assert info == 0
    wh, Yh = host(w), host(Y)
    assert np.max(np.abs(wh - w_ref[:100])) <= 1e-11 * nA
    assert np.max(np.abs(Yh.T @ B @ Yh - np.eye(100))) <= 1e-12
    res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
    assert res <= 1e-13


def test_jacobi_agrees_with_tridiagonal_routes(gep):
    g = gi.known_spectrum(200, seed=9)
    A, B = dev(g["A"]), dev(g["B"])
    w1, _, _ = gep.solve(A, B, sep="jacobi")
    w2, _, _ = gep.solve(A, B, sep="2stage", precision="fp64_emulated")
    assert np.max(np.abs(host(w1) - np.sort(g["lam"]))) <= 1e-11 * 20.0
    assert np.max(np.abs(host(w1) - host(w2))) <= 1e-11 * 20.0
