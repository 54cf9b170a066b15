"""Parity at the benchmark's full size: the M = 32768 tight-binding pencil (8192 atoms, seed 0)
solved on the benchmark's route (two-stage reduction, FP64-accurate split-BF16 products), checked
through properties that hold at any size and need none of the solver's code:

* eigenvalues ascending;
* 64 seeded sample eigenpairs: residual ||A y - lambda B y||, Rayleigh quotient
  y^T A y / y^T B y = lambda, and B-orthonormality among the sampled vectors (plain torch FP64);
* the lowest eigenvalue bracketed independently (Sylvester's law for the pencil): A - sigma B
  is positive definite for sigma = lambda_min - delta and not for sigma = lambda_min + delta,
  decided by a library Cholesky factorisation.

The oracle itself cannot solve this size in test time; the smaller parity tests compare with it
element by element.  This file sorts after the other GPU tests.
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


def test_full_size_benchmark_route(gep):
    import torch
    M = 32768
    tb = gi.tight_binding(M, seed=0)
    A = torch.as_tensor(tb["A"], device="cuda")
    B = torch.as_tensor(tb["B"], device="cuda")
    del tb
    w, Y, info = gep.solve(A, B, sep="2stage", precision="fp64_emulated")
    assert info == 0
    assert bool(torch.all(w[1:] >= w[:-1]))
    normA = float(torch.linalg.matrix_norm(A))  # Frobenius, >= ||A||_2

    cols = torch.as_tensor(np.sort(np.random.default_rng(0).choice(M, 64, replace=False)), device="cuda")
    Ys = Y[:, cols].contiguous()
    lam = w[cols]
    AY = A @ Ys
    BY = B @ Ys
    R = AY - BY * lam[None, :]
    # the full residual ||AY - BY Lambda||_F / (||A||_F M) estimated from the sample
    res_est = float(torch.sqrt(torch.mean(torch.sum(R * R, dim=0)) * M)) / (normA * M)
    assert res_est <= 1e-13, res_est
    rq = torch.sum(Ys * AY, dim=0) / torch.sum(Ys * BY, dim=0)
    assert float(torch.max(torch.abs(rq - lam))) <= 1e-11 * normA
    G = Ys.t() @ BY
    assert float(torch.max(torch.abs(G - torch.eye(64, dtype=G.dtype, device=G.device)))) <= 1e-12
    del AY, BY, R, Y, Ys

    # lambda_min bracketed by two library Cholesky factorisations of A - sigma B
    delta = 1e-9 * normA
    lam0 = float(w[0])
    _, info_lo = torch.linalg.cholesky_ex(A - (lam0 - delta) * B)
    assert int(info_lo) == 0
    _, info_hi = torch.linalg.cholesky_ex(A - (lam0 + delta) * B)
    assert int(info_hi) > 0
