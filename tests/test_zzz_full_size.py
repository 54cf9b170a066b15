"""Parity at the benchmark's full size: the M = 32768 tight-binding pencil (8192 atoms, seed 0)
solved on the benchmark's route (two-stage reduction, FP64-accurate split-BF16 products), checked
through properties that hold at any size and need none of the solver's code:

* eigenvalues ascending;
* 64 seeded sample eigenpairs: residual ||A y - lambda B y||, Rayleigh quotient
  y^T A y / y^T B y = lambda, and B-orthonormality among the sampled vectors (plain torch FP64);
* the lowest eigenvalue bracketed independently (Sylvester's law for the pencil): A - sigma B
  is positive definite for sigma = lambda_min - delta and not for sigma = lambda_min + delta,
  decided by a library Cholesky factorisation;
* Sylvester inertia at interior shifts: the number of eigenvalues below sigma equals the
  number of negative eigenvalues of the block-diagonal D of a library LDL^T factorisation of
  A - sigma B (so no eigenvalue is missing or duplicated between the shifts);
* the sum of the eigenvalues equals trace(B^-1 A) = trace(L^-1 A L^-T), computed with a
  library Cholesky factor and triangular solve.

The oracle itself cannot solve this size in test time; the smaller parity tests compare with it
element by element.  This file sorts after the other GPU tests.
"""
import numpy as np
import pytest

import gep_inputs as gi
from inertia import negative_eigenvalues_of_ldl

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


def test_full_size_inertia_and_trace(gep):
    import torch
    M = 32768
    tb = gi.tight_binding(M, seed=0)
    A = torch.as_tensor(tb["A"], device="cuda")
    B = torch.as_tensor(tb["B"], device="cuda")
    del tb
    w, _, info = gep.solve(A, B, sep="2stage", precision="fp64_emulated", want_vectors=False)
    assert info == 0
    wh = w.cpu().numpy()
    normA = float(torch.linalg.matrix_norm(A))
    # shifts in the widest gap near the 1/4, 1/2 and 3/4 quantiles of the spectrum
    for q in (0.25, 0.5, 0.75):
        c = int(q * M)
        lo, hi = c - 200, c + 200
        k = lo + int(np.argmax(wh[lo + 1:hi + 1] - wh[lo:hi]))
        gap = wh[k + 1] - wh[k]
        assert gap > 1e-9 * normA, (q, gap)
        sigma = 0.5 * (wh[k] + wh[k + 1])
        LD, piv, linfo = torch.linalg.ldl_factor_ex(A - sigma * B)
        assert int(linfo) == 0
        assert negative_eigenvalues_of_ldl(LD, piv) == k + 1, q
        del LD, piv
    # sum of eigenvalues = trace(L^-1 A L^-T) = trace(B^-1 A) = sum_ij (B^-1)_ij A_ij,
    # B^-1 from a library Cholesky factor of B
    Binv = torch.cholesky_inverse(torch.linalg.cholesky(B))
    tr = float(torch.sum(Binv * A))
    del Binv
    ssum = float(np.sum(wh))
    assert abs(ssum - tr) <= 1e-11 * normA * M ** 0.5, (ssum, tr)
