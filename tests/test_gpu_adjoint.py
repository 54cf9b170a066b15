"""Adjoint of the generalized eigenproblem on the GPU (gep_adjoint / eigh_density)
against the FP64 oracle's adjoint and against central finite differences."""
import numpy as np
import pytest

import gep_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gep():
    import torch
    assert torch.cuda.is_available()
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


@pytest.mark.parametrize("M", [128, 260])
def test_adjoint_vs_oracle(gep, oracle_lib, M):
    tb = gi.tight_binding(M, seed=M + 1)
    A, B = tb["A"], tb["B"]
    n = M // 2
    W = gi.random_symmetric(M, seed=3)
    w_ref, Y_ref, info = oracle_lib.gep_solve(A, B)
    assert info == 0 and w_ref[n] - w_ref[n - 1] > 1e-6
    Ab_ref, Bb_ref = oracle_lib.adjoint(w_ref, Y_ref, n, np.ones(n), W)
    w, Y, info = gep.solve(dev(A), dev(B), precision="fp64_emulated")
    assert info == 0
    lbar = np.zeros(M)
    lbar[:n] = 1.0
    Ab, Bb = gep.adjoint(w, Y, n, dev(lbar), dev(W))
    scale = max(np.max(np.abs(Ab_ref)), np.max(np.abs(Bb_ref)))
    gap = w_ref[n] - w_ref[n - 1]
    tol = 1e-11 * scale / min(1.0, gap)
    assert np.max(np.abs(host(Ab) - Ab_ref)) <= tol
    assert np.max(np.abs(host(Bb) - Bb_ref)) <= tol


def test_adjoint_eigenvalue_sum_closed_form(gep):
    """W = 0, lbar = 1 on occupied: Abar = Y_o Y_o^T, Bbar = -Y_o Lambda_o Y_o^T."""
    tb = gi.tight_binding(200, seed=5)
    w, Y, info = gep.solve(dev(tb["A"]), dev(tb["B"]))
    n = 100
    Ab, Bb = gep.adjoint(w, Y, n, None, None)
    Yh, wh = host(Y), host(w)
    Yo = Yh[:, :n]
    assert np.max(np.abs(host(Ab) - Yo @ Yo.T)) <= 1e-13
    assert np.max(np.abs(host(Bb) + (Yo * wh[None, :n]) @ Yo.T)) <= 1e-12 * max(1.0, np.max(np.abs(wh)))


def test_autograd_central_differences(gep):
    """loss = sum_{k<n} lambda_k + <W, P> through eigh_density: autograd gradient vs central
    differences (h = 1e-6) of the GPU forward solve along 6 symmetric directions."""
    import torch
    M, n = 128, 64
    tb = gi.tight_binding(M, seed=12)
    A = dev(tb["A"]).requires_grad_(True)
    B = dev(tb["B"]).requires_grad_(True)
    W = dev(gi.random_symmetric(M, seed=1))

    def loss_of(A_, B_):
        w, P = gep.eigh_density(A_, B_, n)
        return w[:n].sum() + (W * P).sum()

    loss = loss_of(A, B)
    gA, gB = torch.autograd.grad(loss, (A, B))
    rng = np.random.default_rng(2)
    h = 1e-6
    with torch.no_grad():
        for _ in range(6):
            dA = rng.standard_normal((M, M)); dA = dA + dA.T
            dB = rng.standard_normal((M, M)); dB = dB + dB.T
            dA *= 1e-3 * np.linalg.norm(tb["A"]) / np.linalg.norm(dA)
            dB *= 0.05 / np.linalg.norm(dB)
            dAt, dBt = dev(dA), dev(dB)
            fd = (loss_of(A + h * dAt, B + h * dBt) - loss_of(A - h * dAt, B - h * dBt)).item() / (2 * h)
            an = float((gA * dAt).sum() + (gB * dBt).sum())
            assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (fd, an)
