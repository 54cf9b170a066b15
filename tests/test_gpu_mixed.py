"""Mixed-precision solve (FP32-grade split-BF16 products and FP32 SYMVs) followed by FP64
refinement of all eigenpairs must meet the FP64 tolerances against the FP64 oracle."""
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


@pytest.mark.parametrize("M,reducer", [(260, "twosided"), (516, "explicit_inv"), (1280, "twosided")])
def test_mixed_refined_meets_fp64_tolerances(gep, oracle_lib, M, reducer):
    tb = gi.tight_binding(M, seed=M + 7)
    A, B = tb["A"], tb["B"]
    w_ref, _, info = oracle_lib.gep_solve(A, B)
    assert info == 0
    w, Y, info = gep.solve(dev(A), dev(B), precision="mixed_refined", reducer=reducer)
    assert info == 0
    wh, Yh = w.cpu().numpy(), Y.cpu().numpy()
    nA = float(np.max(np.abs(np.linalg.eigvalsh(A))))
    assert np.max(np.abs(wh - w_ref)) <= 1e-11 * nA
    res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Yh.T @ B @ Yh - np.eye(M)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth


def test_mixed_known_spectrum(gep):
    g = gi.known_spectrum(512, seed=3)
    w, Y, info = gep.solve(dev(g["A"]), dev(g["B"]), precision="mixed_refined")
    assert info == 0
    assert np.max(np.abs(w.cpu().numpy() - np.sort(g["lam"]))) <= 1e-11 * 20.0


def test_mixed_clustered_spectrum(gep):
    """Planted clusters (1e-9 spacings and exact repeats) go through the exact cluster
    solve of the refinement; eigenvalues, residual and B-orthogonality reach FP64 level."""
    M = 384
    g = gi.clustered_spectrum(M, seed=11)
    A, B = g["A"], g["B"]
    h = gep.Handle()
    w, Y, info = gep.solve(dev(A), dev(B), precision="mixed_refined", handle=h)
    assert info == 0
    steps = h.refine_steps()
    assert 1 <= steps <= 8
    wh, Yh = w.cpu().numpy(), Y.cpu().numpy()
    assert np.max(np.abs(wh - np.sort(g["lam"]))) <= 1e-11 * 20.0
    res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Yh.T @ B @ Yh - np.eye(M)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth


def test_mixed_fixed_step_count(gep):
    """refine_iters > 0 runs exactly that many steps; the adaptive default stops on its own."""
    tb = gi.tight_binding(260, seed=267)
    h = gep.Handle()
    gep.solve(dev(tb["A"]), dev(tb["B"]), precision="mixed_refined", handle=h, refine_iters=3)
    assert h.refine_steps() == 3
    gep.solve(dev(tb["A"]), dev(tb["B"]), precision="mixed_refined", handle=h)
    assert 1 <= h.refine_steps() <= 8


def test_mixed_oversize_cluster(gep):
    """A run of 40 eigenvalues spaced 1e-9 apart chains into one cluster larger than the 32
    the refinement solves exactly; its inner pairs then only get their B-orthogonality
    restored.  The refined eigenpairs must still reach the FP64 tolerances."""
    M = 384
    g = gi.clustered_spectrum(M, seed=12, big=40)
    A, B = g["A"], g["B"]
    h = gep.Handle()
    w, Y, info = gep.solve(dev(A), dev(B), precision="mixed_refined", handle=h)
    assert info == 0
    assert 1 <= h.refine_steps() <= 8
    wh, Yh = w.cpu().numpy(), Y.cpu().numpy()
    assert np.max(np.abs(wh - np.sort(g["lam"]))) <= 1e-11 * 20.0
    res = np.linalg.norm(A @ Yh - (B @ Yh) * wh[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Yh.T @ B @ Yh - np.eye(M)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth
