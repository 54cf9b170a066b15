"""Parity of the CUDA path with the FP64 CPU oracle, stage by stage and end to end.

Inputs are seeded (gep_inputs); expected values come from the oracle on the same
inputs.  Sizes span several 64/128-wide tiles plus a ragged tail.  Tolerances are
the solver's FP64 accuracy target (|d lambda| <= 1e-11 ||A||_2, residual
||AY - BY Lambda||_F / (||A||_F M) <= 1e-13, ||Y^T B Y - I||_max <= 1e-12) or, for
intermediate quantities, a stated multiple of M * eps relative to the input scale.
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


@pytest.fixture(scope="module")
def torch_mod():
    import torch
    return torch


def dev(x):
    import torch
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def two_norm(A):
    return float(np.max(np.abs(np.linalg.eigvalsh(A))))


# ------------------------------------------------------------------ GEMM engine

@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (67, 130, 33), (200, 64, 129)])
def test_dgemm_fp64(gep, ta, tb, m, n, k):
    rng = np.random.default_rng(m * n + k)
    A = rng.standard_normal((k, m) if ta == "T" else (m, k))
    B = rng.standard_normal((n, k) if tb == "T" else (k, n))
    C = rng.standard_normal((m, n))
    ref = 0.7 * (A.T if ta == "T" else A) @ (B.T if tb == "T" else B) - 0.3 * C
    out = gep.dgemm(dev(A), dev(B), ta, tb, alpha=0.7, beta=-0.3, C=dev(C))
    assert np.max(np.abs(host(out) - ref)) <= 4 * k * EPS * np.max(np.abs(A)) * np.max(np.abs(B)) * 2 + 1e-14


def test_dgemm_lower_only(gep):
    rng = np.random.default_rng(0)
    A = rng.standard_normal((150, 40))
    C = rng.standard_normal((150, 150))
    out = host(gep.dgemm(dev(A), dev(A), "N", "T", alpha=-1.0, beta=1.0, C=dev(C), uplo="L"))
    ref = C - A @ A.T
    il = np.tril_indices(150)
    iu = np.triu_indices(150, 1)
    assert np.max(np.abs(out[il] - ref[il])) <= 1e-12
    assert np.array_equal(out[iu], C[iu])


# ------------------------------------------------------------------ reducer

@pytest.mark.parametrize("M", [1, 31, 128, 129, 300, 513])
def test_cholesky_vs_oracle(gep, oracle_lib, M):
    g = gi.known_spectrum(M, seed=M)
    L_ref, info_ref = oracle_lib.cholesky(g["B"])
    L, info = gep.cholesky(dev(g["B"]))
    assert info == 0 and info_ref == 0
    Lh = np.tril(host(L))
    assert np.max(np.abs(Lh - L_ref)) <= 64 * M * EPS * np.max(np.abs(L_ref))


@pytest.mark.parametrize("k", [1, 77, 130, 256])
def test_cholesky_reports_first_bad_minor(gep, oracle_lib, k):
    M = 300
    B = gi.spd_matrix(M, seed=k)
    L0 = np.linalg.cholesky(B)
    D = np.ones(M)
    D[k - 1] = -1.0
    Bk = (L0 * D[None, :]) @ L0.T
    Bk = 0.5 * (Bk + Bk.T)
    _, info_ref = oracle_lib.cholesky(Bk)
    _, info = gep.cholesky(dev(Bk))
    assert info == info_ref == k


@pytest.mark.parametrize("variant", ["twosided", "explicit_inv"])
@pytest.mark.parametrize("M", [64, 257, 400])
def test_reduce_vs_oracle(gep, oracle_lib, variant, M):
    tb = gi.tight_binding(M if M % 4 == 0 else M - M % 4 + 4, seed=3)
    A, B = tb["A"][:M, :M], tb["B"][:M, :M]
    L_ref, _ = oracle_lib.cholesky(B)
    C_ref = oracle_lib.two_sided(A, L_ref)
    L, info = gep.cholesky(dev(B))
    assert info == 0
    C, LR = gep.reduce(dev(A), L, variant)
    Ch = host(C)
    assert np.max(np.abs(Ch - Ch.T)) == 0.0
    assert np.max(np.abs(Ch - C_ref)) <= 1e-12 * max(1.0, np.max(np.abs(C_ref)))
    if variant == "explicit_inv":
        R = np.tril(host(LR))
        assert np.max(np.abs(R @ L_ref - np.eye(M))) <= 1e-12 * M


# ---------------------------------------------------------- SEP solver stages

@pytest.mark.parametrize("M", [1, 2, 3, 64, 65, 200, 333])
def test_tridiag_vs_oracle(gep, oracle_lib, M):
    rng = np.random.default_rng(M)
    G = rng.standard_normal((M, M))
    C = 0.5 * (G + G.T)
    d_ref, e_ref, Q_ref = oracle_lib.tridiag(C)
    d, e, tau, Cr = gep.tridiag_1stage(dev(C))
    scale = max(1.0, np.max(np.abs(C)))
    assert np.max(np.abs(host(d) - d_ref)) <= 200 * M * EPS * scale
    assert np.max(np.abs(host(e) - e_ref), initial=0.0) <= 200 * M * EPS * scale
    # Q from the reflectors: back-transform the identity and compare with the oracle's Q
    Q = host(gep.sep_backtransform(Cr, tau, dev(np.eye(M))))
    assert np.max(np.abs(Q - Q_ref)) <= 200 * M * EPS


def _tridiag_cases():
    rng = np.random.default_rng(7)
    cases = []
    for M in (1, 2, 31, 32, 33, 64, 100, 257, 700):
        cases.append((f"random{M}", rng.standard_normal(M), rng.standard_normal(max(M - 1, 0))))
    n = 300
    cases.append(("diagonal", rng.standard_normal(n), np.zeros(n - 1)))
    cases.append(("constant", np.full(n, 2.0), np.full(n - 1, 1e-9)))                 # heavy deflation
    k = np.arange(n)
    cases.append(("wilkinson", np.abs(k - n // 2).astype(float), np.ones(n - 1)))      # close pairs
    cases.append(("toeplitz", np.full(n, 0.5), np.full(n - 1, -1.0)))
    d = rng.standard_normal(n)
    e = rng.standard_normal(n - 1)
    e[::37] = 0.0                                                                      # split blocks
    cases.append(("split", d, e))
    cases.append(("graded", np.logspace(-8, 2, n), np.sqrt(np.logspace(-8, 2, n - 1)) * 1e-3))
    return cases


@pytest.mark.parametrize("name,d,e", _tridiag_cases(), ids=lambda x: x if isinstance(x, str) else "")
def test_dc_vs_oracle(gep, oracle_lib, name, d, e):
    M = d.shape[0]
    w_ql, _, st = oracle_lib.tql(d, e)
    w_ref = np.sort(w_ql)
    w_bi = oracle_lib.bisect(d, e)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    nT = max(1e-300, np.max(np.abs(w_ref)))
    w, Z, info = gep.tridiag_eig(dev(d), dev(e), want_vectors=True)
    assert info == 0
    wh, Zh = host(w), host(Z)
    assert np.all(np.diff(wh) >= 0)
    assert np.max(np.abs(wh - w_ref)) <= 64 * M * EPS * nT + 1e-300
    assert np.max(np.abs(wh - w_bi)) <= 64 * M * EPS * nT + 1e-300
    assert np.max(np.abs(Zh.T @ Zh - np.eye(M))) <= 64 * M * EPS
    assert np.max(np.abs(T @ Zh - Zh * wh[None, :])) <= 64 * M * EPS * nT
    w0, Z0, info0 = gep.tridiag_eig(dev(d), dev(e), want_vectors=False)
    assert Z0 is None and info0 == 0
    assert np.max(np.abs(host(w0) - w_bi)) <= 16 * EPS * nT * 4 + 1e-300


@pytest.mark.parametrize("variant", ["twosided", "explicit_inv"])
def test_backsub_vs_oracle(gep, oracle_lib, variant):
    M = 300
    g = gi.known_spectrum(M, seed=1)
    L_ref, _ = oracle_lib.cholesky(g["B"])
    Z = np.random.default_rng(2).standard_normal((M, 70))
    Y_ref = oracle_lib.backsub(L_ref, Z)
    L, _ = gep.cholesky(dev(g["B"]))
    if variant == "explicit_inv":
        _, LR = gep.reduce(dev(g["A"]), L, "explicit_inv")
    else:
        LR = L
    Y = host(gep.gep_backtransform(LR, dev(Z), variant))
    assert np.max(np.abs(Y - Y_ref)) <= 1e-12 * np.max(np.abs(Y_ref))


# -------------------------------------------------------------- whole workflow

def _check_solution(A, B, w, Y, w_ref):
    M = A.shape[0]
    nA = two_norm(A)
    assert np.max(np.abs(w - w_ref)) <= 1e-11 * nA
    res = np.linalg.norm(A @ Y - (B @ Y) * w[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Y.T @ B @ Y - np.eye(M)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth


@pytest.mark.parametrize("precision", ["fp64", "fp64_emulated"])
@pytest.mark.parametrize("reducer", ["twosided", "explicit_inv"])
@pytest.mark.parametrize("seed", [0, 1])
def test_solve_known_spectrum_M512(gep, oracle_lib, reducer, seed, precision):
    """Workload of the M=512 known-spectrum configuration: exact lambda and the oracle."""
    g = gi.known_spectrum(512, seed)
    A, B = g["A"], g["B"]
    w_ref, Y_ref, info = oracle_lib.gep_solve(A, B)
    assert info == 0
    w, Y, info = gep.solve(dev(A), dev(B), reducer=reducer, precision=precision)
    assert info == 0
    wh, Yh = host(w), host(Y)
    _check_solution(A, B, wh, Yh, w_ref)
    assert np.max(np.abs(wh - np.sort(g["lam"]))) <= 1e-11 * two_norm(A)
    # isolated eigenpairs compare elementwise (sign convention applied by both sides)
    gaps = np.minimum(np.diff(w_ref, prepend=-np.inf), np.diff(w_ref, append=np.inf))
    iso = gaps > 1e-6 * two_norm(A)
    assert np.max(np.abs(Yh[:, iso] - Y_ref[:, iso])) <= 1e-8


@pytest.mark.parametrize("precision", ["fp64", "fp64_emulated"])
@pytest.mark.parametrize("M", [4, 36, 260, 516, 1280])
def test_solve_tight_binding_vs_oracle(gep, oracle_lib, M, precision):
    tb = gi.tight_binding(M, seed=M)
    A, B = tb["A"], tb["B"]
    w_ref, Y_ref, info = oracle_lib.gep_solve(A, B)
    assert info == 0
    w, Y, info = gep.solve(dev(A), dev(B), precision=precision)
    assert info == 0
    _check_solution(A, B, host(w), host(Y), w_ref)
    w0, Y0, info0 = gep.solve(dev(A), dev(B), want_vectors=False, precision=precision)
    assert Y0 is None and info0 == 0
    assert np.max(np.abs(host(w0) - w_ref)) <= 1e-11 * two_norm(A)


def test_solve_not_positive_definite(gep):
    M = 200
    B = np.eye(M)
    B[150, 150] = -1.0
    A = gi.random_symmetric(M, 0)
    _, _, info = gep.solve(dev(A), dev(B))
    assert info == 151


def test_solve_nonfinite_input(gep):
    M = 64
    A = gi.random_symmetric(M, 1)
    A[10, 3] = np.nan
    A[3, 10] = np.nan
    _, _, info = gep.solve(dev(A), dev(np.eye(M)))
    assert info == -102


def test_solve_host_buffers_match_device(gep):
    tb = gi.tight_binding(256, seed=9)
    w_d, Y_d, _ = gep.solve(dev(tb["A"]), dev(tb["B"]))
    w_h, Y_h, info = gep.solve_host(tb["A"], tb["B"])
    assert info == 0
    assert np.array_equal(host(w_d), w_h)
    assert np.array_equal(host(Y_d), Y_h)


def test_solve_edge_sizes(gep, oracle_lib):
    for M in (1, 2, 3, 33, 127, 129):
        rng = np.random.default_rng(M)
        A = gi.random_symmetric(M, M)
        B = gi.spd_matrix(M, M, cond=5.0)
        w_ref, _, _ = oracle_lib.gep_solve(A, B)
        w, Y, info = gep.solve(dev(A), dev(B))
        assert info == 0
        _check_solution(A, B, host(w), host(Y), w_ref)
