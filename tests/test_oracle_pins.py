"""Pins for the FP64 CPU oracle, checked against what the mathematics fixes.

None of these compares the oracle with itself: every expected value is a
closed form, an exact spectrum built into the input, a library routine on a
case that reduces to it (numpy / scipy), an independent algorithm in the
oracle that shares no step with the pipeline (Jacobi, Bunch-Parlett inertia),
or an invariant of the paper's formulation (Eq. 2-6).
"""
import json
import math
import os

import numpy as np
import pytest

import gep_inputs as gi

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EPS = 2.0 ** -52


def _two_norm(A):
    return float(np.max(np.abs(np.linalg.eigvalsh(A))))


# ------------------------------------------------------------ Eq. 4 Cholesky

@pytest.mark.parametrize("M", [1, 7, 64, 129])
def test_cholesky_recovers_L0(oracle_lib, M):
    """B = L0 L0^T with positive diagonal: the Cholesky factor is unique, so L = L0."""
    g = gi.known_spectrum(M, seed=3)
    L, info = oracle_lib.cholesky(g["B"])
    assert info == 0
    assert np.allclose(np.triu(L, 1), 0.0)
    assert np.max(np.abs(L - g["L0"])) <= 1e-12
    assert np.max(np.abs(L @ L.T - g["B"])) <= 50 * M * EPS * np.max(np.abs(g["B"]))


@pytest.mark.parametrize("k", [1, 5, 20])
def test_cholesky_reports_first_bad_minor(oracle_lib, k):
    """Leading minor of order k not positive definite -> info = k (LAPACK convention)."""
    M = 24
    B = gi.spd_matrix(M, seed=k)
    L = np.linalg.cholesky(B)
    D = np.ones(M)
    D[k - 1] = -1.0
    Bk = (L * D[None, :]) @ L.T   # leading minors 1..k-1 stay SPD, order k is not
    _, info = oracle_lib.cholesky(0.5 * (Bk + Bk.T))
    assert info == k


# ---------------------------------------------------------- Eq. 5 reduction

@pytest.mark.parametrize("M", [5, 64, 130])
def test_two_sided_equals_known_Q_Lambda_QT(oracle_lib, M):
    """With L = L0: L^-1 A L^-T = Q diag(lam) Q^T exactly (up to rounding)."""
    g = gi.known_spectrum(M, seed=11)
    L, info = oracle_lib.cholesky(g["B"])
    C = oracle_lib.two_sided(g["A"], L)
    expect = (g["Q"] * g["lam"][None, :]) @ g["Q"].T
    assert np.max(np.abs(C - C.T)) == 0.0
    assert np.max(np.abs(C - expect)) <= 1e-11 * np.max(np.abs(g["lam"]))
    assert abs(np.trace(C) - g["lam"].sum()) <= 1e-10 * M


def test_two_sided_reconstructs_A(oracle_lib):
    """L C L^T = A on a tight-binding pencil (Eq. 5 inverted)."""
    tb = gi.tight_binding(128, seed=2)
    L, info = oracle_lib.cholesky(tb["B"])
    assert info == 0
    C = oracle_lib.two_sided(tb["A"], L)
    assert np.max(np.abs(L @ C @ L.T - tb["A"])) <= 1e-12 * np.max(np.abs(tb["A"])) * 128


# --------------------------------------------- Householder tridiagonalisation

@pytest.mark.parametrize("M", [1, 2, 3, 33, 100])
def test_tridiag_similarity(oracle_lib, M):
    """C = Q T Q^T, Q orthogonal; trace and Frobenius norm preserved."""
    rng = np.random.default_rng(M)
    G = rng.standard_normal((M, M))
    C = 0.5 * (G + G.T)
    d, e, Q = oracle_lib.tridiag(C)
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.max(np.abs(Q.T @ Q - np.eye(M))) <= 50 * M * EPS
    assert np.max(np.abs(Q @ T @ Q.T - C)) <= 50 * M * EPS * max(1.0, np.max(np.abs(C)))
    assert abs(d.sum() - np.trace(C)) <= 1e-12 * M
    assert abs((d ** 2).sum() + 2 * (e ** 2).sum() - (C ** 2).sum()) <= 1e-11 * (C ** 2).sum()


def test_tridiag_spectrum_matches_library(oracle_lib):
    """eig(T) from the oracle's bisection equals numpy's eigvalsh(C) (library routine)."""
    rng = np.random.default_rng(5)
    G = rng.standard_normal((90, 90))
    C = G + G.T
    d, e, _ = oracle_lib.tridiag(C, want_q=False)
    w = oracle_lib.bisect(d, e)
    ref = np.linalg.eigvalsh(C)
    assert np.max(np.abs(w - ref)) <= 1e-12 * _two_norm(C) * 10


# --------------------------------------------------- tridiagonal eigensolvers

def test_tql_against_bisection_and_closed_form(oracle_lib):
    """Toeplitz tridiagonal (a, b): eigenvalues a + 2b cos(pi k/(n+1)) (closed form)."""
    n, a, b = 50, 0.3, -1.7
    d = np.full(n, a)
    e = np.full(n - 1, b)
    k = np.arange(1, n + 1)
    exact = np.sort(a + 2 * b * np.cos(np.pi * k / (n + 1)))
    w_ql, Z, st = oracle_lib.tql(d, e, np.eye(n))
    assert st == 0
    order = np.argsort(w_ql)
    assert np.max(np.abs(w_ql[order] - exact)) <= 1e-13 * 4
    w_bi = oracle_lib.bisect(d, e)
    assert np.max(np.abs(w_bi - exact)) <= 1e-13 * 4
    T = np.diag(d) + np.diag(e, 1) + np.diag(e, -1)
    assert np.max(np.abs(T @ Z - Z * w_ql[None, :])) <= 1e-13 * 10
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) <= 1e-13 * 10


def test_tql_diagonal_and_split(oracle_lib):
    """e = 0 -> eigenvalues are d; a zero in e splits T into independent blocks."""
    d = np.array([3.0, -1.0, 2.0, 7.0])
    w, Z, st = oracle_lib.tql(d, np.zeros(3), np.eye(4))
    assert st == 0 and np.array_equal(np.sort(w), np.sort(d))
    d2 = np.array([1.0, 2.0, 5.0, 6.0])
    e2 = np.array([1.0, 0.0, 1.0])
    w2, _, _ = oracle_lib.tql(d2, e2)
    s5 = math.sqrt(5.0)
    # 2x2 blocks [[1,1],[1,2]] and [[5,1],[1,6]]: (3 -+ sqrt5)/2, (11 -+ sqrt5)/2
    exact = np.sort([(3 - s5) / 2, (3 + s5) / 2, (11 - s5) / 2, (11 + s5) / 2])
    assert np.max(np.abs(np.sort(w2) - exact)) <= 1e-14 * 8


def test_sturm_count_matches_known(oracle_lib):
    g = gi.known_spectrum(60, seed=8)
    L, _ = oracle_lib.cholesky(g["B"])
    C = oracle_lib.two_sided(g["A"], L)
    d, e, _ = oracle_lib.tridiag(C, want_q=False)
    for sigma in (-15.0, -3.3, 0.0, 4.4, 19.0):
        assert oracle_lib.sturm_count(d, e, sigma) == int(np.sum(g["lam"] < sigma))


def test_jacobi_matches_library(oracle_lib):
    """The Jacobi pin itself is pinned: a random symmetric matrix vs numpy eigh."""
    rng = np.random.default_rng(1)
    G = rng.standard_normal((20, 20))
    S = G + G.T
    w, V, sweeps = oracle_lib.jacobi(S)
    assert sweeps > 0
    assert np.max(np.abs(w - np.linalg.eigvalsh(S))) <= 1e-13 * 20
    assert np.max(np.abs(S @ V - V * w[None, :])) <= 1e-12


# ------------------------------------------------------------ Eq. 6 backsub

def test_backsub_solves_LT(oracle_lib):
    g = gi.known_spectrum(40, seed=4)
    Z = np.random.default_rng(0).standard_normal((40, 7))
    Y = oracle_lib.backsub(g["L0"], Z)
    assert np.max(np.abs(g["L0"].T @ Y - Z)) <= 1e-13 * 10


# ----------------------------------------------------------- Eq. 2 full GEP

def _check_gep(A, B, w, Y, tol_lam=None, lam_ref=None):
    M = A.shape[0]
    nA = _two_norm(A)
    res = np.linalg.norm(A @ Y - (B @ Y) * w[None, :]) / (np.linalg.norm(A) * M)
    orth = np.max(np.abs(Y.T @ B @ Y - np.eye(M)))
    assert res <= 1e-13, res
    assert orth <= 1e-12, orth
    if lam_ref is not None:
        assert np.max(np.abs(w - lam_ref)) <= (tol_lam or 1e-11) * nA
    assert np.all(np.diff(w) >= 0)


@pytest.mark.parametrize("M,seed", [(1, 0), (2, 1), (17, 2), (64, 3), (200, 4)])
def test_gep_known_spectrum(oracle_lib, M, seed):
    """Known-spectrum recipe: exact lambda known; eigenvectors are L0^-T Q up to sign."""
    g = gi.known_spectrum(M, seed)
    w, Y, info = oracle_lib.gep_solve(g["A"], g["B"])
    assert info == 0
    lam = np.sort(g["lam"])
    _check_gep(g["A"], g["B"], w, Y, lam_ref=lam)
    Yx = np.linalg.solve(g["L0"].T, g["Q"])[:, np.argsort(g["lam"])]
    # sign convention: largest-magnitude entry positive
    idx = np.argmax(np.abs(Yx), axis=0)
    Yx = Yx * np.sign(Yx[idx, np.arange(M)])[None, :]
    gaps = np.diff(lam)
    if M > 1 and np.min(gaps) > 1e-3:
        assert np.max(np.abs(Y - Yx)) <= 1e-9


def test_gep_closed_forms(oracle_lib):
    with open(os.path.join(GOLDEN, "gep_closed_forms.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        A = np.array(c["A"])
        B = np.array(c["B"])
        w, Y, info = oracle_lib.gep_solve(A, B)
        assert info == 0
        assert np.max(np.abs(w - np.array(c["lambda"]))) <= 1e-14 * 8, c["name"]
        w2, _, _ = oracle_lib.gep_solve(A, B, want_vectors=False)
        assert np.max(np.abs(w2 - np.array(c["lambda"]))) <= 1e-14 * 8, c["name"]


def test_gep_identity_B_is_standard_problem(oracle_lib):
    """B = I reduces the GEP to the SEP: compare with numpy eigh (library)."""
    rng = np.random.default_rng(9)
    G = rng.standard_normal((75, 75))
    A = G + G.T
    w, Y, info = oracle_lib.gep_solve(A, np.eye(75))
    assert info == 0
    assert np.max(np.abs(w - np.linalg.eigvalsh(A))) <= 1e-13 * _two_norm(A)
    _check_gep(A, np.eye(75), w, Y)


def test_gep_diagonal_pencil(oracle_lib):
    rng = np.random.default_rng(10)
    a = rng.standard_normal(30)
    b = rng.uniform(0.5, 3.0, 30)
    w, Y, info = oracle_lib.gep_solve(np.diag(a), np.diag(b))
    assert info == 0
    assert np.max(np.abs(w - np.sort(a / b))) <= 4 * EPS * np.max(np.abs(a / b))


def test_gep_vs_library_and_jacobi_tight_binding(oracle_lib):
    """Tight-binding pencil (M=32, 8 atoms): oracle vs scipy.linalg.eigh(A, B) and vs
    Jacobi on L^-1 A L^-T built with numpy's Cholesky/solve (no oracle stage used)."""
    import scipy.linalg as sla
    tb = gi.tight_binding(32, seed=5)
    A, B = tb["A"], tb["B"]
    w, Y, info = oracle_lib.gep_solve(A, B)
    assert info == 0
    ref = sla.eigh(A, B, eigvals_only=True)
    nA = _two_norm(A)
    assert np.max(np.abs(w - ref)) <= 1e-12 * nA
    Ln = np.linalg.cholesky(B)
    C = np.linalg.solve(Ln, np.linalg.solve(Ln, A).T)
    wj, _, _ = oracle_lib.jacobi(0.5 * (C + C.T), want_v=False)
    assert np.max(np.abs(w - wj)) <= 1e-12 * nA
    _check_gep(A, B, w, Y)


@pytest.mark.parametrize("M", [64, 256])
def test_gep_inertia_counts(oracle_lib, M):
    """Sylvester: #(lambda < sigma) = #negative eigenvalues of A - sigma B (Bunch-Parlett)."""
    tb = gi.tight_binding(M, seed=M)
    w, _, info = oracle_lib.gep_solve(tb["A"], tb["B"], want_vectors=False)
    assert info == 0
    rng = np.random.default_rng(0)
    for sigma in rng.uniform(w[0] - 0.5, w[-1] + 0.5, size=8):
        if np.min(np.abs(w - sigma)) < 1e-8:
            continue
        neg, zero, pos = oracle_lib.inertia(tb["A"], tb["B"], sigma)
        assert neg == int(np.sum(w < sigma)) and zero == 0 and neg + pos == M


def test_gep_trace_invariant(oracle_lib):
    """sum lambda = trace(B^-1 A) (library solve)."""
    tb = gi.tight_binding(160, seed=1)
    w, _, _ = oracle_lib.gep_solve(tb["A"], tb["B"], want_vectors=False)
    tr = np.trace(np.linalg.solve(tb["B"], tb["A"]))
    assert abs(w.sum() - tr) <= 1e-11 * 160 * _two_norm(tb["A"])


def test_gep_eigenvalue_only_matches_full(oracle_lib):
    """T_evo route (bisection, no vectors) gives the same eigenvalues as the full route."""
    tb = gi.tight_binding(128, seed=6)
    w1, _, _ = oracle_lib.gep_solve(tb["A"], tb["B"], want_vectors=True)
    w0, Y0, _ = oracle_lib.gep_solve(tb["A"], tb["B"], want_vectors=False)
    assert Y0 is None
    assert np.max(np.abs(w1 - w0)) <= 1e-12 * _two_norm(tb["A"])


def test_gep_not_positive_definite(oracle_lib):
    M = 12
    B = np.eye(M)
    B[4, 4] = -0.5
    w, Y, info = oracle_lib.gep_solve(np.eye(M), B)
    assert info == 5


# ----------------------------------------------------------------- adjoint

def test_adjoint_eigenvalue_sum_closed_form(oracle_lib):
    """W = 0, lbar = 1: Abar = Y_o Y_o^T and Bbar = -Y_o Lambda_o Y_o^T."""
    tb = gi.tight_binding(48, seed=7)
    w, Y, _ = oracle_lib.gep_solve(tb["A"], tb["B"])
    n = 24
    Ab, Bb = oracle_lib.adjoint(w, Y, n, np.ones(n), None)
    Yo = Y[:, :n]
    assert np.max(np.abs(Ab - Yo @ Yo.T)) <= 1e-13
    assert np.max(np.abs(Bb + (Yo * w[None, :n]) @ Yo.T)) <= 1e-12 * max(1.0, np.max(np.abs(w)))


def test_adjoint_central_differences(oracle_lib):
    """Full loss sum lambda_o + <W, P>: adjoint vs central differences of a library
    forward solve (scipy.linalg.eigh on the pencil), h = 1e-6."""
    import scipy.linalg as sla
    M, n = 40, 20
    tb = gi.tight_binding(M, seed=12)
    A, B = tb["A"], tb["B"]
    W = gi.random_symmetric(M, seed=1)

    def loss(A_, B_):
        ww, YY = sla.eigh(A_, B_)
        Yo = YY[:, :n]
        return ww[:n].sum() + np.sum(W * (Yo @ Yo.T))

    w, Y, _ = oracle_lib.gep_solve(A, B)
    assert w[n] - w[n - 1] > 1e-3
    Ab, Bb = oracle_lib.adjoint(w, Y, n, np.ones(n), W)
    rng = np.random.default_rng(2)
    h = 1e-6
    for _ in range(6):
        dA = rng.standard_normal((M, M)); dA = dA + dA.T
        dB = rng.standard_normal((M, M)); dB = dB + dB.T
        dA *= 1e-3 * np.linalg.norm(A) / np.linalg.norm(dA)
        dB *= 0.05 / np.linalg.norm(dB)
        fd = (loss(A + h * dA, B + h * dB) - loss(A - h * dA, B - h * dB)) / (2 * h)
        an = np.sum(Ab * dA) + np.sum(Bb * dB)
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(fd)), (fd, an)


# ------------------------------------------- Eq. 7-9 Cholesky-free reducer

@pytest.mark.parametrize("M,seed", [(1, 0), (2, 1), (17, 2), (64, 3), (150, 4)])
def test_eigenexa_known_spectrum(oracle_lib, M, seed):
    """SEP of B, A' = D^-1/2 W^T A W D^-1/2, Y = W D^-1/2 Z: the planted spectrum and
    B-orthonormal eigenvectors L0^-T Q (up to sign) come out, as with Eq. 4-6."""
    g = gi.known_spectrum(M, seed)
    w, Y, info = oracle_lib.gep_solve_eigenexa(g["A"], g["B"])
    assert info == 0
    lam = np.sort(g["lam"])
    _check_gep(g["A"], g["B"], w, Y, lam_ref=lam)
    Yx = np.linalg.solve(g["L0"].T, g["Q"])[:, np.argsort(g["lam"])]
    idx = np.argmax(np.abs(Yx), axis=0)
    Yx = Yx * np.sign(Yx[idx, np.arange(M)])[None, :]
    if M > 1 and np.min(np.diff(lam)) > 1e-3:
        assert np.max(np.abs(Y - Yx)) <= 1e-9


def test_eigenexa_closed_forms_and_special_cases(oracle_lib):
    with open(os.path.join(GOLDEN, "gep_closed_forms.json")) as f:
        cases = json.load(f)["cases"]
    for c in cases:
        w, _, info = oracle_lib.gep_solve_eigenexa(np.array(c["A"]), np.array(c["B"]))
        assert info == 0
        assert np.max(np.abs(w - np.array(c["lambda"]))) <= 1e-14 * 8, c["name"]
    # B = I: the standard problem (library eigensolver)
    rng = np.random.default_rng(21)
    G = rng.standard_normal((60, 60))
    A = G + G.T
    w, Y, info = oracle_lib.gep_solve_eigenexa(A, np.eye(60))
    assert info == 0
    assert np.max(np.abs(w - np.linalg.eigvalsh(A))) <= 1e-13 * _two_norm(A)
    _check_gep(A, np.eye(60), w, Y)
    # diagonal pencil: lambda_i = A_ii / B_ii
    a = rng.standard_normal(25)
    b = rng.uniform(0.5, 3.0, 25)
    w, _, info = oracle_lib.gep_solve_eigenexa(np.diag(a), np.diag(b))
    assert info == 0
    assert np.max(np.abs(w - np.sort(a / b))) <= 8 * EPS * np.max(np.abs(a / b))


def test_eigenexa_matches_cholesky_route_tight_binding(oracle_lib):
    """The paper's reducers all solve the same GEP (Table 1): the Cholesky-free route agrees
    with the Cholesky route (Eq. 4-6) and with scipy's generalized eigensolver."""
    import scipy.linalg
    tb = gi.tight_binding(128, seed=5)
    A, B = tb["A"], tb["B"]
    w1, Y1, i1 = oracle_lib.gep_solve(A, B)
    w2, Y2, i2 = oracle_lib.gep_solve_eigenexa(A, B)
    assert i1 == i2 == 0
    nA = _two_norm(A)
    assert np.max(np.abs(w1 - w2)) <= 1e-12 * nA
    assert np.max(np.abs(w2 - scipy.linalg.eigh(A, B, eigvals_only=True))) <= 1e-12 * nA
    _check_gep(A, B, w2, Y2)
    iso = np.ones(128, dtype=bool)
    gaps = np.diff(w1)
    iso[1:] &= gaps > 1e-6 * nA
    iso[:-1] &= gaps > 1e-6 * nA
    assert np.max(np.abs(Y1[:, iso] - Y2[:, iso])) <= 1e-8
    w3, _, i3 = oracle_lib.gep_solve_eigenexa(A, B, want_vectors=False)
    assert i3 == 0 and np.max(np.abs(w3 - w2)) <= 1e-12 * nA


def test_eigenexa_reports_indefinite_B(oracle_lib):
    """B with two negative eigenvalues: no Cholesky here, the count of non-positive
    eigenvalues of B is reported instead."""
    rng = np.random.default_rng(22)
    Q, _ = np.linalg.qr(rng.standard_normal((12, 12)))
    dB = np.array([1.0, -0.5, 2.0, 3.0, -4.0, 1.5, 2.5, 0.7, 1.1, 1.9, 2.2, 3.3])
    B = (Q * dB[None, :]) @ Q.T
    B = 0.5 * (B + B.T)
    _, _, info = oracle_lib.gep_solve_eigenexa(np.eye(12), B)
    assert info == 2


# --------------------------------- lowest eigenpairs: bisection + inverse iteration

@pytest.mark.parametrize("M,n", [(1, 1), (40, 13), (129, 64), (200, 200)])
def test_partial_spectrum_matches_full_solve(oracle_lib, M, n):
    """Inverse iteration on T shares no step with QL: its lowest n eigenpairs agree with the
    full solve's first n (eigenvectors column by column where isolated)."""
    tb = gi.tight_binding(M, seed=M) if M % 4 == 0 else gi.known_spectrum(M, seed=M)
    A, B = tb["A"], tb["B"]
    w, Y, info = oracle_lib.gep_solve(A, B)
    wp, Yp, ip = oracle_lib.gep_solve_partial(A, B, n)
    assert info == ip == 0 and wp.shape == (n,) and Yp.shape == (M, n)
    nA = _two_norm(A)
    assert np.max(np.abs(wp - w[:n])) <= 1e-12 * nA
    res = np.linalg.norm(A @ Yp - (B @ Yp) * wp[None, :]) / (np.linalg.norm(A) * M)
    assert res <= 1e-13, res
    assert np.max(np.abs(Yp.T @ B @ Yp - np.eye(n))) <= 1e-12
    gaps = np.diff(w)
    iso = np.ones(M, dtype=bool)
    iso[1:] &= gaps > 1e-6 * nA
    iso[:-1] &= gaps > 1e-6 * nA
    iso = iso[:n]
    assert np.max(np.abs(Yp[:, iso] - Y[:, :n][:, iso]), initial=0.0) <= 1e-8


def test_partial_spectrum_known_and_clustered(oracle_lib):
    g = gi.known_spectrum(90, seed=6)
    w, Y, info = oracle_lib.gep_solve_partial(g["A"], g["B"], 30)
    assert info == 0
    assert np.max(np.abs(w - np.sort(g["lam"])[:30])) <= 1e-11 * 20
    # exactly repeated and 1e-9-spaced eigenvalues: the cluster's vectors stay B-orthonormal
    c = gi.clustered_spectrum(120, seed=7)
    w, Y, info = oracle_lib.gep_solve_partial(c["A"], c["B"], 60)
    assert info == 0
    assert np.max(np.abs(w - np.sort(c["lam"])[:60])) <= 1e-11 * 20
    assert np.max(np.abs(Y.T @ c["B"] @ Y - np.eye(60))) <= 1e-12
    res = np.linalg.norm(c["A"] @ Y - (c["B"] @ Y) * w[None, :]) / (np.linalg.norm(c["A"]) * 120)
    assert res <= 1e-13, res


def test_partial_spectrum_standard_problem_and_edges(oracle_lib):
    rng = np.random.default_rng(31)
    G = rng.standard_normal((70, 70))
    A = G + G.T
    w, Y, info = oracle_lib.gep_solve_partial(A, np.eye(70), 20)
    assert info == 0
    assert np.max(np.abs(w - np.linalg.eigvalsh(A)[:20])) <= 1e-13 * _two_norm(A)
    w0, Y0, i0 = oracle_lib.gep_solve_partial(A, np.eye(70), 0)
    assert i0 == 0 and w0.shape == (0,) and Y0.shape == (70, 0)
    # B not positive definite: the Cholesky failure index, as in the full solve
    Bbad = np.eye(70)
    Bbad[5, 5] = -1.0
    _, _, ib = oracle_lib.gep_solve_partial(A, Bbad, 10)
    assert ib == 6
