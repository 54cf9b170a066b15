"""Seeded synthetic inputs for the generalized eigenproblem A y = lambda B y.

Shared by the GPU tests, the benchmark and the oracle tests.  This module holds
no step of the solver's method (no Cholesky, no reduction, no tridiagonal or
eigenvector arithmetic on A or B); it only draws matrices.

Two families, standing in for the ELSES matrices of the paper (section 2: carbon
materials in an sp-orbital tight-binding form with 4 orbitals per atom; the
matrices are sparse but solved densely):

* ``known_spectrum(M, seed)``: A = (L0 Q) diag(lam) (L0 Q)^T, B = L0 L0^T with
  L0 lower (diag U(1,2), off-diagonal N(0, 0.05^2)), Q orthogonal from the QR of
  an N(0,1) matrix (R's diagonal made positive), lam ~ U[-20, 20].  The exact
  eigenvalues are lam and the exact B-orthonormal eigenvectors are L0^-T Q.
* ``tight_binding(M, seed)``: M = 4 N orbitals (s, px, py, pz) on N atoms placed
  uniformly in a periodic cube at density 0.1 / A^3 (minimum-image distances,
  hard cutoff 8 A).  A: on-site diagonal N(0,1) eV, zero intra-atom
  off-diagonals, and for each atom pair within the cutoff the 16 orbital
  couplings -t exp(-r/1.5 A) g with independent g ~ N(0,1), t = 1 eV.  B: the
  identity plus alpha * 0.3 exp(-r/1.2 A) on every orbital pair of two distinct
  atoms within the cutoff; alpha = 1 unless that would put lambda_min(B) below
  0.1, in which case alpha = 0.9 / (-lambda_min(E)) rounded down to 4
  significant digits (E = B - I).  Because every 4x4 block of E is constant,
  E = K (x) J4 and lambda_min(E) = min(0, 4 lambda_min(K)) for the N x N atom
  kernel K; lambda_min(K) comes from a library eigensolver on K (scipy).

All matrices are returned as float64 numpy arrays; they are symmetric, so their
row-major buffer is also their column-major buffer.
"""
from __future__ import annotations

import math

import numpy as np

DENSITY = 0.1      # atoms per cubic angstrom
CUTOFF = 8.0       # angstrom
T_HOP = 1.0        # eV
R_HOP = 1.5        # angstrom, hopping decay length
S_OVL = 0.3        # overlap prefactor
R_OVL = 1.2        # angstrom, overlap decay length
LAMBDA_MIN_B = 0.1


def known_spectrum(M: int, seed: int):
    """Returns dict(A, B, lam, L0, Q); lam unsorted as drawn."""
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.normal(0.0, 0.05, size=(M, M)), -1)
    L0[np.diag_indices(M)] = rng.uniform(1.0, 2.0, size=M)
    G = rng.standard_normal((M, M))
    Q, R = np.linalg.qr(G)
    Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
    lam = rng.uniform(-20.0, 20.0, size=M)
    X = L0 @ Q
    A = (X * lam[None, :]) @ X.T
    A = 0.5 * (A + A.T)
    B = L0 @ L0.T
    B = 0.5 * (B + B.T)
    return dict(A=np.ascontiguousarray(A), B=np.ascontiguousarray(B), lam=lam, L0=L0, Q=Q)


def clustered_spectrum(M: int, seed: int, big: int = 0):
    """known_spectrum's construction with tight clusters planted in the spectrum: groups
    of 2..6 eigenvalues spaced 1e-9 apart and groups of exactly repeated eigenvalues
    (the case first-order eigenpair corrections cannot take).  big > 0 also plants one
    run of `big` consecutive eigenvalues spaced 1e-9 apart in the middle of the spectrum.
    Returns dict(A, B, lam)."""
    rng = np.random.default_rng(seed)
    L0 = np.tril(rng.normal(0.0, 0.05, size=(M, M)), -1)
    L0[np.diag_indices(M)] = rng.uniform(1.0, 2.0, size=M)
    G = rng.standard_normal((M, M))
    Q, R = np.linalg.qr(G)
    Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
    lam = rng.uniform(-20.0, 20.0, size=M)
    i = 0
    while i + 6 < M:
        k = int(rng.integers(2, 7))
        if rng.random() < 0.5:
            lam[i:i + k] = lam[i] + 1e-9 * np.arange(k)
        else:
            lam[i:i + k] = lam[i]
        i += k + int(rng.integers(5, 40))
    if big > 0:
        s0 = (M - big) // 2
        lam[s0:s0 + big] = 1.5 + 1e-9 * np.arange(big)
    X = L0 @ Q
    A = (X * lam[None, :]) @ X.T
    A = 0.5 * (A + A.T)
    B = L0 @ L0.T
    B = 0.5 * (B + B.T)
    return dict(A=np.ascontiguousarray(A), B=np.ascontiguousarray(B), lam=lam)


def _box(n_atoms: int) -> float:
    return (n_atoms / DENSITY) ** (1.0 / 3.0)


def _pairs(pos: np.ndarray, L: float):
    """All atom pairs a < b within the cutoff (minimum image); sorted (a, b)."""
    N = pos.shape[0]
    ia, ib, rr = [], [], []
    chunk = 256
    for a0 in range(0, N, chunk):
        a1 = min(N, a0 + chunk)
        dx = pos[a0:a1, None, :] - pos[None, :, :]
        dx -= L * np.round(dx / L)
        r = np.sqrt(np.einsum("abk,abk->ab", dx, dx))
        a_idx = np.arange(a0, a1)[:, None]
        b_idx = np.arange(N)[None, :]
        mask = (b_idx > a_idx) & (r <= CUTOFF)
        aa, bb = np.nonzero(mask)
        ia.append(aa + a0)
        ib.append(bb)
        rr.append(r[aa, bb])
    ia = np.concatenate(ia) if ia else np.zeros(0, np.int64)
    ib = np.concatenate(ib) if ib else np.zeros(0, np.int64)
    rr = np.concatenate(rr) if rr else np.zeros(0)
    order = np.lexsort((ib, ia))
    return ia[order], ib[order], rr[order]


def _lambda_min_sym(K):
    """Smallest eigenvalue of the symmetric atom kernel K (library routine)."""
    N = K.shape[0]
    if N == 0:
        return 0.0
    if N <= 4096:
        return float(np.linalg.eigvalsh(K.toarray() if hasattr(K, "toarray") else K)[0])
    from scipy.sparse.linalg import eigsh
    v0 = np.ones(N) / math.sqrt(N)
    val = eigsh(K, k=1, which="SA", v0=v0, tol=1e-10, maxiter=20000, return_eigenvectors=False)
    return float(val[0])


def tight_binding(M: int, seed: int, dtype=np.float64):
    """Returns dict(A, B, n_atoms, box, alpha, n_pairs, lam_min_K)."""
    if M % 4 != 0 or M <= 0:
        raise ValueError("tight-binding order M must be a positive multiple of 4")
    from scipy import sparse

    N = M // 4
    L = _box(N)
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, L, size=(N, 3))
    onsite = rng.standard_normal(M)
    ia, ib, r = _pairs(pos, L)
    g = rng.standard_normal((ia.shape[0], 4, 4))

    A = np.zeros((M, M), dtype=dtype)
    A[np.diag_indices(M)] = onsite
    hop = (-T_HOP * np.exp(-r / R_HOP))[:, None, None] * g          # (P, 4, 4)
    oi = np.arange(4)
    rows = (4 * ia)[:, None, None] + oi[None, :, None]              # (P, 4, 1)
    cols = (4 * ib)[:, None, None] + oi[None, None, :]              # (P, 1, 4)
    rows_b = np.broadcast_to(rows, hop.shape)
    cols_b = np.broadcast_to(cols, hop.shape)
    A[rows_b, cols_b] = hop
    A[cols_b, rows_b] = hop

    kval = S_OVL * np.exp(-r / R_OVL)
    K = sparse.coo_matrix((np.concatenate([kval, kval]),
                           (np.concatenate([ia, ib]), np.concatenate([ib, ia]))), shape=(N, N)).tocsr()
    lam_min_K = _lambda_min_sym(K)
    lam_min_E = min(0.0, 4.0 * lam_min_K)
    alpha = 1.0
    if 1.0 + lam_min_E < LAMBDA_MIN_B:
        raw = (1.0 - LAMBDA_MIN_B) / (-lam_min_E)
        digits = 4 - int(math.floor(math.log10(raw))) - 1
        alpha = math.floor(raw * 10 ** digits) / 10 ** digits
    B = np.zeros((M, M), dtype=dtype)
    B[np.diag_indices(M)] = 1.0
    ov = np.broadcast_to((alpha * kval)[:, None, None], hop.shape)
    B[rows_b, cols_b] = ov
    B[cols_b, rows_b] = ov
    return dict(A=A, B=B, n_atoms=N, box=L, alpha=alpha, n_pairs=int(ia.shape[0]), lam_min_K=lam_min_K)


def batch_orders(count: int = 512, seed: int = 1000, lo: int = 64, hi: int = 2048):
    """Orders M_i for a batch: log-uniform in [lo, hi], multiples of 4 (N_i = round(M_i/4))."""
    rng = np.random.default_rng(seed)
    m = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    n = np.clip(np.rint(m / 4.0).astype(np.int64), lo // 4, hi // 4)
    return (4 * n).tolist()


def random_symmetric(M: int, seed: int):
    """W = (G + G^T)/sqrt(2), G ~ N(0,1): the weight matrix of the density-matrix loss."""
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((M, M))
    return (G + G.T) / math.sqrt(2.0)


def spd_matrix(M: int, seed: int, cond: float = 10.0):
    """A random symmetric positive definite matrix with eigenvalues in [1, cond]."""
    rng = np.random.default_rng(seed)
    Q, R = np.linalg.qr(rng.standard_normal((M, M)))
    Q = Q * np.where(np.diag(R) < 0, -1.0, 1.0)[None, :]
    ev = np.exp(rng.uniform(0.0, math.log(cond), size=M))
    S = (Q * ev[None, :]) @ Q.T
    return 0.5 * (S + S.T)
