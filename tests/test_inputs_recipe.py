"""The seeded input recipe (stand-ins for the paper's ELSES matrices, section 2) checked
against its written definition: structure, value distributions and the exactness claims the
parity tests rely on.  CPU only; library eigensolvers serve as independent checks."""
import math

import numpy as np
import pytest
import scipy.linalg

import gep_inputs as gi


def test_known_spectrum_is_exact_and_deterministic():
    g = gi.known_spectrum(96, seed=3)
    A, B, lam = g["A"], g["B"], g["lam"]
    assert np.array_equal(A, A.T) and np.array_equal(B, B.T)
    # L0 lower with diagonal in [1, 2]; Q orthogonal
    L0, Q = g["L0"], g["Q"]
    assert np.array_equal(L0, np.tril(L0))
    assert np.all((np.diag(L0) >= 1.0) & (np.diag(L0) <= 2.0))
    assert np.max(np.abs(Q.T @ Q - np.eye(96))) < 1e-13
    assert np.all((lam >= -20.0) & (lam <= 20.0))
    # the pencil's eigenvalues are lam (library generalized eigensolver, independent of ours)
    w = scipy.linalg.eigh(A, B, eigvals_only=True)
    assert np.max(np.abs(w - np.sort(lam))) < 1e-11 * 20
    # eigenvectors L0^-T Q: A Y = B Y diag(lam), Y^T B Y = I
    Y = scipy.linalg.solve_triangular(L0.T, Q, lower=False)
    assert np.max(np.abs(A @ Y - (B @ Y) * lam[None, :])) < 1e-11
    assert np.max(np.abs(Y.T @ B @ Y - np.eye(96))) < 1e-12
    g2 = gi.known_spectrum(96, seed=3)
    assert np.array_equal(g2["A"], A) and np.array_equal(g2["B"], B)
    assert not np.array_equal(gi.known_spectrum(96, seed=4)["A"], A)


def test_clustered_spectrum_plants_clusters():
    g = gi.clustered_spectrum(200, seed=2)
    lam = np.sort(g["lam"])
    gaps = np.diff(lam)
    assert np.sum(gaps == 0.0) >= 5                       # exactly repeated eigenvalues
    assert np.sum((gaps > 0) & (gaps < 1e-8)) >= 5         # 1e-9 spaced groups
    w = scipy.linalg.eigh(g["A"], g["B"], eigvals_only=True)
    assert np.max(np.abs(w - lam)) < 1e-10 * 20


@pytest.mark.parametrize("M", [64, 400, 1024])
def test_tight_binding_structure(M):
    tb = gi.tight_binding(M, seed=M)
    A, B, N = tb["A"], tb["B"], tb["n_atoms"]
    assert N == M // 4 and A.shape == (M, M) and B.shape == (M, M)
    assert np.array_equal(A, A.T) and np.array_equal(B, B.T)
    assert tb["box"] == pytest.approx((N / 0.1) ** (1.0 / 3.0))
    # on-atom blocks: A diagonal only (on-site energies), B the identity
    for a in range(N):
        blk = slice(4 * a, 4 * a + 4)
        assert np.array_equal(A[blk, blk], np.diag(np.diag(A[blk, blk])))
        assert np.array_equal(B[blk, blk], np.eye(4))
    # couplings only between atom pairs within the cutoff; overlap blocks constant
    Ab = A.reshape(N, 4, N, 4).transpose(0, 2, 1, 3)
    Bb = B.reshape(N, 4, N, 4).transpose(0, 2, 1, 3)
    coupled = np.any(Ab != 0.0, axis=(2, 3)) & ~np.eye(N, dtype=bool)
    overl = np.any(Bb != 0.0, axis=(2, 3)) & ~np.eye(N, dtype=bool)
    assert np.array_equal(coupled, overl)
    assert coupled.sum() == 2 * tb["n_pairs"]
    ia, ib = np.nonzero(np.triu(overl, 1))
    blocks = Bb[ia, ib]
    assert np.all(blocks == blocks[:, :1, :1])
    # the overlap value fixes the distance: alpha 0.3 exp(-r / 1.2) with r <= 8
    r = -1.2 * np.log(blocks[:, 0, 0] / (0.3 * tb["alpha"]))
    assert np.all(r <= 8.0 + 1e-9) and np.all(r > 0.0)
    # hopping magnitudes bounded by t exp(-r / 1.5) |g| with g ~ N(0, 1): scaled couplings
    # are standard normal
    g = Ab[ia, ib] / (-1.0 * np.exp(-r / 1.5))[:, None, None]
    if g.size > 2000:
        assert abs(g.mean()) < 0.1 and abs(g.std() - 1.0) < 0.1
    # lambda_min(B) >= 0.1 after the alpha rescaling (library eigensolver)
    assert np.linalg.eigvalsh(B)[0] >= 0.1 - 1e-12
    if tb["alpha"] < 1.0:
        assert float(f"{tb['alpha']:.4g}") == tb["alpha"]


def test_tight_binding_neighbour_density():
    """At density 0.1 / A^3 and an 8 A cutoff an atom has (4/3) pi 8^3 0.1 = 214.5 neighbours
    on average (periodic box, minimum image; the box is wider than 16 A here)."""
    tb = gi.tight_binding(2048, seed=0)
    N = tb["n_atoms"]
    assert tb["box"] > 16.0
    mean_nb = 2 * tb["n_pairs"] / N
    expect = 4.0 / 3.0 * math.pi * 8.0 ** 3 * 0.1 * (N - 1) / N
    assert abs(mean_nb - expect) < 0.05 * expect


def test_tight_binding_rejects_bad_orders():
    for M in (0, 6, -4):
        with pytest.raises(ValueError):
            gi.tight_binding(M, seed=0)


def test_batch_orders_recipe():
    orders = gi.batch_orders(512, seed=1000)
    assert len(orders) == 512
    assert all(o % 4 == 0 and 64 <= o <= 2048 for o in orders)
    logs = np.log(np.asarray(orders, dtype=float))
    # log-uniform on [log 64, log 2048]: mean and spread of a uniform law
    lo, hi = math.log(64), math.log(2048)
    assert abs(logs.mean() - 0.5 * (lo + hi)) < 0.1
    assert abs(logs.std() - (hi - lo) / math.sqrt(12.0)) < 0.1
    assert gi.batch_orders(512, seed=1000) == orders


def test_random_symmetric_and_spd():
    W = gi.random_symmetric(300, seed=1)
    assert np.array_equal(W, W.T)
    off = W[np.triu_indices(300, 1)]
    assert abs(off.mean()) < 0.02 and abs(off.std() - 1.0) < 0.02
    S = gi.spd_matrix(200, seed=2, cond=10.0)
    ev = np.linalg.eigvalsh(S)
    assert ev[0] >= 1.0 - 1e-12 and ev[-1] <= 10.0 + 1e-11
