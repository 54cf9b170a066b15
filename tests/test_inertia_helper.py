"""The LDL^T inertia count used by the full-size GPU test, checked on the CPU against the
eigenvalues of small symmetric matrices (torch's CPU LDL^T and numpy's eigvalsh)."""
import numpy as np
import pytest

from inertia import negative_eigenvalues_of_ldl


@pytest.mark.parametrize("M,seed", [(1, 0), (2, 1), (7, 2), (30, 3), (101, 4)])
def test_ldl_inertia_matches_eigenvalues(M, seed):
    import torch
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((M, M))
    S = G + G.T
    LD, piv, info = torch.linalg.ldl_factor_ex(torch.as_tensor(S))
    assert int(info) == 0
    assert negative_eigenvalues_of_ldl(LD, piv) == int(np.sum(np.linalg.eigvalsh(S) < 0.0))


def test_ldl_inertia_of_shifted_pencil():
    """#(lambda < sigma) of a pencil (A, B) with B SPD equals the negative count of A - sigma B."""
    import torch
    import gep_inputs as gi
    g = gi.known_spectrum(60, seed=5)
    lam = np.sort(g["lam"])
    for k in (0, 17, 41, 58):
        sigma = 0.5 * (lam[k] + lam[k + 1])
        LD, piv, info = torch.linalg.ldl_factor_ex(torch.as_tensor(g["A"] - sigma * g["B"]))
        assert negative_eigenvalues_of_ldl(LD, piv) == k + 1
