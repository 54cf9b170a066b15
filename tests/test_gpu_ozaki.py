"""The split-BF16 tensor-core product engine against FP64 references.

Small-integer operands are split exactly (one digit each), so the product must be
bit-identical to the FP64 result.  General operands must agree with a
componentwise bound 1e-14 * (|A||B|)_ij, far inside the FP64 engine's own
rounding bound k * eps * (|A||B|)_ij for these depths.
"""
import numpy as np
import pytest

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


@pytest.mark.parametrize("m,n,k", [(128, 64, 32), (300, 200, 500), (1000, 130, 4500)])
def test_integer_products_are_exact(gep, m, n, k):
    rng = np.random.default_rng(m + n + k)
    A = rng.integers(-100, 101, size=(m, k)).astype(np.float64)
    B = rng.integers(-100, 101, size=(k, n)).astype(np.float64)
    out = host(gep.dgemm(dev(A), dev(B), engine="fp64_emulated"))
    assert np.array_equal(out, A @ B)


@pytest.mark.parametrize("ta,tb", [("N", "N"), ("N", "T"), ("T", "N"), ("T", "T")])
@pytest.mark.parametrize("m,n,k", [(128, 64, 16), (257, 130, 333), (640, 512, 5000)])
def test_random_products_fp64_accurate(gep, ta, tb, m, n, k):
    rng = np.random.default_rng(7 * m + n + k)
    A = rng.standard_normal((k, m) if ta == "T" else (m, k)) * np.exp(rng.uniform(-3, 3, size=(1, 1)))
    B = rng.standard_normal((n, k) if tb == "T" else (k, n))
    C = rng.standard_normal((m, n))
    Ao = A.T if ta == "T" else A
    Bo = B.T if tb == "T" else B
    ref = 1.5 * Ao @ Bo - 0.25 * C
    bound = 1e-14 * (1.5 * np.abs(Ao) @ np.abs(Bo) + 0.25 * np.abs(C))
    out = host(gep.dgemm(dev(A), dev(B), ta, tb, alpha=1.5, beta=-0.25, C=dev(C), engine="fp64_emulated"))
    assert np.all(np.abs(out - ref) <= bound)


def test_wide_dynamic_range_rows(gep):
    """Rows scaled over 2^-200 .. 2^200: per-row exponents keep relative accuracy."""
    rng = np.random.default_rng(3)
    m, n, k = 256, 128, 700
    A = rng.standard_normal((m, k)) * np.exp2(rng.integers(-200, 200, size=(m, 1)))
    B = rng.standard_normal((k, n)) * np.exp2(rng.integers(-50, 50, size=(1, n)))
    ref = A @ B
    out = host(gep.dgemm(dev(A), dev(B), engine="fp64_emulated"))
    assert np.all(np.abs(out - ref) <= 1e-14 * (np.abs(A) @ np.abs(B)))


def test_lower_only_and_zero_rows(gep):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((300, 90))
    A[17] = 0.0
    C = rng.standard_normal((300, 300))
    out = host(gep.dgemm(dev(A), dev(A), "N", "T", alpha=-1.0, beta=1.0, C=dev(C), uplo="L",
                         engine="fp64_emulated"))
    ref = C - A @ A.T
    il = np.tril_indices(300)
    iu = np.triu_indices(300, 1)
    assert np.max(np.abs(out[il] - ref[il])) <= 1e-13
    assert np.array_equal(out[iu], C[iu])


def test_mixed_levels_are_fp32_grade(gep):
    rng = np.random.default_rng(5)
    A = rng.standard_normal((512, 512))
    B = rng.standard_normal((512, 512))
    out = host(gep.dgemm(dev(A), dev(B), engine="mixed_refined"))
    rel = np.max(np.abs(out - A @ B) / (np.abs(A) @ np.abs(B)))
    assert rel <= 2e-6, rel


@pytest.mark.parametrize("engine", ["fp64", "fp64_emulated"])
@pytest.mark.parametrize("m,n", [(130, 64), (300, 70), (5000, 64)])
def test_symmetric_lower_operand(gep, engine, m, n):
    """transa 'S': A symmetric, only its lower triangle read (the upper one holds NaN);
    m = 5000 spans two K panels of the split-BF16 engine."""
    rng = np.random.default_rng(m + n)
    G = rng.standard_normal((m, m))
    S = (G + G.T) / 2
    A = np.tril(S) + np.triu(np.full((m, m), np.nan), 1)
    B = rng.standard_normal((m, n))
    ref = S @ B
    out = host(gep.dgemm(dev(A), dev(B), "S", "N", engine=engine))
    bound = 1e-14 * (np.abs(S) @ np.abs(B)) + 1e-300
    assert np.all(np.isfinite(out))
    assert np.all(np.abs(out - ref) <= bound * (4 if engine == "fp64" else 1) + 4 * m * 2.0 ** -52 * (np.abs(S) @ np.abs(B)) * (engine == "fp64"))
