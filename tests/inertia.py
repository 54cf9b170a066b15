"""Inertia of a symmetric matrix from a library LDL^T factorisation (test helper)."""


def negative_eigenvalues_of_ldl(LD, piv):
    """Number of negative eigenvalues of the block-diagonal D of a Bunch-Kaufman LDL^T
    factorisation (lower storage, LAPACK pivot convention: piv[i] < 0 marks the 2 x 2 block
    (i, i+1)); by Sylvester's law of inertia it is the negative count of the factored matrix."""
    d = LD.diagonal().cpu().numpy()
    sub = LD.diagonal(-1).cpu().numpy()
    piv = piv.cpu().numpy()
    n, neg, i = d.shape[0], 0, 0
    while i < n:
        if piv[i] > 0:
            neg += int(d[i] < 0.0)
            i += 1
        else:
            a, b, c = d[i], sub[i], d[i + 1]
            det = a * c - b * b
            neg += 1 if det < 0.0 else (2 if a < 0.0 else 0)
            i += 2
    return neg
