"""Small GF(2) / symplectic helpers used only by the tests.

A Pauli on n qubits is a 2n-bit row (x | z).  These routines are textbook
linear algebra and are independent of both the oracle and the CUDA path.
"""
import numpy as np


def pauli_rows(labels):
    """labels: (k, n) uint8 with I=0, Z=1, X=2, Y=3 -> (k, 2n) uint8 rows (x|z)."""
    labels = np.asarray(labels, np.uint8)
    x = (labels >> 1) & 1
    z = labels & 1
    return np.concatenate([x, z], axis=1).astype(np.uint8)


def symplectic(A, B):
    """Matrix of symplectic products (1 = anticommute) between rows of A and B."""
    n = A.shape[1] // 2
    Ax, Az = A[:, :n].astype(np.int64), A[:, n:].astype(np.int64)
    Bx, Bz = B[:, :n].astype(np.int64), B[:, n:].astype(np.int64)
    return ((Ax @ Bz.T + Az @ Bx.T) & 1).astype(np.uint8)


def rank(M):
    M = np.array(M, dtype=np.uint8) & 1
    rows, cols = M.shape
    r = 0
    for c in range(cols):
        piv = None
        for i in range(r, rows):
            if M[i, c]:
                piv = i
                break
        if piv is None:
            continue
        M[[r, piv]] = M[[piv, r]]
        for i in range(rows):
            if i != r and M[i, c]:
                M[i] ^= M[r]
        r += 1
        if r == rows:
            break
    return r
