"""Oracle: unblocked column-by-column Householder QR (definition oracle).

Test infrastructure only (see the package docstring).

Column j of the M x N matrix is reduced by one Householder reflector in the
same sign convention as the tile kernels (``oracle.kernels.householder``), and
the reflector is applied to the columns right of it. The R factor of a
full-rank matrix is unique up to the signs of its rows, so |R| from any tile
QR must agree with |R| from here up to rounding.
"""

import numpy as np

from .kernels import householder


def householder_qr(A):
    """Returns (R, V, tau): R is N x N upper triangular, V (M x N) holds the
    unit lower Householder vectors, tau their scalars."""
    A = np.array(A, dtype=np.float64, copy=True)
    M, N = A.shape
    V = np.zeros((M, N))
    tau = np.zeros(N)
    for j in range(N):
        beta, t, v2 = householder(A[j, j], A[j + 1:, j])
        v = np.concatenate(([1.0], v2))
        C = A[j:, j + 1:]
        C -= t * np.outer(v, v @ C)
        A[j, j] = beta
        A[j + 1:, j] = 0.0
        V[j:, j] = v
        tau[j] = t
    return np.triu(A[:N, :N]), V, tau


def householder_apply_qt(V, tau, B):
    """Q^T B for the reflectors of ``householder_qr``."""
    B = np.array(B, dtype=np.float64, copy=True)
    for j in range(V.shape[1]):
        v = V[j:, j]
        B[j:] -= tau[j] * np.outer(v, v @ B[j:]) if B.ndim == 2 else tau[j] * v * (v @ B[j:])
    return B
