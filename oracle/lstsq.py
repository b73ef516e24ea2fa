"""Oracle: least squares through the tile QR, with accurate refinement.

Test infrastructure only (see the package docstring).

* ``dot2_residual`` / ``dot2_atr``: b - A x and A^T r computed as if in twice
  the working precision, with the compensated dot product "Dot2" of Ogita,
  Rump and Oishi (2005). TwoProduct uses Dekker's splitting (Dekker 1971) so
  that no fused multiply-add is needed; TwoSum is Knuth's.
* ``lstsq``: x from the tile QR (x = R^{-1} (Q^T b)[0:N]), then refinement of
  the augmented system [I A; A^T 0][r; x] = [b; 0] (Bjorck 1967) with the
  compensated residuals, which also converges for large-residual problems.
* ``csne``: corrected semi-normal equations (Bjorck 1987):
  x0 = R^{-1} R^{-T} A^T b, then repeat r = b - A x, R^T R d = A^T r, x += d.
"""

import numpy as np

from .householder import householder_apply_qt, householder_qr
from .tile_qr import apply_q, tile_qr

_SPLIT = 134217729.0  # 2^27 + 1


def _split(a):
    c = _SPLIT * a
    hi = c - (c - a)
    return hi, a - hi


def two_prod(a, b):
    """a * b = p + e exactly (Dekker)."""
    p = a * b
    ah, al = _split(a)
    bh, bl = _split(b)
    e = al * bl - (((p - ah * bh) - al * bh) - ah * bl)
    return p, e


def two_sum(a, b):
    """a + b = s + e exactly (Knuth)."""
    s = a + b
    z = s - a
    e = (a - (s - z)) + (b - z)
    return s, e


def dot2_residual(A, x, b, r=None):
    """b - A x (or b - r - A x), each entry accumulated with Dot2 over the
    columns."""
    A = np.asarray(A, dtype=np.float64)
    s = np.array(b, dtype=np.float64, copy=True)
    c = np.zeros_like(s)
    if r is not None:
        s, e = two_sum(s, -np.asarray(r, dtype=np.float64))
        c += e
    for j in range(A.shape[1]):
        p, e1 = two_prod(A[:, j], -float(x[j]))
        s, e2 = two_sum(s, p)
        c += e1 + e2
    return s + c


def dot2_atr(A, r):
    """A^T r, each entry accumulated with Dot2 over the rows."""
    A = np.asarray(A, dtype=np.float64)
    s = np.zeros(A.shape[1])
    c = np.zeros(A.shape[1])
    for i in range(A.shape[0]):
        p, e1 = two_prod(A[i, :], float(r[i]))
        s, e2 = two_sum(s, p)
        c += e1 + e2
    return s + c


def back_substitute(R, y):
    """Solve R x = y for upper triangular R, row by row."""
    n = R.shape[0]
    x = np.zeros(n)
    for i in range(n - 1, -1, -1):
        x[i] = (y[i] - R[i, i + 1:] @ x[i + 1:]) / R[i, i]
    return x


def forward_substitute_t(R, y):
    """Solve R^T x = y for upper triangular R, row by row."""
    n = R.shape[0]
    x = np.zeros(n)
    for i in range(n):
        x[i] = (y[i] - R[:i, i] @ x[:i]) / R[i, i]
    return x


def lstsq(A, b, nb, ib, records, refine=3):
    """Least-squares solution of min ||b - A x|| through the tile QR with
    ``refine`` steps of augmented-system refinement. Returns (x, F)."""
    A = np.asarray(A, dtype=np.float64)
    F = tile_qr(A, nb, ib, records)
    M, N = A.shape
    R = F.R()
    c = apply_q(F, b, trans=True)
    x = back_substitute(R, c[:N])
    d = c.copy()
    d[:N] = 0.0
    r = apply_q(F, d, trans=False)
    for _ in range(refine):
        f = dot2_residual(A, x, b, r)
        g = -dot2_atr(A, r)
        h = forward_substitute_t(R, g)
        dd = apply_q(F, f, trans=True)
        dx = back_substitute(R, dd[:N] - h)
        e = dd.copy()
        e[:N] = h
        r = r + apply_q(F, e, trans=False)
        x = x + dx
    return x, F


def csne(A, R, b, iters):
    """Corrected semi-normal equations with the given R (any precision, used
    in FP64) and FP64 compensated residuals. Returns the list of iterates."""
    A = np.asarray(A, dtype=np.float64)
    R = np.asarray(R, dtype=np.float64)
    x = back_substitute(R, forward_substitute_t(R, dot2_atr(A, b)))
    xs = [x]
    for _ in range(iters):
        r = dot2_residual(A, x, b)
        d = back_substitute(R, forward_substitute_t(R, dot2_atr(A, r)))
        x = x + d
        xs.append(x)
    return xs


def lstsq_unblocked(A, b, refine=3):
    """Least squares for any shape M >= N through the unblocked Householder
    QR, with the same augmented-system refinement and Dot2 residuals as
    ``lstsq``. Used where the tile shape does not divide the matrix."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    M, N = A.shape
    R, V, tau = householder_qr(A)

    def qt(v):
        return householder_apply_qt(V, tau, v)

    def q(v):
        v = np.array(v, dtype=np.float64, copy=True)
        for j in range(N - 1, -1, -1):
            w = V[j:, j]
            v[j:] -= tau[j] * w * (w @ v[j:])
        return v

    c = qt(b)
    x = back_substitute(R, c[:N])
    d = c.copy()
    d[:N] = 0.0
    r = q(d)
    for _ in range(refine):
        f = dot2_residual(A, x, b, r)
        g = -dot2_atr(A, r)
        h = forward_substitute_t(R, g)
        dd = qt(f)
        dx = back_substitute(R, dd[:N] - h)
        e = dd.copy()
        e[:N] = h
        r = r + q(e)
        x = x + dx
    return x
