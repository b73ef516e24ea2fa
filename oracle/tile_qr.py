"""Oracle: tile QR that follows an elimination list, and Q / Q^T application.

Test infrastructure only (see the package docstring).

``tile_qr`` runs Alg. 1 with the elimination ``elim(i, killer, k)`` expanded as
in Alg. 2: the killer (and, for a TT elimination, the killed row) is first made
a triangle by GEQRT and its trailing tiles updated by UNMQR, once per row and
panel; then TSQRT + TSMQR (TS) or TTQRT + TTMQR (TT) zero tile (i, k) and
update the pairs of tiles (killer, j), (i, j) for j > k. Records are replayed
one panel at a time in the list's order, which satisfies every dependency of
Sec. 2.

The factorization is stored as the operation sequence it ran, so that Q^T B is
that sequence replayed forward and Q B the same sequence replayed backwards
with untransposed blocks (Sec. 5.1 forms Q by applying the reverse trees to
the identity).
"""

import numpy as np

from . import kernels
from .elim_list import TS, TT


class TileQR:
    """Result of ``tile_qr``: the factored matrix (R in the upper triangles
    of the tiles on and above the diagonal, V parts elsewhere), the T factors
    and the list of operations in execution order."""

    def __init__(self, A, b, ib, ops, Tg, Tk):
        self.A = A
        self.b = b
        self.ib = ib
        self.ops = ops
        self.Tg = Tg
        self.Tk = Tk

    @property
    def m(self):
        return self.A.shape[0] // self.b

    @property
    def n(self):
        return self.A.shape[1] // self.b

    def tile(self, i, j):
        b = self.b
        return self.A[i * b:(i + 1) * b, j * b:(j + 1) * b]

    def R(self):
        """The N x N upper triangular factor."""
        N = self.A.shape[1]
        return np.triu(self.A[:N, :N])


def panel_ops(records, k):
    """Operations of panel k in execution order: ("geqrt", r) the first time
    row r is used as a triangle, then ("ts"|"tt", i, killer) per record."""
    ops = []
    done = set()
    recs = [r for r in records if r[0] == k]
    for (kk, i, killer, kind, level, step) in recs:
        if killer not in done:
            ops.append(("geqrt", k, killer))
            done.add(killer)
        if kind == TT and i not in done:
            ops.append(("geqrt", k, i))
            done.add(i)
        ops.append(("ts" if kind == TS else "tt", k, i, killer))
    if not recs:
        ops.append(("geqrt", k, k))
    return ops


def tile_qr(A, b, ib, records):
    """Factor a copy of A (M x N, M = m b, N = n b, m >= n) with tile size b,
    inner block ib and the given elimination list."""
    A = np.array(A, dtype=np.float64, copy=True)
    M, N = A.shape
    if M % b or N % b:
        raise ValueError("M and N must be multiples of b")
    m, n = M // b, N // b
    Tg, Tk = {}, {}
    ops = []
    F = TileQR(A, b, ib, ops, Tg, Tk)
    for k in range(min(m, n)):
        for op in panel_ops(records, k):
            ops.append(op)
            if op[0] == "geqrt":
                _, _, r = op
                Tg[(r, k)] = kernels.geqrt(F.tile(r, k), ib)
                for j in range(k + 1, n):
                    kernels.unmqr(F.tile(r, k), Tg[(r, k)], F.tile(r, j), ib)
            elif op[0] == "ts":
                _, _, i, killer = op
                Tk[(i, k)] = kernels.tsqrt(F.tile(killer, k), F.tile(i, k), ib)
                for j in range(k + 1, n):
                    kernels.tsmqr(F.tile(i, k), Tk[(i, k)], F.tile(killer, j), F.tile(i, j), ib)
            else:
                _, _, i, killer = op
                Tk[(i, k)] = kernels.ttqrt(F.tile(killer, k), F.tile(i, k), ib)
                for j in range(k + 1, n):
                    kernels.ttmqr(F.tile(i, k), Tk[(i, k)], F.tile(killer, j), F.tile(i, j), ib)
    return F


def apply_q(F, B, trans):
    """Return Q^T B (trans=True) or Q B (trans=False) for the factorization F.
    B has M rows (any number of columns)."""
    B = np.array(B, dtype=np.float64, copy=True)
    b, ib = F.b, F.ib
    if B.ndim == 1:
        B = B[:, None]
        squeeze = True
    else:
        squeeze = False

    def rows(r):
        return B[r * b:(r + 1) * b, :]

    seq = F.ops if trans else F.ops[::-1]
    for op in seq:
        if op[0] == "geqrt":
            _, k, r = op
            kernels.unmqr(F.tile(r, k), F.Tg[(r, k)], rows(r), ib, trans)
        elif op[0] == "ts":
            _, k, i, killer = op
            kernels.tsmqr(F.tile(i, k), F.Tk[(i, k)], rows(killer), rows(i), ib, trans)
        else:
            _, k, i, killer = op
            kernels.ttmqr(F.tile(i, k), F.Tk[(i, k)], rows(killer), rows(i), ib, trans)
    return B[:, 0] if squeeze else B


def explicit_q(F, ncols=None):
    """The first ``ncols`` columns of Q (default N): Q applied to I."""
    M, N = F.A.shape
    ncols = N if ncols is None else ncols
    E = np.zeros((M, ncols))
    E[np.arange(ncols), np.arange(ncols)] = 1.0
    return apply_q(F, E, trans=False)
