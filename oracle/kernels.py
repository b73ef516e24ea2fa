"""Oracle: the six FP64 tile kernels of tile Householder QR.

Test infrastructure only (see the package docstring).

The paper names the kernels, their roles and their weights (Sec. 2, Alg. 2):
GEQRT (square -> triangle), TSQRT (a triangle kills a square), TTQRT (a
triangle kills a triangle), and the updates UNMQR, TSMQR and TTMQR that apply
the same transformations to the tiles of the trailing columns. It does not
print their arithmetic; the form used here is the standard compact-WY
Householder formulation (Schreiber and Van Loan 1989), with the reflectors of a
tile grouped ``ib`` at a time:

* Householder vector of a column x = (alpha, x2): s = ||x2||_2. If s == 0 the
  reflector is the identity (tau = 0, beta = alpha). Otherwise
  beta = -sign(alpha) * sqrt(alpha^2 + s^2) with sign(+-0) = +1,
  tau = (beta - alpha) / beta, v = (1, x2 / (alpha - beta)).
  H = I - tau v v^T maps x to (beta, 0, ..., 0).
* A block of w reflectors H_0 H_1 ... H_{w-1} = I - V T V^T with T upper
  triangular: T[j, j] = tau_j, T[:j, j] = -tau_j * T[:j, :j] @ (V[:, :j]^T v_j).
* The block's transpose is applied as C <- C - V (T^T (V^T C)).
* A tile's T is an ib x b array: block q (columns q*ib ...) holds its w x w
  triangle in rows 0..w-1 of columns q*ib .. q*ib+w-1.

Storage (in place, LAPACK-style):

* GEQRT: R on and above the diagonal of the tile, V strictly below (unit
  diagonal implied).
* TSQRT: R updated in the upper triangle of the killer tile (its strict lower
  part, the killer's own GEQRT V, is neither read nor written); the killed
  tile is overwritten by the full b x b V2 (the reflectors are [e_j; V2[:, j]]).
* TTQRT: as TSQRT but both tiles are upper triangles; V2 is upper triangular
  and overwrites the upper triangle (with the diagonal) of the killed tile,
  whose strict lower part (its GEQRT V) is untouched.
"""

import numpy as np


def householder(alpha, x2):
    """Householder vector of the column (alpha, x2) in the convention above.
    Returns (beta, tau, v2) with v2 = x2 / (alpha - beta)."""
    s = float(np.linalg.norm(x2)) if x2.size else 0.0
    if s == 0.0:
        return alpha, 0.0, np.zeros_like(x2)
    nrm = float(np.hypot(alpha, s))
    beta = -nrm if alpha >= 0.0 else nrm
    tau = (beta - alpha) / beta
    return beta, tau, x2 / (alpha - beta)


def _t_column(T, V, j, tau):
    """Column j of the block T factor: T[j, j] = tau and
    T[:j, j] = -tau * T[:j, :j] @ (V[:, :j]^T V[:, j])."""
    T[j, j] = tau
    if j > 0:
        T[:j, j] = -tau * (T[:j, :j] @ (V[:, :j].T @ V[:, j]))


def _blocks(b, ib):
    return [(j0, min(ib, b - j0)) for j0 in range(0, b, ib)]


def geqrt(A, ib):
    """QR of a square b x b tile in place (A <- R and V). Returns T (ib x b)."""
    b = A.shape[0]
    T = np.zeros((ib, b))
    for j0, w in _blocks(b, ib):
        Tb = np.zeros((w, w))
        Vb = np.zeros((b - j0, w))
        for jj in range(w):
            j = j0 + jj
            beta, tau, v2 = householder(A[j, j], A[j + 1:, j])
            A[j, j] = beta
            A[j + 1:, j] = v2
            v = np.concatenate(([1.0], v2))
            Vb[jj:, jj] = v
            # apply H_j to the rest of the block's columns
            C = A[j:, j + 1:j0 + w]
            C -= tau * np.outer(v, v @ C)
            _t_column(Tb, Vb, jj, tau)
        # apply the block's transpose to the trailing columns of the tile
        C = A[j0:, j0 + w:]
        if C.shape[1]:
            C -= Vb @ (Tb.T @ (Vb.T @ C))
        T[:w, j0:j0 + w] = Tb
    return T


def geqrt_v(A, j0, w):
    """The unit lower V of columns j0..j0+w-1 of a GEQRT-factored tile, rows
    j0..b-1."""
    b = A.shape[0]
    V = np.tril(A[j0:, j0:j0 + w], -1)
    for jj in range(w):
        V[jj, jj] = 1.0
    return V


def unmqr(Af, T, C, ib, trans=True):
    """C <- Q^T C (trans) or Q C, with Q from the GEQRT-factored tile Af."""
    b = Af.shape[0]
    blocks = _blocks(b, ib)
    if not trans:
        blocks = blocks[::-1]
    for j0, w in blocks:
        V = geqrt_v(Af, j0, w)
        Tb = T[:w, j0:j0 + w]
        Cb = C[j0:, :]
        W = V.T @ Cb
        W = (Tb.T if trans else Tb) @ W
        Cb -= V @ W


def tsqrt(R, A, ib):
    """QR of [triangle R; square A] in place. R's upper triangle is updated,
    A becomes V2. Returns T (ib x b)."""
    b = R.shape[0]
    T = np.zeros((ib, b))
    for j0, w in _blocks(b, ib):
        Tb = np.zeros((w, w))
        for jj in range(w):
            j = j0 + jj
            beta, tau, v2 = householder(R[j, j], A[:, j])
            R[j, j] = beta
            A[:, j] = v2
            # the top part of this reflector is e_j, so it only touches row j
            # of R and all of A
            cols = slice(j + 1, j0 + w)
            wv = R[j, cols] + v2 @ A[:, cols]
            R[j, cols] -= tau * wv
            A[:, cols] -= tau * np.outer(v2, wv)
            # V^T v for the stacked vectors reduces to the A parts
            _t_column(Tb, A[:, j0:j0 + w], jj, tau)
        cols = slice(j0 + w, b)
        if j0 + w < b:
            V2 = A[:, j0:j0 + w]
            W = R[j0:j0 + w, cols] + V2.T @ A[:, cols]
            W = Tb.T @ W
            R[j0:j0 + w, cols] -= W
            A[:, cols] -= V2 @ W
        T[:w, j0:j0 + w] = Tb
    return T


def tsmqr(V2, T, C1, C2, ib, trans=True):
    """[C1; C2] <- Q^T [C1; C2] (trans) or Q [C1; C2], with Q from TSQRT
    (reflectors [e_j; V2[:, j]])."""
    b = V2.shape[0]
    blocks = _blocks(b, ib)
    if not trans:
        blocks = blocks[::-1]
    for j0, w in blocks:
        V = V2[:, j0:j0 + w]
        Tb = T[:w, j0:j0 + w]
        W = C1[j0:j0 + w, :] + V.T @ C2
        W = (Tb.T if trans else Tb) @ W
        C1[j0:j0 + w, :] -= W
        C2 -= V @ W


def ttqrt(R1, R2, ib):
    """QR of [triangle R1; triangle R2] in place. R1's upper triangle is
    updated; R2's upper triangle (with the diagonal) becomes the upper
    triangular V2. Strict lower parts of both tiles are not touched.
    Returns T (ib x b)."""
    b = R1.shape[0]
    T = np.zeros((ib, b))
    for j0, w in _blocks(b, ib):
        Tb = np.zeros((w, w))
        Vb = np.zeros((j0 + w, w))
        for jj in range(w):
            j = j0 + jj
            beta, tau, v2 = householder(R1[j, j], R2[:j + 1, j])
            R1[j, j] = beta
            R2[:j + 1, j] = v2
            Vb[:j + 1, jj] = v2
            cols = slice(j + 1, j0 + w)
            wv = R1[j, cols] + v2 @ R2[:j + 1, cols]
            R1[j, cols] -= tau * wv
            R2[:j + 1, cols] -= tau * np.outer(v2, wv)
            _t_column(Tb, Vb, jj, tau)
        if j0 + w < b:
            cols = slice(j0 + w, b)
            W = R1[j0:j0 + w, cols] + Vb.T @ R2[:j0 + w, cols]
            W = Tb.T @ W
            R1[j0:j0 + w, cols] -= W
            R2[:j0 + w, cols] -= Vb @ W
        T[:w, j0:j0 + w] = Tb
    return T


def ttqrt_v(R2f, j0, w):
    """Upper triangular V2 of columns j0..j0+w-1 of a TTQRT-factored tile,
    rows 0..j0+w-1 (entries below each column's diagonal are zero)."""
    return np.triu(R2f[:j0 + w, j0:j0 + w], -j0)


def ttmqr(R2f, T, C1, C2, ib, trans=True):
    """[C1; C2] <- Q^T [C1; C2] (trans) or Q [C1; C2], with Q from TTQRT
    (upper triangular V2 stored in the upper triangle of R2f)."""
    b = R2f.shape[0]
    blocks = _blocks(b, ib)
    if not trans:
        blocks = blocks[::-1]
    for j0, w in blocks:
        V = ttqrt_v(R2f, j0, w)
        Tb = T[:w, j0:j0 + w]
        W = C1[j0:j0 + w, :] + V.T @ C2[:j0 + w, :]
        W = (Tb.T if trans else Tb) @ W
        C1[j0:j0 + w, :] -= W
        C2[:j0 + w, :] -= V @ W
