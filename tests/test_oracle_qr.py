"""Pins for the oracle's FP64 tile kernels, tile QR, apply-Q and least squares.

Pinned against: LAPACK (numpy.linalg.qr) on single tiles and stacked pairs, the
defining property Q^T A = [R; 0] of every kernel (catches a transposed T or a
wrong sign), the uniqueness of |R| (unblocked Householder QR and LAPACK),
closed forms (triangular and orthogonal inputs, one column), inner-blocking
invariance, the backward-error bounds of Sec. 5.1, and exactly solvable least
squares problems.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

from oracle import kernels
from oracle.elim_list import BINARY, FIBONACCI, FLAT, GREEDY, hqr_elim_list
from oracle.householder import householder_qr
from oracle.lstsq import csne, dot2_atr, dot2_residual, lstsq
from oracle.tile_qr import apply_q, explicit_q, tile_qr

TREES = (FLAT, BINARY, GREEDY, FIBONACCI)


def rng(seed):
    return np.random.default_rng(seed)


def test_householder_reflector():
    r = rng(1)
    for alpha in (1.3, -0.7, 0.0, -0.0):
        x2 = r.standard_normal(7)
        beta, tau, v2 = kernels.householder(alpha, x2)
        v = np.concatenate(([1.0], v2))
        H = np.eye(8) - tau * np.outer(v, v)
        y = H @ np.concatenate(([alpha], x2))
        assert abs(y[0] - beta) < 1e-14 * abs(beta)
        assert np.max(np.abs(y[1:])) < 1e-14 * abs(beta)
        assert np.allclose(H @ H.T, np.eye(8), atol=1e-14)
        # sign rule: beta has the opposite sign of alpha, sign(+-0) = +1
        assert beta < 0 if alpha >= 0 else beta > 0
    # s = 0: identity reflector, beta = alpha exactly
    beta, tau, v2 = kernels.householder(-2.5, np.zeros(5))
    assert beta == -2.5 and tau == 0.0 and not v2.any()


def _rt(R):
    """|R| with rows made sign-consistent (positive diagonal)."""
    s = np.sign(np.diag(R))
    s[s == 0] = 1
    return R * s[:, None]


@pytest.mark.parametrize("b,ib", [(16, 4), (16, 16), (24, 5), (8, 3)])
def test_geqrt_unmqr(b, ib):
    A0 = rng(b + ib).standard_normal((b, b))
    A = A0.copy()
    T = kernels.geqrt(A, ib)
    R = np.triu(A)
    assert np.allclose(_rt(R), _rt(np.linalg.qr(A0)[1]), atol=1e-13)
    # Q^T A0 = R (defining property; fails for a transposed T or a sign slip)
    C = A0.copy()
    kernels.unmqr(A, T, C, ib, trans=True)
    assert np.max(np.abs(C - R)) < 1e-13
    # Q (Q^T A0) = A0 and Q is orthogonal
    kernels.unmqr(A, T, C, ib, trans=False)
    assert np.max(np.abs(C - A0)) < 1e-13
    Q = np.eye(b)
    kernels.unmqr(A, T, Q, ib, trans=False)
    assert np.max(np.abs(Q.T @ Q - np.eye(b))) < 1e-14
    assert np.max(np.abs(Q @ R - A0)) < 1e-13


@pytest.mark.parametrize("b,ib", [(16, 4), (16, 16), (12, 5)])
def test_tsqrt_tsmqr(b, ib):
    r = rng(10 + b)
    R0 = np.triu(r.standard_normal((b, b)))
    Vjunk = np.tril(r.standard_normal((b, b)), -1)  # killer's own GEQRT V
    A0 = r.standard_normal((b, b))
    R = R0 + Vjunk
    A = A0.copy()
    T = kernels.tsqrt(R, A, ib)
    assert np.array_equal(np.tril(R, -1), Vjunk)  # V part untouched
    Rn = np.triu(R)
    stacked = np.vstack([R0, A0])
    assert np.allclose(_rt(Rn), _rt(np.linalg.qr(stacked)[1]), atol=1e-13)
    C1, C2 = R0.copy(), A0.copy()
    kernels.tsmqr(A, T, C1, C2, ib, trans=True)
    assert np.max(np.abs(C1 - Rn)) < 1e-13 and np.max(np.abs(C2)) < 1e-13
    kernels.tsmqr(A, T, C1, C2, ib, trans=False)
    assert np.max(np.abs(C1 - R0)) < 1e-13 and np.max(np.abs(C2 - A0)) < 1e-13


@pytest.mark.parametrize("b,ib", [(16, 4), (16, 16), (12, 5)])
def test_ttqrt_ttmqr(b, ib):
    r = rng(20 + b)
    R10 = np.triu(r.standard_normal((b, b)))
    R20 = np.triu(r.standard_normal((b, b)))
    J1 = np.tril(r.standard_normal((b, b)), -1)
    J2 = np.tril(r.standard_normal((b, b)), -1)
    R1, R2 = R10 + J1, R20 + J2
    T = kernels.ttqrt(R1, R2, ib)
    assert np.array_equal(np.tril(R1, -1), J1) and np.array_equal(np.tril(R2, -1), J2)
    Rn = np.triu(R1)
    assert np.allclose(_rt(Rn), _rt(np.linalg.qr(np.vstack([R10, R20]))[1]), atol=1e-13)
    C1, C2 = R10.copy(), R20.copy()
    kernels.ttmqr(R2, T, C1, C2, ib, trans=True)
    assert np.max(np.abs(C1 - Rn)) < 1e-13 and np.max(np.abs(C2)) < 1e-13
    # a full (non-triangular) C is mapped back exactly by Q after Q^T
    D1, D2 = r.standard_normal((b, 3)), r.standard_normal((b, 3))
    E1, E2 = D1.copy(), D2.copy()
    kernels.ttmqr(R2, T, E1, E2, ib, trans=True)
    kernels.ttmqr(R2, T, E1, E2, ib, trans=False)
    assert np.max(np.abs(E1 - D1)) < 1e-13 and np.max(np.abs(E2 - D2)) < 1e-13


def _list(m, n, a, p, low, high):
    return hqr_elim_list(m, n, a, p, low, high)


@pytest.mark.parametrize("low,high", list(itertools.product(TREES, TREES)))
def test_tile_qr_matches_unblocked(low, high):
    b, ib, m, n = 8, 3, 7, 4
    A = rng(5).standard_normal((m * b, n * b))
    Ru = _rt(householder_qr(A)[0])
    nrm = np.linalg.norm(A)
    for a, p in ((1, 1), (2, 1), (2, 3), (4, 2), (m, 1)):
        F = tile_qr(A, b, ib, _list(m, n, a, p, low, high))
        assert np.max(np.abs(_rt(F.R()) - Ru)) <= 1e-12 * nrm


@pytest.mark.parametrize("low,high", [(FLAT, FLAT), (GREEDY, FIBONACCI), (BINARY, GREEDY)])
def test_tile_qr_with_coupling_level_matches_unblocked(low, high):
    """Lists with the coupling (domino) level of Sec. 4.2 are valid factorization orders too."""
    b, ib, m, n = 8, 3, 12, 6
    A = rng(15).standard_normal((m * b, n * b))
    Ru = _rt(householder_qr(A)[0])
    nrm = np.linalg.norm(A)
    for a, p in ((1, 3), (2, 3), (2, 4)):
        F = tile_qr(A, b, ib, hqr_elim_list(m, n, a, p, low, high, domino=True))
        assert np.max(np.abs(_rt(F.R()) - Ru)) <= 1e-12 * nrm


def test_unblocked_matches_lapack():
    A = rng(6).standard_normal((50, 20))
    assert np.allclose(_rt(householder_qr(A)[0]), _rt(np.linalg.qr(A)[1]), atol=1e-13)


@pytest.mark.parametrize("low,high,a,p", [(FLAT, FLAT, 8, 1), (GREEDY, FIBONACCI, 2, 3),
                                          (BINARY, GREEDY, 1, 2), (FIBONACCI, BINARY, 3, 4)])
def test_backward_error_and_orthogonality(low, high, a, p):
    b, ib, m, n = 8, 4, 9, 5
    A = rng(7).standard_normal((m * b, n * b))
    F = tile_qr(A, b, ib, _list(m, n, a, p, low, high))
    Q = explicit_q(F)
    R = F.R()
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= 1e-13
    assert np.linalg.norm(Q.T @ Q - np.eye(n * b)) <= 1e-12
    # Q^T A = [R; 0]
    QtA = apply_q(F, A, trans=True)
    assert np.max(np.abs(QtA[:n * b] - R)) <= 1e-12 * np.linalg.norm(A)
    assert np.max(np.abs(QtA[n * b:])) <= 1e-12 * np.linalg.norm(A)
    # full Q is orthogonal too
    Qf = apply_q(F, np.eye(m * b), trans=False)
    assert np.linalg.norm(Qf.T @ Qf - np.eye(m * b)) <= 1e-12


def test_triangular_input_is_exact():
    b, ib, m, n = 8, 3, 6, 6
    A = np.triu(rng(8).standard_normal((m * b, n * b)))
    for low, high in itertools.product(TREES, TREES):
        for a, p in ((1, 1), (3, 2), (6, 1)):
            F = tile_qr(A, b, ib, _list(m, n, a, p, low, high))
            assert np.array_equal(F.R(), A)
            assert np.array_equal(explicit_q(F), np.eye(m * b))


def test_orthogonal_input():
    b, ib, m, n = 8, 4, 6, 6
    Q0 = np.linalg.qr(rng(9).standard_normal((m * b, m * b)))[0]
    F = tile_qr(Q0, b, ib, _list(m, n, 2, 2, GREEDY, FIBONACCI))
    assert np.max(np.abs(np.abs(F.R()) - np.eye(m * b))) <= 1e-14 * 10


def test_one_column():
    b, ib, m = 8, 4, 5
    A = rng(10).standard_normal((m * b, b))
    F = tile_qr(A, b, ib, _list(m, 1, 1, 2, BINARY, GREEDY))
    assert abs(abs(F.R()[0, 0]) - np.linalg.norm(A[:, 0])) <= 1e-14 * np.linalg.norm(A[:, 0])


def test_inner_blocking_invariance():
    b, m, n = 12, 4, 3
    A = rng(11).standard_normal((m * b, n * b))
    L = _list(m, n, 2, 1, GREEDY, FLAT)
    R0 = tile_qr(A, b, b, L).R()
    for ib in (1, 2, 3, 4, 5, 6):
        R = tile_qr(A, b, ib, L).R()
        assert np.max(np.abs(R - R0)) <= 1e-13 * np.linalg.norm(A)


def test_ts_vs_tt_same_r():
    # Sec. 2: a TS kill does the work of GEQRT + TTQRT; same |R| either way
    b, ib, m, n = 8, 4, 6, 3
    A = rng(12).standard_normal((m * b, n * b))
    Rts = tile_qr(A, b, ib, _list(m, n, m, 1, FLAT, FLAT)).R()
    Rtt = tile_qr(A, b, ib, _list(m, n, 1, 1, FLAT, FLAT)).R()
    assert np.max(np.abs(_rt(Rts) - _rt(Rtt))) <= 1e-13 * np.linalg.norm(A)


def test_dot2_exact_rational():
    r = rng(13)
    A = r.standard_normal((6, 40)) * np.logspace(0, 12, 40)
    x = r.standard_normal(40)
    b = A @ x  # residual is pure cancellation
    res = dot2_residual(A, x, b)
    for i in range(6):
        exact = Fraction(b[i]) - sum(Fraction(A[i, j]) * Fraction(x[j]) for j in range(40))
        scale = sum(abs(Fraction(A[i, j]) * Fraction(x[j])) for j in range(40))
        assert abs(Fraction(res[i]) - exact) <= Fraction(1e-26) * scale + abs(exact) * Fraction(2.3e-16)
    y = r.standard_normal(6)
    g = dot2_atr(A, y)
    for j in range(40):
        exact = sum(Fraction(A[i, j]) * Fraction(y[i]) for i in range(6))
        assert abs(Fraction(g[j]) - exact) <= abs(exact) * Fraction(2.3e-16) + Fraction(1e-300)


def test_lstsq_consistent_and_large_residual():
    b, ib, m, n = 8, 4, 8, 3
    r = rng(14)
    A = r.standard_normal((m * b, n * b))
    xt = r.standard_normal(n * b)
    L = _list(m, n, 2, 2, GREEDY, FIBONACCI)
    x, _ = lstsq(A, A @ xt, b, ib, L)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= 1e-14
    # large residual: the solution is fixed by the normal equations
    bb = r.standard_normal(m * b)
    x, _ = lstsq(A, bb, b, ib, L)
    xe = np.linalg.lstsq(A, bb, rcond=None)[0]
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 1e-13
    assert np.linalg.norm(A.T @ (bb - A @ x)) <= 1e-12 * np.linalg.norm(A) * np.linalg.norm(bb)


def test_csne_converges_with_perturbed_r():
    b, ib, m, n = 8, 4, 8, 4
    r = rng(15)
    A = r.standard_normal((m * b, n * b))
    xt = r.standard_normal(n * b)
    bb = A @ xt + 1e-8 * r.standard_normal(m * b)
    xe, F = lstsq(A, bb, b, ib, _list(m, n, 1, 1, GREEDY, FLAT))
    # R from a single-precision QR
    R32 = np.linalg.qr(A.astype(np.float32))[1].astype(np.float64)
    xs = csne(A, R32, bb, 6)
    errs = [np.linalg.norm(x - xe) / np.linalg.norm(xe) for x in xs]
    assert errs[-1] <= 1e-13 and errs[-1] < errs[0]


def test_lstsq_unblocked_any_shape():
    from oracle.lstsq import lstsq_unblocked
    r = rng(16)
    for M, N in ((70, 23), (33, 33), (100, 1)):
        A = r.standard_normal((M, N))
        xt = r.standard_normal(N)
        x = lstsq_unblocked(A, A @ xt)
        assert np.linalg.norm(x - xt) / np.linalg.norm(xt) <= 1e-13
        b = r.standard_normal(M)
        x = lstsq_unblocked(A, b)
        xe = np.linalg.lstsq(A, b, rcond=None)[0]
        assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 1e-12
