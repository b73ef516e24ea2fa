"""GPU parity of the list variants beyond the plain HQR list, through the C
ABI, against the CPU oracle on the same list and the same seeded inputs:

* the coupling ("domino") level of Sec. 4.2 (lists from
  hqr_elim_list_domino), every tree pair, p in {3, 4, 16}, a in {1, 2, 4};
  FP64, FP32 CUDA-core and tensor-core arithmetic; Q and Q^T applied;
* the prior-art lists the paper compares with in Sec. 5, run on the same
  kernels: [SLHD10] (p = 1, TS domains of a = m / r tiles, binary low tree)
  and [BBD+10] (the flat tile QR: p = 1, one TS domain, a = m);
* the look-ahead priority policy 0 (Sec. 4.3 priority function), which must
  give the same bits as the default critical-path priorities, because the
  graph fixes the order of the operations on every tile.

Tolerances as in the other parity tests: FP64 R within 1e-11 ||A||_F, V and
T within 1e-10; FP32 R within 5e-6 ||A||_F.
"""
import itertools

import numpy as np
import pytest

from oracle.elim_list import BINARY, FIBONACCI, FLAT, GREEDY, TREE_NAMES, hqr_elim_list, validate
from oracle.tile_qr import apply_q as o_apply_q
from oracle.tile_qr import tile_qr
from paper_1110_1553_gb300 import inputs

torch = pytest.importorskip("torch")
hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")

pytestmark = pytest.mark.gpu
TREES = (FLAT, BINARY, GREEDY, FIBONACCI)
R_TOL = 1e-11
VT_TOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()
    hqr.set_timeout_ms(20000)


def lib_list(m, n, a, p, low, high, domino=False):
    """The library's list, checked bit for bit against the oracle's."""
    recs = hqr.as_records(hqr.elim_list(m, n, a, p, TREE_NAMES[low], TREE_NAMES[high], domino=domino))
    ref = hqr_elim_list(m, n, a, p, low, high, domino=domino)
    assert [tuple(r) for r in recs] == [tuple(r) for r in ref]
    assert validate(ref, m, n) is None
    return ref


def factor_fp64(A, nb, ib, recs):
    Fo = tile_qr(A, nb, ib, recs)
    Fg = hqr.geqrf(torch.from_numpy(np.ascontiguousarray(A)).cuda(), nb, ib, recs)
    return Fo, Fg


def compare_fp64(Fo, Fg, A):
    nrm = np.linalg.norm(A)
    N = Fg.N
    Rg = Fg.R().cpu().numpy()
    assert np.max(np.abs(Rg - np.triu(Fo.A[:N, :N]))) <= R_TOL * nrm
    tiles = Fg.tiles().cpu().numpy()
    d = np.abs(tiles - Fo.A)
    assert np.max(d) <= max(VT_TOL, R_TOL * nrm), np.unravel_index(np.argmax(d), d.shape)
    T = Fg.T().cpu().numpy()
    for (r, k), To in Fo.Tg.items():
        assert np.max(np.abs(T[k, r, 0].T - To)) <= VT_TOL, ("Tg", r, k)
    for (i, k), To in Fo.Tk.items():
        assert np.max(np.abs(T[k, i, 1].T - To)) <= VT_TOL, ("Tk", i, k)


# ------------------------------------------------------ coupling level --

@pytest.mark.parametrize("low,high", list(itertools.product(TREES, TREES)))
def test_domino_all_tree_pairs(low, high):
    nb, ib, m, n = 16, 4, 24, 4
    A = inputs.gaussian(m * nb, n * nb, seed=801)
    for a, p in ((1, 3), (2, 4), (4, 16), (2, 3)):
        recs = lib_list(m, n, a, p, low, high, domino=True)
        assert any(r[4] == 2 for r in recs)  # the coupling level is there
        Fo, Fg = factor_fp64(A, nb, ib, recs)
        compare_fp64(Fo, Fg, A)


def test_domino_paper_example_shape_and_apply_q():
    """The shape of the worked example of Sec. 4.2 (m = 24, n = 10, p = 3,
    a = 2), with Q^T and Q applied to a block of right-hand sides."""
    nb, ib, m, n = 16, 8, 24, 10
    A = inputs.gaussian(m * nb, n * nb, seed=802)
    recs = lib_list(m, n, 2, 3, GREEDY, FLAT, domino=True)
    Fo, Fg = factor_fp64(A, nb, ib, recs)
    compare_fp64(Fo, Fg, A)
    B = inputs.gaussian(m * nb, 7, seed=803)
    for trans in (True, False):
        out = Fg.apply_q(torch.from_numpy(B.copy()).cuda(), trans=trans).cpu().numpy()
        ref = o_apply_q(Fo, B, trans=trans)
        assert np.max(np.abs(out - ref)) <= 1e-12 * np.linalg.norm(B)


@pytest.mark.parametrize("nb,ib", [(64, 16), (256, 32)])
def test_domino_split_panels_fp64(nb, ib):
    """Tiles from nb = 64 run split panels (one task per ib block)."""
    m, n = 10, 3
    A = inputs.gaussian(m * nb, n * nb, seed=804 + nb)
    recs = lib_list(m, n, 2, 3, GREEDY, FIBONACCI, domino=True)
    Fo, Fg = factor_fp64(A, nb, ib, recs)
    compare_fp64(Fo, Fg, A)


def test_domino_fp32_cuda_cores():
    nb, ib, m, n = 32, 8, 16, 5
    A = inputs.gaussian(m * nb, n * nb, seed=805).astype(np.float32)
    recs = lib_list(m, n, 2, 4, BINARY, GREEDY, domino=True)
    Fo = tile_qr(A.astype(np.float64), nb, ib, recs)
    Fg = hqr.geqrf(torch.from_numpy(A).cuda(), nb, ib, recs)
    nrm = np.linalg.norm(A.astype(np.float64))
    assert np.max(np.abs(Fg.R().cpu().numpy().astype(np.float64) - Fo.R())) <= 5e-6 * nrm
    tiles = Fg.tiles().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(tiles - Fo.A)) <= 5e-5 * max(1.0, nrm)


def test_domino_tensor_cores():
    nb, m, n = 128, 9, 3
    A = inputs.gaussian(m * nb, n * nb, seed=806).astype(np.float32)
    recs = lib_list(m, n, 1, 3, GREEDY, FIBONACCI, domino=True)
    Fo = tile_qr(A.astype(np.float64), nb, nb, recs)
    Fg = hqr.geqrf(torch.from_numpy(A).cuda(), nb, nb, recs, tensor=True)
    nrm = np.linalg.norm(A.astype(np.float64))
    assert np.max(np.abs(Fg.R().cpu().numpy().astype(np.float64) - Fo.R())) <= 5e-6 * nrm
    tiles = Fg.tiles().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(tiles - Fo.A)) <= 5e-5 * max(1.0, nrm)
    B = inputs.gaussian(m * nb, 3, seed=807).astype(np.float32)
    out = Fg.apply_q(torch.from_numpy(B.copy()).cuda(), trans=True).cpu().numpy()
    ref = o_apply_q(Fo, B.astype(np.float64), trans=True)
    assert np.max(np.abs(out - ref)) <= 5e-6 * np.linalg.norm(B.astype(np.float64))


# ------------------------------------------------------ prior-art lists --

def slhd10(m, n, r):
    """[SLHD10] on r processors as HQR parameters (Sec. 5): p = 1, TS domains
    of a = m / r tiles, binary low-level tree."""
    return (max(1, m // r), 1, BINARY, FLAT)


def bbd10(m, n):
    """[BBD+10], the flat tile QR (Sec. 5): p = 1, one TS domain (a = m),
    flat trees."""
    return (m, 1, FLAT, FLAT)


@pytest.mark.parametrize("which", ["slhd10", "bbd10"])
def test_prior_art_lists(which):
    nb, ib, m, n = 32, 8, 32, 4
    a, p, low, high = slhd10(m, n, 4) if which == "slhd10" else bbd10(m, n)
    A = inputs.gaussian(m * nb, n * nb, seed=810)
    recs = lib_list(m, n, a, p, low, high)
    if which == "bbd10":
        assert all(r[3] == 0 for r in recs)  # only TS kernels
    else:
        assert {r[4] for r in recs} == {0, 1}  # TS domains and the binary tree over their heads
    Fo, Fg = factor_fp64(A, nb, ib, recs)
    compare_fp64(Fo, Fg, A)


# ---------------------------------------------------- priority policies --

@pytest.mark.parametrize("domino", [False, True])
def test_priority_policy_0_matches_oracle_and_default_bitwise(domino):
    nb, ib, m, n = 32, 8, 12, 4
    A = inputs.gaussian(m * nb, n * nb, seed=820)
    recs = lib_list(m, n, 2, 3, GREEDY, FIBONACCI, domino=domino)
    Ad = torch.from_numpy(A).cuda()
    F1 = hqr.geqrf(Ad, nb, ib, recs)
    hqr.set_priority_policy(0)
    try:
        F0 = hqr.geqrf(Ad, nb, ib, recs)
    finally:
        hqr.set_priority_policy(1)
    assert torch.equal(F0.tiles(), F1.tiles())
    Fo = tile_qr(A, nb, ib, recs)
    compare_fp64(Fo, F0, A)
