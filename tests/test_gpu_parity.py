"""GPU parity of the FP64 tile QR against the CPU oracle (same list, same
seeded inputs), through the C ABI.

Tolerances: the factor R within max|dR| / ||A||_F <= 1e-11; the Householder
vectors (|v| <= 1 by construction) and T factors within 1e-10 absolute; Q
within 1e-12. Integer outputs (lists) are compared bit-exactly elsewhere.
"""
import itertools

import numpy as np
import pytest

from oracle.elim_list import BINARY, FIBONACCI, FLAT, GREEDY, hqr_elim_list
from oracle.householder import householder_qr
from oracle.lstsq import lstsq, lstsq_unblocked
from oracle.tile_qr import apply_q as o_apply_q
from oracle.tile_qr import explicit_q, tile_qr
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


def pad(A, nb):
    M, N = A.shape
    Mp, Np = -(-M // nb) * nb, -(-N // nb) * nb
    P = np.zeros((Mp, Np))
    P[:M, :N] = A
    return P


def run_both(A, nb, ib, recs):
    Fo = tile_qr(pad(A, nb), nb, ib, recs)
    Fg = hqr.geqrf(torch.from_numpy(np.ascontiguousarray(A)).cuda(), nb, ib, recs)
    return Fo, Fg


def compare_factors(Fo, Fg, A):
    nrm = np.linalg.norm(A)
    tiles = Fg.tiles().cpu().numpy()
    N = Fg.N
    Rg = Fg.R().cpu().numpy()
    Ro = np.triu(Fo.A[:N, :N])
    assert np.max(np.abs(Rg - Ro)) <= R_TOL * nrm
    # every stored V / R entry of every tile
    d = np.abs(tiles - Fo.A)
    assert np.max(d) <= max(VT_TOL, R_TOL * nrm), np.unravel_index(np.argmax(d), d.shape)
    T = Fg.T().cpu().numpy()
    for (r, k), To in Fo.Tg.items():
        assert np.max(np.abs(T[k, r, 0].T - To)) <= VT_TOL, ("Tg", r, k)
    for (i, k), To in Fo.Tk.items():
        assert np.max(np.abs(T[k, i, 1].T - To)) <= VT_TOL, ("Tk", i, k)


@pytest.mark.parametrize("nb,ib", [(16, 4), (64, 16), (256, 32)])
@pytest.mark.parametrize("shape,a,p", [((1, 1), 1, 1), ((2, 1), 2, 1), ((2, 1), 1, 1), ((2, 2), 2, 1),
                                       ((2, 2), 1, 1), ((3, 2), 1, 2)])
def test_each_kernel(nb, ib, shape, a, p):
    # (1,1): GEQRT; (2,1) a=2: +TSQRT; a=1: +TTQRT; (2,2): +UNMQR and TSMQR / TTMQR
    m, n = shape
    A = inputs.gaussian(m * nb, n * nb, seed=100 + nb + 7 * m + n + a)
    recs = hqr_elim_list(m, n, a, p, FLAT, FLAT)
    Fo, Fg = run_both(A, nb, ib, recs)
    compare_factors(Fo, Fg, A)


@pytest.mark.parametrize("low,high", list(itertools.product(TREES, TREES)))
def test_all_tree_pairs(low, high):
    nb, ib, m, n = 16, 4, 9, 4
    A = inputs.gaussian(m * nb, n * nb, seed=3)
    for a, p in ((1, 1), (2, 3), (4, 2), (m, 1)):
        recs = hqr_elim_list(m, n, a, p, low, high)
        Fo, Fg = run_both(A, nb, ib, recs)
        compare_factors(Fo, Fg, A)


def test_square_flat_ts_c1_shape():
    # 512 x 512, nb = 64, ib = 16, flat TS domains a = 8, p = 1: R, T and Q I
    nb, ib = 64, 16
    A = inputs.gaussian(512, 512, seed=1)
    recs = hqr_elim_list(8, 8, 8, 1, FLAT, FLAT)
    Fo, Fg = run_both(A, nb, ib, recs)
    compare_factors(Fo, Fg, A)
    I = torch.eye(512, dtype=torch.float64, device="cuda").t().contiguous().t()
    Qg = Fg.apply_q(I.clone(), trans=False).cpu().numpy()
    Qo = explicit_q(Fo)
    assert np.max(np.abs(Qg - Qo)) <= 1e-12
    assert np.linalg.norm(Qg.T @ Qg - np.eye(512)) <= 1e-12
    Rg = Fg.R().cpu().numpy()
    assert np.linalg.norm(A - Qg @ Rg) / np.linalg.norm(A) <= 1e-13


def test_apply_q_both_ways():
    nb, ib, m, n = 32, 8, 6, 3
    A = inputs.gaussian(m * nb, n * nb, seed=5)
    recs = hqr_elim_list(m, n, 2, 2, GREEDY, FIBONACCI)
    Fo, Fg = run_both(A, nb, ib, recs)
    B = inputs.gaussian(m * nb, 37, seed=6)  # ragged number of columns
    for trans in (True, False):
        Bg = torch.from_numpy(B.copy()).cuda()
        out = Fg.apply_q(Bg, trans=trans).cpu().numpy()
        ref = o_apply_q(Fo, B, trans=trans)
        assert np.max(np.abs(out - ref)) <= 1e-12 * np.linalg.norm(B)
    # Q^T A = [R; 0]
    QtA = Fg.apply_q(torch.from_numpy(A.copy()).cuda(), trans=True).cpu().numpy()
    R = Fg.R().cpu().numpy()
    assert np.max(np.abs(QtA[:n * nb] - R)) <= 1e-12 * np.linalg.norm(A)
    assert np.max(np.abs(QtA[n * nb:])) <= 1e-12 * np.linalg.norm(A)


def test_gels_matches_oracle():
    nb, ib, m, n = 32, 8, 8, 3
    A = inputs.gaussian(m * nb, n * nb, seed=7)
    b = inputs.gaussian(m * nb, 2, seed=8)
    recs = hqr_elim_list(m, n, 2, 2, GREEDY, FIBONACCI)
    x = hqr.gels_qr(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), nb, ib, recs).cpu().numpy()
    for c in range(2):
        xo, _ = lstsq(A, b[:, c], nb, ib, recs)
        kappa = np.linalg.cond(A)
        assert np.linalg.norm(x[:, c] - xo) / np.linalg.norm(xo) <= 1e-15 * kappa * kappa * 10 + 1e-13


@pytest.mark.parametrize("M,N,nb,ib", [(100, 37, 16, 4), (65, 65, 32, 8), (300, 20, 64, 16), (17, 3, 8, 2)])
def test_ragged_shapes(M, N, nb, ib):
    A = inputs.gaussian(M, N, seed=M + N)
    m, n = -(-M // nb), -(-N // nb)
    recs = hqr_elim_list(m, n, 2, 2, GREEDY, BINARY)
    Fo, Fg = run_both(A, nb, ib, recs)
    compare_factors(Fo, Fg, pad(A, nb))
    Ru = householder_qr(A)[0]
    Rg = Fg.R().cpu().numpy()
    s = np.sign(np.diag(Rg)) * np.sign(np.diag(Ru))
    assert np.max(np.abs(Rg * s[:, None] - Ru)) <= 1e-12 * np.linalg.norm(A)


def test_triangular_input_is_exact():
    nb, ib, m = 16, 4, 5
    A = np.triu(inputs.gaussian(m * nb, m * nb, seed=9))
    for low, high, a, p in ((FLAT, FLAT, 1, 1), (GREEDY, FIBONACCI, 2, 2), (BINARY, GREEDY, 5, 1)):
        Fg = hqr.geqrf(torch.from_numpy(A).cuda(), nb, ib, hqr_elim_list(m, m, a, p, low, high))
        assert np.array_equal(Fg.R().cpu().numpy(), A)


def test_zero_matrix_and_single_tile():
    Z = np.zeros((40, 24))
    Fg = hqr.geqrf(torch.from_numpy(Z).cuda(), 8, 4)
    assert not Fg.R().cpu().numpy().any()
    A = inputs.gaussian(8, 8, seed=10)
    Fg = hqr.geqrf(torch.from_numpy(A).cuda(), 8, 2)
    Ro = np.triu(tile_qr(A, 8, 2, hqr_elim_list(1, 1, 1, 1, FLAT, FLAT)).A)
    assert np.max(np.abs(Fg.R().cpu().numpy() - Ro)) <= 1e-13


def test_refactor_is_bitwise_deterministic():
    nb, ib, m, n = 32, 8, 12, 4
    A = torch.from_numpy(inputs.gaussian(m * nb, n * nb, seed=11)).cuda()
    Fg = hqr.geqrf(A, nb, ib, hqr_elim_list(m, n, 2, 3, GREEDY, FIBONACCI))
    t1 = Fg.tiles()
    for _ in range(3):
        Fg.refactor(A)
        assert torch.equal(Fg.tiles(), t1)


def test_invalid_list_rejected():
    recs = hqr_elim_list(4, 2, 1, 1, FLAT, FLAT)
    bad = recs[:-1]
    A = torch.from_numpy(inputs.gaussian(32, 16, seed=12)).cuda()
    with pytest.raises(hqr.HQRError) as e:
        hqr.geqrf(A, 8, 4, bad)
    assert e.value.status == -8


def test_device_wait_times_out_instead_of_hanging():
    # a task given an input that never arrives: the persistent kernel must
    # give up after the time limit, report HQR_ERR_TIMEOUT and leave the
    # context usable
    nb, ib, m, n = 16, 4, 4, 2
    A = torch.from_numpy(inputs.gaussian(m * nb, n * nb, seed=13)).cuda()
    recs = hqr_elim_list(m, n, 1, 1, FLAT, FLAT)
    Fg = hqr.geqrf(A, nb, ib, recs)
    good = Fg.tiles().clone()
    hqr.set_timeout_ms(300)
    try:
        Fg.debug_block_task(Fg.ntasks // 2, 1)
        with pytest.raises(hqr.HQRError) as e:
            Fg.refactor(A)
        assert e.value.status == hqr.ERR_TIMEOUT
        Fg.debug_block_task(Fg.ntasks // 2, 0)
    finally:
        hqr.set_timeout_ms(20000)
    Fg.refactor(A)
    assert torch.equal(Fg.tiles(), good)


# ---------------------------------------------------------------- FP32 --
# FP32 storage and arithmetic against the FP64 oracle run on the same
# (float-rounded) input: R within 5e-6 ||A||_F, Q^T B within 5e-6 ||B||.

@pytest.mark.parametrize("nb,ib", [(16, 4), (64, 16), (256, 32)])
@pytest.mark.parametrize("shape,a,p", [((1, 1), 1, 1), ((2, 1), 2, 1), ((2, 1), 1, 1), ((2, 2), 2, 1),
                                       ((2, 2), 1, 1), ((3, 2), 1, 2)])
def test_each_kernel_fp32(nb, ib, shape, a, p):
    m, n = shape
    A = inputs.gaussian(m * nb, n * nb, seed=300 + nb + 7 * m + n + a).astype(np.float32)
    recs = hqr_elim_list(m, n, a, p, FLAT, FLAT)
    Fo = tile_qr(A.astype(np.float64), nb, ib, recs)
    Fg = hqr.geqrf(torch.from_numpy(np.ascontiguousarray(A)).cuda(), nb, ib, recs)
    Rg = Fg.R().cpu().numpy().astype(np.float64)
    nrm = np.linalg.norm(A.astype(np.float64))
    assert np.max(np.abs(Rg - Fo.R())) <= 5e-6 * nrm
    tiles = Fg.tiles().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(tiles - Fo.A)) <= 5e-5 * max(1.0, nrm)


@pytest.mark.parametrize("low,high", [(FLAT, FLAT), (GREEDY, FIBONACCI), (BINARY, GREEDY), (FIBONACCI, BINARY)])
def test_tree_pairs_fp32_and_apply_q(low, high):
    nb, ib, m, n = 32, 8, 9, 4
    A = inputs.gaussian(m * nb, n * nb, seed=41).astype(np.float32)
    recs = hqr_elim_list(m, n, 2, 3, low, high)
    Fo = tile_qr(A.astype(np.float64), nb, ib, recs)
    Fg = hqr.geqrf(torch.from_numpy(A).cuda(), nb, ib, recs)
    nrm = np.linalg.norm(A.astype(np.float64))
    assert np.max(np.abs(Fg.R().cpu().numpy() - Fo.R())) <= 5e-6 * nrm
    B = inputs.gaussian(m * nb, 5, seed=42).astype(np.float32)
    for trans in (True, False):
        out = Fg.apply_q(torch.from_numpy(B.copy()).cuda(), trans=trans).cpu().numpy()
        ref = o_apply_q(Fo, B.astype(np.float64), trans=trans)
        assert np.max(np.abs(out - ref)) <= 5e-6 * np.linalg.norm(B.astype(np.float64))


# ------------------------------------------------------- split panels --
# CUDA-core panels of tiles with nb >= 64 run as one task per ib block plus
# the updates of the panel's own trailing columns. Same tolerances as whole
# panels; R also against a whole-panel run (split turned off).

@pytest.mark.parametrize("low,high,a,p,ib", [(FLAT, FLAT, 4, 1, 16), (GREEDY, FIBONACCI, 2, 2, 16),
                                             (BINARY, GREEDY, 1, 3, 16), (GREEDY, GREEDY, 2, 1, 8)])
def test_split_panels_fp64(low, high, a, p, ib):
    """ib = 8: blocks narrower than the 16-column update slabs (a block's trailing work starts
    inside its own slab)."""
    nb, m, n = 64, 7, 4
    A = inputs.gaussian(m * nb, n * nb - 3, seed=61 + a)  # ragged last tile column
    recs = hqr_elim_list(m, n, a, p, low, high)
    Fo, Fs = run_both(A, nb, ib, recs)
    compare_factors(Fo, Fs, pad(A, nb))
    B = inputs.gaussian(A.shape[0], 3, seed=62)
    for trans in (True, False):
        out = Fs.apply_q(torch.from_numpy(B.copy()).cuda(), trans=trans).cpu().numpy()
        ref = o_apply_q(Fo, B, trans=trans)
        assert np.max(np.abs(out - ref)) <= 1e-12 * np.linalg.norm(B)
    hqr.set_panel_split(0)
    try:
        Fw = hqr.geqrf(torch.from_numpy(np.ascontiguousarray(A)).cuda(), nb, ib, recs)
    finally:
        hqr.set_panel_split(64)
    assert np.max(np.abs(Fs.R().cpu().numpy() - Fw.R().cpu().numpy())) <= 1e-13 * np.linalg.norm(A)


@pytest.mark.parametrize("nb,ib", [(128, 16), (128, 32), (256, 32)])
def test_split_panels_fp32(nb, ib):
    """FP32 panels are split where a block spans whole update slabs (here slabs of 16)."""
    m, n = 6, 3
    A = inputs.gaussian(m * nb, n * nb, seed=63 + ib).astype(np.float32)
    recs = hqr_elim_list(m, n, 2, 2, GREEDY, FIBONACCI)
    Fo = tile_qr(A.astype(np.float64), nb, ib, recs)
    hqr.set_slab_widths(16, 0, 0)
    try:
        Fg = hqr.geqrf(torch.from_numpy(A).cuda(), nb, ib, recs)
    finally:
        hqr.set_slab_widths(0, 0, 0)
    nrm = np.linalg.norm(A.astype(np.float64))
    assert np.max(np.abs(Fg.R().cpu().numpy().astype(np.float64) - Fo.R())) <= 5e-6 * nrm
    tiles = Fg.tiles().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(tiles - Fo.A)) <= 5e-5 * max(1.0, nrm)


def test_split_panels_least_squares_plan():
    """A least-squares plan whose panels are split: x equals the FP64 oracle's."""
    nb, ib = 64, 16
    A = inputs.gaussian(700, 190, seed=64)
    b = inputs.rng(64, 1).standard_normal(700)
    x = torch.zeros(190, dtype=torch.float64, device="cuda")
    plan = hqr.LSPlan([(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), x)], refine_iters=0,
                      configs=[hqr.tile_config(nb, ib, 2, 2, "greedy", "fibonacci")])
    plan.run()
    assert plan.status() == 0
    xo = lstsq_unblocked(A, b)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-12
