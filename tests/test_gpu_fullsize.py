"""Parity at the full tall-skinny size in the benchmark's launch configuration
(131072 x 2048 FP64, nb = 256, ib = 32, a = 4, p = 16, Greedy / Fibonacci).

The oracle cannot factor the whole matrix in seconds, so:
* the first tile column is compared element by element with the oracle's
  tile QR of A[:, :256] under the same list (panel 0 of the list does not
  depend on n, and R[:256, :256] depends only on A[:, :256]);
* properties that hold at any size are checked on the whole result: column
  norms of R equal those of A, sampled entries of R^T R equal those of A^T A,
  Q^T (A x) = [R x; 0] and ||Q^T b|| = ||b|| for random x and b.
"""
import numpy as np
import pytest

from oracle.elim_list import FIBONACCI, GREEDY, hqr_elim_list
from oracle.tile_qr import tile_qr
from paper_1110_1553_gb300 import inputs

torch = pytest.importorskip("torch")
hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")

pytestmark = pytest.mark.gpu
M, N, NB, IB, A_, P_ = 131072, 2048, 256, 32, 4, 16


@pytest.fixture(scope="module")
def fullsize():
    from paper_1110_1553_gb300 import _build
    _build.build()
    A = inputs.gaussian(M, N, seed=21)
    recs = hqr.elim_list(M // NB, N // NB, A_, P_, "greedy", "fibonacci")
    Ad = torch.from_numpy(A.T.copy()).cuda().t()  # column-major on the device
    F = hqr.geqrf(Ad, NB, IB, recs)
    return A, Ad, F


def test_first_tile_column_matches_oracle(fullsize):
    A, Ad, F = fullsize
    recs0 = hqr_elim_list(M // NB, 1, A_, P_, GREEDY, FIBONACCI)
    full = hqr.as_records(hqr.elim_list(M // NB, N // NB, A_, P_, "greedy", "fibonacci"))
    assert [r for r in full if r[0] == 0] == [tuple(r) for r in recs0]
    Fo = tile_qr(A[:, :NB], NB, IB, recs0)
    Rg = F.R()[:NB, :NB].cpu().numpy()
    assert np.max(np.abs(Rg - Fo.R())) <= 1e-11 * np.linalg.norm(A[:, :NB])


def test_properties_at_full_size(fullsize):
    A, Ad, F = fullsize
    R = F.R()
    cn = (R.norm(dim=0) - Ad.norm(dim=0)).abs() / Ad.norm(dim=0)
    assert cn.max().item() <= 1e-13
    rng = np.random.default_rng(0)
    idx = rng.integers(0, N, size=(300, 2))
    Rc = R.cpu().numpy()
    nrmA = np.linalg.norm(A)
    for i, j in idx:
        g = A[:, i] @ A[:, j]
        h = Rc[:, i] @ Rc[:, j]
        assert abs(g - h) <= 1e-12 * nrmA * nrmA / N
    x = torch.randn(N, 2, dtype=torch.float64, device="cuda")
    y = (Ad @ x).t().contiguous().t()
    F.apply_q(y, trans=True)
    rx = R @ x
    assert ((y[:N] - rx).abs().max() / rx.abs().max()).item() <= 1e-12
    assert (y[N:].abs().max() / rx.abs().max()).item() <= 1e-12
    b = torch.randn(M, 2, dtype=torch.float64, device="cuda").t().contiguous().t()
    nb0 = b.norm(dim=0)
    F.apply_q(b, trans=True)
    assert ((b.norm(dim=0) - nb0).abs() / nb0).max().item() <= 1e-13


# ------------------------------------------------- with the coupling level --
# The same workload with the coupling ("domino") level of Sec. 4.2. Panel 0
# has no coupled rows, so R[:512, :512] (panels 0 and 1 on the first two tile
# columns) is compared with the oracle; properties that hold at any size are
# checked on the whole result.

@pytest.fixture(scope="module")
def fullsize_domino(fullsize):
    A, Ad, _ = fullsize
    recs = hqr.elim_list(M // NB, N // NB, A_, P_, "greedy", "fibonacci", domino=True)
    assert any(int(r["level"]) == 2 for r in recs)
    return A, Ad, hqr.geqrf(Ad, NB, IB, recs)


def test_domino_first_two_tile_columns_match_oracle(fullsize_domino):
    A, Ad, F = fullsize_domino
    recs2 = hqr_elim_list(M // NB, 2, A_, P_, GREEDY, FIBONACCI, domino=True)
    full = hqr.as_records(hqr.elim_list(M // NB, N // NB, A_, P_, "greedy", "fibonacci", domino=True))
    assert [r for r in full if r[0] < 2] == [tuple(r) for r in recs2]
    Fo = tile_qr(A[:, :2 * NB], NB, IB, recs2)
    Rg = F.R()[:2 * NB, :2 * NB].cpu().numpy()
    assert np.max(np.abs(Rg - Fo.R())) <= 1e-11 * np.linalg.norm(A[:, :2 * NB])


def test_domino_properties_at_full_size(fullsize_domino):
    A, Ad, F = fullsize_domino
    R = F.R()
    cn = (R.norm(dim=0) - Ad.norm(dim=0)).abs() / Ad.norm(dim=0)
    assert cn.max().item() <= 1e-13
    x = torch.randn(N, 2, dtype=torch.float64, device="cuda")
    y = (Ad @ x).t().contiguous().t()
    F.apply_q(y, trans=True)
    rx = R @ x
    assert ((y[:N] - rx).abs().max() / rx.abs().max()).item() <= 1e-12
    assert (y[N:].abs().max() / rx.abs().max()).item() <= 1e-12
