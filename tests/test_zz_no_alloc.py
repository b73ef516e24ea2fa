"""The allocation-free entry point hqr_geqrf_r_noalloc, called through the C
ABI, against the regular hqr_geqrf on two calls in a row.

It exists for callers that may not allocate memory during the call: their
device memory belongs to another allocator's pool, or cudaMalloc's implicit
device synchronization is not acceptable where they run. Its scratch is one
static device array shared by all calls, so the second call here also checks
that nothing left over from the first call leaks into its result.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
from paper_1110_1553_gb300 import hqr, inputs  # noqa: E402

pytestmark = pytest.mark.gpu
R_TOL = 1e-11  # max|dR| / ||A||_F, as the other parity tests


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()


def test_noalloc_matches_geqrf_on_two_calls():
    nb, ib = 64, 16
    for call, (M, N, seed, a, p) in enumerate([(512, 256, 31, 2, 2), (300, 200, 32, 1, 3)]):
        m, n = -(-M // nb), -(-N // nb)
        recs = hqr.elim_list(m, n, a, p, "greedy", "fibonacci")
        A = torch.from_numpy(inputs.gaussian(M, N, seed=seed)).cuda()
        R = hqr.empty_colmajor(N, N)
        R.fill_(np.nan)
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = hqr.geqrf_r_noalloc(A, nb, ib, recs, R)
        free_after = torch.cuda.mem_get_info()[0]
        assert st == 0, st
        if call == 1:
            # after the one-time set-up of the first call, no device memory moves
            assert free_after == free_before
        Rref = hqr.geqrf(A, nb, ib, recs).R()
        err = ((R - Rref).abs().max() / torch.linalg.norm(A)).item()
        assert err <= R_TOL, (call, err)


def test_noalloc_rejects_oversized_problems():
    nb, ib = 64, 16
    M, N = 65 * nb, nb  # 65 tile rows: over the 64-row limit
    recs = hqr.elim_list(65, 1, 1, 1, "flat", "flat")
    A = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    R = hqr.empty_colmajor(N, N)
    assert hqr.geqrf_r_noalloc(A, nb, ib, recs, R) == hqr.ERR_TOO_LARGE
    recs = hqr.elim_list(2, 1, 1, 1, "flat", "flat")
    A = torch.zeros((256, 128), dtype=torch.float64, device="cuda")
    R = hqr.empty_colmajor(128, 128)
    assert hqr.geqrf_r_noalloc(A, 128, 16, recs, R) == hqr.ERR_TOO_LARGE  # nb > 64


def test_noalloc_layout_over_the_scratch_size_then_a_normal_call():
    # 64 x 4 tiles of 64 with ib = 32: within the tile-count limits, but the
    # tiles (8 MiB) and T factors (8 MiB) with the task graph exceed the
    # 16 MiB scratch: rejected before any device work
    nb, ib = 64, 32
    M, N = 64 * nb, 4 * nb
    recs = hqr.elim_list(64, 4, 4, 1, "greedy", "greedy")
    A = torch.zeros((M, N), dtype=torch.float64, device="cuda")
    R = hqr.empty_colmajor(N, N)
    assert hqr.geqrf_r_noalloc(A, nb, ib, recs, R) == hqr.ERR_TOO_LARGE
    # the next call that fits still gives the regular factorization's R
    M, N = 512, 256
    recs = hqr.elim_list(M // nb, N // nb, 2, 2, "greedy", "fibonacci")
    A = torch.from_numpy(inputs.gaussian(M, N, seed=33)).cuda()
    R = hqr.empty_colmajor(N, N)
    R.fill_(np.nan)
    assert hqr.geqrf_r_noalloc(A, nb, ib, recs, R) == 0
    Rref = hqr.geqrf(A, nb, ib, recs).R()
    assert ((R - Rref).abs().max() / torch.linalg.norm(A)).item() <= R_TOL


def test_noalloc_refuses_a_capturing_stream():
    """The call stages its task graph from host memory and synchronizes its
    stream, so it cannot be captured: on a stream under capture it returns -11
    (the stream argument) before any work, and the capture stays usable."""
    import ctypes
    nb, ib, M, N = 64, 16, 256, 128
    recs = hqr.elim_list(M // nb, N // nb, 2, 1, "greedy", "greedy")
    arr = np.ascontiguousarray(hqr.to_array(recs), dtype=hqr.ELIM_DTYPE)
    A = torch.from_numpy(inputs.gaussian(M, N, seed=33)).cuda()
    R = hqr.empty_colmajor(N, N)
    lib = hqr.load()
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        st = lib.hqr_geqrf_r_noalloc(ctypes.c_void_p(A.data_ptr()), M, N, M, nb, ib, ctypes.c_void_p(arr.ctypes.data),
                                     len(arr), ctypes.c_void_p(R.data_ptr()), N, ctypes.c_void_p(s.cuda_stream))
        R.add_(0.0)  # the capture goes on after the refused call
    assert st == -11
    torch.cuda.synchronize()
    assert hqr.geqrf_r_noalloc(A, nb, ib, recs, R) == 0  # and a normal call after it works
