"""GPU parity of the tensor-core FP32 path (HQR_FP32_BF16X3: tiles of 128,
register-resident unblocked panels with one full T per tile, tcgen05
updates on BF16x3-split operands) against the FP64 oracle run on the same
float-rounded input, with the same elimination list.

Tolerances: R within 5e-6 ||A||_F and every stored V / R entry within 5e-5
(as for the FP32 CUDA-core path: the split products keep FP32 accuracy); T (full 128 x 128, upper triangular) within 3e-4
(the 128-wide T accumulates the FP32 perturbations of V through its merges);
Q and Q^T applied to B within 5e-6 ||B||; least-squares solutions after
corrected semi-normal-equation refinement within 1e-12 relative.
"""
import numpy as np
import pytest

from oracle.elim_list import BINARY, FIBONACCI, FLAT, GREEDY, hqr_elim_list
from oracle.lstsq import lstsq_unblocked
from oracle.tile_qr import apply_q as o_apply_q
from oracle.tile_qr import tile_qr
from paper_1110_1553_gb300 import inputs, workloads

torch = pytest.importorskip("torch")
hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")

pytestmark = pytest.mark.gpu
NB = 128


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()
    hqr.set_timeout_ms(20000)


def pad(A, nb):
    M, N = A.shape
    P = np.zeros((-(-M // nb) * nb, -(-N // nb) * nb))
    P[:M, :N] = A
    return P


def factor(A32, recs):
    Fo = tile_qr(pad(A32.astype(np.float64), NB), NB, NB, recs)
    Fg = hqr.geqrf(torch.from_numpy(np.ascontiguousarray(A32)).cuda(), NB, NB, recs, tensor=True)
    return Fo, Fg


def check_factors(Fo, Fg, A32):
    nrm = np.linalg.norm(A32.astype(np.float64))
    N = Fg.N
    Rg = Fg.R().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Rg - np.triu(Fo.A[:N, :N]))) <= 5e-6 * nrm
    tiles = Fg.tiles().cpu().numpy().astype(np.float64)
    d = np.abs(tiles - Fo.A)
    assert np.max(d) <= 5e-5 * max(1.0, nrm), np.unravel_index(np.argmax(d), d.shape)
    T = Fg.T().cpu().numpy().astype(np.float64)
    for (r, k), To in Fo.Tg.items():
        assert np.max(np.abs(T[k, r, 0].T - To)) <= 3e-4, ("Tg", r, k)
    for (i, k), To in Fo.Tk.items():
        assert np.max(np.abs(T[k, i, 1].T - To)) <= 3e-4, ("Tk", i, k)


@pytest.mark.parametrize("shape,a,p", [((1, 1), 1, 1), ((2, 1), 2, 1), ((2, 1), 1, 1), ((2, 2), 2, 1),
                                       ((2, 2), 1, 1), ((3, 2), 1, 2), ((4, 3), 2, 1)])
def test_each_kernel_tc(shape, a, p):
    """GEQRT alone, TSQRT (a = 2), TTQRT (a = 1) with their updates, and a
    mix of both over two and three tile columns."""
    m, n = shape
    A = inputs.gaussian(m * NB, n * NB, seed=700 + 7 * m + n + a).astype(np.float32)
    recs = hqr_elim_list(m, n, a, p, FLAT, FLAT)
    Fo, Fg = factor(A, recs)
    check_factors(Fo, Fg, A)


@pytest.mark.parametrize("low,high", [(GREEDY, FIBONACCI), (BINARY, GREEDY), (FIBONACCI, BINARY)])
def test_tree_pairs_tc_and_apply_q(low, high):
    m, n = 6, 3
    A = inputs.gaussian(m * NB, n * NB, seed=710).astype(np.float32)
    recs = hqr_elim_list(m, n, 2, 2, low, high)
    Fo, Fg = factor(A, recs)
    nrm = np.linalg.norm(A.astype(np.float64))
    assert np.max(np.abs(Fg.R().cpu().numpy() - Fo.R())) <= 5e-6 * nrm
    B = inputs.gaussian(m * NB, 21, seed=711).astype(np.float32)
    for trans in (True, False):
        out = Fg.apply_q(torch.from_numpy(B.copy()).cuda(), trans=trans).cpu().numpy()
        ref = o_apply_q(Fo, B.astype(np.float64), trans=trans)
        assert np.max(np.abs(out - ref)) <= 5e-6 * np.linalg.norm(B.astype(np.float64)), trans


@pytest.mark.parametrize("M,N", [(1000, 300), (130, 129), (700, 128)])
def test_ragged_tc(M, N):
    """Zero padding to whole tiles: padded rows and columns stay zero and the
    factor of the true part matches."""
    A = inputs.gaussian(M, N, seed=720 + M).astype(np.float32)
    m, n = -(-M // NB), -(-N // NB)
    recs = hqr_elim_list(m, n, 2, 1, GREEDY, GREEDY)
    Fo, Fg = factor(A, recs)
    nrm = np.linalg.norm(A.astype(np.float64))
    assert np.max(np.abs(Fg.R().cpu().numpy() - np.triu(Fo.A[:N, :N]))) <= 5e-6 * nrm


def test_triangular_and_zero_inputs_tc():
    """An upper-triangular matrix is its own R (identity reflectors: every
    column below the diagonal is zero), and a zero matrix gives R = 0."""
    U = np.triu(inputs.gaussian(2 * NB, 2 * NB, seed=730)).astype(np.float32)
    recs = hqr_elim_list(2, 2, 1, 1, FLAT, FLAT)
    Fg = hqr.geqrf(torch.from_numpy(U).cuda(), NB, NB, recs, tensor=True)
    assert np.array_equal(Fg.R().cpu().numpy(), U)
    Z = np.zeros((3 * NB, NB), dtype=np.float32)
    Fz = hqr.geqrf(torch.from_numpy(Z).cuda(), NB, NB, hqr_elim_list(3, 1, 2, 1, FLAT, FLAT), tensor=True)
    assert not np.any(Fz.R().cpu().numpy())


def test_tc_matches_cuda_core_fp32():
    """The tensor-core factor and the FP32 CUDA-core factor of the same
    input agree to FP32 rounding (same list, different arithmetic order)."""
    m, n = 8, 4
    A = inputs.gaussian(m * NB, n * NB, seed=740).astype(np.float32)
    recs = hqr_elim_list(m, n, 4, 2, GREEDY, FIBONACCI)
    At = torch.from_numpy(A).cuda()
    Rt = hqr.geqrf(At, NB, NB, recs, tensor=True).R().cpu().numpy().astype(np.float64)
    Rs = hqr.geqrf(At, NB, 16, recs).R().cpu().numpy().astype(np.float64)
    assert np.max(np.abs(Rt - Rs)) <= 5e-6 * np.linalg.norm(A.astype(np.float64))


def test_refactor_is_bitwise_deterministic_tc():
    m, n = 5, 3
    A = torch.from_numpy(inputs.gaussian(m * NB, n * NB, seed=750).astype(np.float32)).cuda()
    F = hqr.geqrf(A, NB, NB, hqr_elim_list(m, n, 2, 2, GREEDY, GREEDY), tensor=True)
    first = F.tiles().clone()
    for _ in range(3):
        F.refactor(A)
        assert torch.equal(F.tiles(), first)


def to_dev(A, b, N):
    Ad = torch.from_numpy(np.asfortranarray(A).T.copy()).cuda().t()
    return Ad, torch.from_numpy(b).cuda(), torch.zeros(N, dtype=torch.float64, device="cuda")


def test_ls_plan_tc_matches_oracle():
    """Mixed-precision solves with tensor-core tiles (and CUDA-core tiles for
    the shapes whose default tile is smaller) in one plan, refined to the
    FP64 oracle's solution."""
    shapes = [(64, 32), (1000, 333), (2048, 256), (512, 500), (4096, 129)]
    probs, host = [], []
    for q, (M, N) in enumerate(shapes):
        A = inputs.gaussian(M, N, seed=760 + q).astype(np.float32)
        b = inputs.rng(760 + q, 1).standard_normal(M)
        host.append((A.astype(np.float64), b))
        probs.append(to_dev(A, b, N))
    cfgs = [hqr.tile_config(128, 128, 2, 1, "greedy", "greedy") if N > 64 else hqr.tile_config()
            for (M, N) in shapes]
    plan = hqr.LSPlan(probs, refine_iters=8, configs=cfgs, tensor=True)
    plan.run()
    assert plan.status() == 0
    for (A, b), (_, _, x) in zip(host, probs):
        xo = lstsq_unblocked(A, b)
        err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err <= 1e-12, err


@pytest.mark.parametrize("kappa,iters", [(1e4, 10), (1e6, 24)])
def test_ls_conditioned_tc(kappa, iters):
    """Square, conditioned as U diag(sigma) V^T with geometric sigma, at the
    accuracy goal after refinement."""
    n = 1024
    A = workloads.conditioned(torch, n, n, kappa, seed=770 + int(np.log10(kappa)))
    g = torch.Generator(device="cuda")
    g.manual_seed(771)
    xt = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    b = A.double() @ xt + 1e-8 * torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    plan = hqr.LSPlan([(A, b, x)], refine_iters=iters, configs=[hqr.tile_config(128, 128, 2, 1)], tensor=True)
    plan.run()
    assert plan.status() == 0
    xo = lstsq_unblocked(A.double().cpu().numpy(), b.cpu().numpy())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-12, err


def test_split_launch_equals_one_launch():
    """A plan with tensor-core and CUDA-core problems runs them as two
    launches side by side (hqr_set_split_launch): every x is bitwise the
    one of a single launch of the tensor-core kernel (each task's arithmetic
    does not depend on the kernel variant that runs it), also on CUDA-graph
    replay and after the SM share is rebalanced between runs."""
    shapes = [(64, 32), (300, 60), (1000, 333), (2048, 256), (200, 100), (4096, 129), (90, 90)]
    host, outs = [], {}
    for q, (M, N) in enumerate(shapes):
        A = inputs.gaussian(M, N, seed=780 + q).astype(np.float32)
        host.append((A, inputs.rng(780 + q, 1).standard_normal(M)))
    cfgs = [hqr.tile_config(128, 128, 2, 1, "greedy", "greedy") if N > 128 else hqr.tile_config(32, 16, 2, 1)
            for (M, N) in shapes]
    for split in (0, 1):
        hqr.set_split_launch(split)
        try:
            probs = [to_dev(A, b, A.shape[1]) for A, b in host]
            plan = hqr.LSPlan(probs, refine_iters=6, configs=cfgs, tensor=True)
        finally:
            hqr.set_split_launch(1)
        for _ in range(3):  # timed runs: the split plan rebalances its SM share
            plan.run()
            assert plan.status() == 0
        outs[split] = [p[2].clone() for p in probs]
        if split:
            s = torch.cuda.Stream()
            plan.capture(s)
            plan.run(s)
            assert plan.status(s) == 0
            assert all(torch.equal(p[2], x) for p, x in zip(probs, outs[1]))
    assert all(torch.equal(a, b) for a, b in zip(outs[0], outs[1]))
    for (A, b), x in zip(host, outs[1]):
        xo = lstsq_unblocked(A.astype(np.float64), b)
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-12
