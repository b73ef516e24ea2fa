"""hqr_gels and tolerance-stopped least-squares plans, through the C ABI,
against the CPU oracle (the paper's problem of Sec. 2: min ||b - A x|| by
the tile QR, Q^T applied by replaying the trees, Sec. 5.1).

The oracle solution is the FP64 tile QR plus Dot2-compensated
augmented-system refinement, accurate to about u (1 + kappa u); for the
mixed-precision solves the oracle factors the FP32 matrix widened exactly to
FP64. Tolerance: x within 1e-12 relative (2-norm) of the oracle's, for
kappa up to 1e6.
"""
import numpy as np
import pytest

from oracle.elim_list import GREEDY, hqr_elim_list
from oracle.lstsq import lstsq, lstsq_unblocked
from paper_1110_1553_gb300 import inputs, workloads

torch = pytest.importorskip("torch")
hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")

pytestmark = pytest.mark.gpu
X_TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()
    hqr.set_timeout_ms(20000)


def rel(x, y):
    return float(np.linalg.norm(x - y) / np.linalg.norm(y))


def test_gels_fp64_large_residual_matches_oracle():
    M, N = 700, 190  # ragged: not multiples of the tile size
    A = inputs.gaussian(M, N, seed=901)
    b = inputs.rng(901, 1).standard_normal(M)
    x, st, info = hqr.gels(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), tol=1e-14, max_iter=10)
    assert st == hqr.SUCCESS, (st, info)
    assert info["converged"] == 1 and 1 <= info["iters"] <= 10
    assert 0 <= info["rel_correction"] <= 1e-14
    xo = lstsq_unblocked(A, b)
    assert rel(x.cpu().numpy(), xo) <= X_TOL
    # a large-residual problem: b - A x is not small, A^T (b - A x) is
    assert info["normal_residual"] <= 1e-13
    assert info["singular_index"] == -1


def test_gels_fp64_plain_qr_solve():
    M, N = 512, 320
    A = inputs.gaussian(M, N, seed=902)
    xt = inputs.rng(902, 1).standard_normal(N)
    b = A @ xt
    x, st, info = hqr.gels(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), tol=0.0, max_iter=0)
    assert st == hqr.SUCCESS
    assert info["iters"] == 0 and info["converged"] == 1 and info["rel_correction"] == -1
    assert rel(x.cpu().numpy(), lstsq_unblocked(A, b)) <= 1e-13
    assert info["backward_error"] <= 1e-14  # consistent system: b - A x at rounding level


@pytest.mark.parametrize("tensor", [True, False])
def test_gels_mixed_kappa_1e6_n4096_matches_oracle(tensor):
    """The mixed-precision solve at kappa = 1e6 (A = U diag(s) V^T, s
    geometric from 1 to 1e-6, b = A x_true + 1e-8 noise): FP32 tile QR (tiles
    of 128 on the tensor cores, or FP32 CUDA cores), FP64 refinement stopped
    at a tolerance, against the FP64 oracle solution of the same FP32 A."""
    n = 4096
    A = workloads.conditioned(torch, n, n, 1e6, seed=903, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(904)
    xt = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    b = A.double() @ xt + 1e-8 * torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    x, st, info = hqr.gels(A, b, tol=1e-12, max_iter=60, tensor=tensor)
    assert st == hqr.SUCCESS, (st, info)
    assert info["converged"] == 1 and info["rel_correction"] <= 1e-12
    A64 = A.double().cpu().numpy()
    bh = b.cpu().numpy()
    nb = 256
    xo, _ = lstsq(A64, bh, nb, 32, hqr_elim_list(n // nb, n // nb, 4, 1, GREEDY, GREEDY), refine=3)
    err = rel(x.cpu().numpy(), xo)
    assert err <= X_TOL, (err, info)
    assert info["backward_error"] <= 1e-14


def test_gels_stops_when_the_refinement_stalls():
    """A tolerance below what the FP32 R allows: the refinement stops once two
    compensated rounds in a row no longer shrink the correction, well before
    max_iter, and reports that the tolerance was not met."""
    n = 1024
    A = workloads.conditioned(torch, n, n, 1e6, seed=908, device="cuda")
    b = A.double() @ torch.randn(n, dtype=torch.float64, device="cuda")
    x, st, info = hqr.gels(A, b, tol=1e-18, max_iter=60, tensor=True)
    assert st == hqr.ERR_NOCONV
    assert info["converged"] == 0 and info["iters"] < 60
    assert info["rel_correction"] <= 1e-12  # it stalls near the attainable accuracy (~1e-13 here)
    assert info["backward_error"] <= 1e-14


def test_gels_reports_no_convergence():
    n = 1024
    A = workloads.conditioned(torch, n, n, 1e6, seed=905, device="cuda")
    b = torch.randn(n, dtype=torch.float64, device="cuda")
    x, st, info = hqr.gels(A, b, tol=1e-14, max_iter=3, tensor=True)
    assert st == hqr.ERR_NOCONV
    assert info["iters"] == 3 and info["converged"] == 0 and info["rel_correction"] > 1e-14


@pytest.mark.parametrize("max_iter", [0, 4])
def test_gels_singular_reports_the_column(max_iter):
    M, N, j = 300, 100, 37
    A = inputs.gaussian(M, N, seed=906)
    A[:, j] = 0.0  # R(j, j) is then an exact zero (identity reflector on a zero column)
    b = inputs.rng(906, 1).standard_normal(M)
    x, st, info = hqr.gels(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), tol=1e-14, max_iter=max_iter)
    assert st == hqr.ERR_SINGULAR
    assert info["singular_index"] == j


def test_gels_argument_errors():
    A = torch.zeros((8, 4), dtype=torch.float64, device="cuda")
    b = torch.zeros(8, dtype=torch.float64, device="cuda")
    with pytest.raises(hqr.HQRError) as e:
        hqr.gels(A, b, tol=-1.0)
    assert e.value.status == -8
    with pytest.raises(hqr.HQRError) as e:
        hqr.gels(A, b, max_iter=65)
    assert e.value.status == -9


def test_tolerance_plan_mixed_batch_matches_oracle_and_is_deterministic():
    """One launch over problems of different conditioning: each stops at its
    own round; x matches the oracle; a second run and a CUDA-graph replay
    give the same bits and the same round counts."""
    # tall problems with a random right-hand side (a large residual: their
    # solutions' sensitivity to rounding grows like kappa tan(theta), so
    # kappa stays at 1e3 there) and a square, consistent one at kappa 1e6
    shapes = [(600, 200, 1e2), (512, 512, 1e6), (1024, 300, 1e3), (257, 129, 1e3)]
    probs, host = [], []
    g = torch.Generator(device="cuda")
    g.manual_seed(907)
    for q, (M, N, kappa) in enumerate(shapes):
        A = workloads.conditioned(torch, M, N, kappa, seed=910 + q, device="cuda")
        if M == N:
            b = A.double() @ torch.randn(N, dtype=torch.float64, device="cuda", generator=g)
        else:
            b = torch.randn(M, dtype=torch.float64, device="cuda", generator=g)
        probs.append((A, b, torch.zeros(N, dtype=torch.float64, device="cuda")))
        host.append((A.double().cpu().numpy(), b.cpu().numpy()))
    plan = hqr.LSPlan(probs, refine_iters=40, tensor=True, tol=1e-12)
    plan.run()
    assert plan.status() == 0
    iters = [plan.refine_info(q)[0] for q in range(len(shapes))]
    assert all(plan.refine_info(q)[2] for q in range(len(shapes)))
    assert iters[0] < iters[1]  # better conditioned problems stop earlier
    xs = [p[2].clone() for p in probs]
    for q, (A64, bh) in enumerate(host):
        assert rel(xs[q].cpu().numpy(), lstsq_unblocked(A64, bh)) <= X_TOL, q
    plan.run()
    assert plan.status() == 0
    assert all(torch.equal(p[2], x) for p, x in zip(probs, xs))
    s = torch.cuda.Stream()
    plan.capture(s)
    plan.run(s)
    assert plan.status(s) == 0
    assert all(torch.equal(p[2], x) for p, x in zip(probs, xs))
    assert [plan.refine_info(q, s)[0] for q in range(len(shapes))] == iters
    assert plan.correction(0, s) == plan.refine_info(0, s)[1]
