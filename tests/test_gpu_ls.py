"""Least-squares plans on the GPU (merged task graph, one persistent launch):
the FP64 QR solve and the mixed-precision solve (FP32 tile QR + FP64
corrected semi-normal equations) against the FP64 oracle, batches of uneven
shapes, "alone vs in the mix" equality, CUDA-graph replay and a singular
problem. Tolerance: x within 1e-12 relative of the oracle (the accuracy goal
for kappa <= 1e6 after refinement); FP64 QR solve within 1e-13 * kappa."""
import numpy as np
import pytest

from oracle.lstsq import lstsq_unblocked
from paper_1110_1553_gb300 import inputs

torch = pytest.importorskip("torch")
hqr = pytest.importorskip("paper_1110_1553_gb300.hqr")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1110_1553_gb300 import _build
    _build.build()
    hqr.load()


def make(M, N, seed, dtype):
    A = inputs.gaussian(M, N, seed=seed)
    b = inputs.rng(seed, 1).standard_normal(M)
    if dtype == np.float32:
        A = A.astype(np.float32)
    return A, b


def to_dev(A, b, N):
    Ad = torch.from_numpy(np.asfortranarray(A).T.copy()).cuda().t()
    return Ad, torch.from_numpy(b).cuda(), torch.zeros(N, dtype=torch.float64, device="cuda")


SHAPES = [(64, 32), (200, 37), (512, 128), (1000, 333), (96, 96), (2048, 64)]


@pytest.mark.parametrize("mixed", [False, True])
def test_batched_solves_match_oracle(mixed):
    dt = np.float32 if mixed else np.float64
    probs, host = [], []
    for q, (M, N) in enumerate(SHAPES):
        A, b = make(M, N, 50 + q, dt)
        host.append((A.astype(np.float64), b))
        probs.append(to_dev(A, b, N))
    plan = hqr.LSPlan(probs, refine_iters=6 if mixed else 0)
    plan.run()
    assert plan.status() == 0
    if not mixed:  # no refinement rounds: no correction to report
        assert plan.correction(0) == -1.0
    for (A, b), (_, _, x) in zip(host, probs):
        xo = lstsq_unblocked(A, b)
        err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
        if mixed:
            assert err <= 1e-12, err
        else:
            assert err <= 1e-13 * np.linalg.cond(A), err


def test_alone_and_in_the_mix_are_identical():
    A, b = make(700, 150, 61, np.float32)
    alone = to_dev(A, b, 150)
    cfg = [hqr.tile_config(64, 16, 2, 2, "greedy", "fibonacci")]
    p1 = hqr.LSPlan([alone], refine_iters=5, configs=cfg)
    p1.run()
    assert p1.status() == 0
    mix = []
    for q, (M, N) in enumerate(SHAPES):
        A2, b2 = make(M, N, 70 + q, np.float32)
        mix.append(to_dev(A2, b2, N))
    mine = to_dev(A, b, 150)
    allp = mix[:3] + [mine] + mix[3:]
    cfgs = [hqr.tile_config()] * 3 + cfg + [hqr.tile_config()] * 3
    p2 = hqr.LSPlan(allp, refine_iters=5, configs=cfgs)
    p2.run()
    assert p2.status() == 0
    assert torch.equal(alone[2], mine[2])


def test_graph_replay_and_autotuned_configs():
    probs = [to_dev(*make(M, N, 80 + q, np.float32), N) for q, (M, N) in enumerate(SHAPES)]
    plan = hqr.LSPlan(probs, refine_iters=5)
    s = torch.cuda.Stream()
    plan.capture(s)
    for _ in range(2):
        for _, _, x in probs:
            x.zero_()
        torch.cuda.synchronize()
        plan.run(s)
        assert plan.status(s) == 0
        xs = [x.clone() for _, _, x in probs]
    plan.run(s)
    assert plan.status(s) == 0
    for x0, (_, _, x) in zip(xs, probs):
        assert torch.equal(x0, x)
    info = plan.info()
    assert info["tasks"] > 0 and info["kernel_ms"] > 0
    for q in range(len(SHAPES)):
        nb = plan.config(q)[0]
        assert nb in (32, 64, 128)


def test_singular_problem_reported():
    A, b = make(128, 64, 90, np.float32)
    A[:, 5] = 0.0
    p = hqr.LSPlan([to_dev(A, b, 64)], refine_iters=2, configs=[hqr.tile_config(32, 8, 1, 1)])
    p.run()
    assert p.status() == hqr.ERR_SINGULAR


@pytest.mark.parametrize("kappa,iters", [(1e4, 8), (1e6, 20)])
def test_mixed_square_conditioned_matches_oracle(kappa, iters):
    # the square mixed-precision recipe at n = 1024: A = U diag(s) V^T with s
    # geometric from 1 to 1/kappa, b = A x_true + 1e-8 N(0,1)
    from paper_1110_1553_gb300 import workloads
    n = 1024
    A = workloads.conditioned(torch, n, n, kappa, seed=30 + int(np.log10(kappa)))
    g = torch.Generator(device="cuda")
    g.manual_seed(31)
    xt = torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    b = A.double() @ xt + 1e-8 * torch.randn(n, dtype=torch.float64, device="cuda", generator=g)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    plan = hqr.LSPlan([(A, b, x)], refine_iters=iters, configs=[hqr.tile_config(128, 16, 4, 1)])
    plan.run()
    assert plan.status() == 0
    xo = lstsq_unblocked(A.double().cpu().numpy(), b.cpu().numpy())
    err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
    assert err <= 1e-12, err
    # converged: the last correction is at the rounding level of x; two rounds are not enough
    assert 0.0 <= plan.correction(0) <= 1e-11
    x2 = torch.zeros(n, dtype=torch.float64, device="cuda")
    plan2 = hqr.LSPlan([(A, b, x2)], refine_iters=2, configs=[hqr.tile_config(128, 16, 4, 1)])
    plan2.run()
    assert plan2.status() == 0 and plan2.correction(0) > 1e-9
