"""Continuous-batching server on the GPU: requests submitted while others
run are admitted as room frees up; every result equals the one the same
problem gets alone in a plan (bitwise: same per-task arithmetic), and
matches the FP64 oracle within 1e-12. Admission against the HBM budget."""
import time

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
    hqr.set_tuning({})


def problem(M, N, seed):
    A = inputs.gaussian(M, N, seed=seed).astype(np.float32)
    b = inputs.rng(seed, 1).standard_normal(M)
    Ad = torch.from_numpy(np.asfortranarray(A).T.copy()).cuda().t()
    return A, b, Ad, torch.from_numpy(b).cuda(), torch.zeros(N, dtype=torch.float64, device="cuda")


def wait_all(srv, tickets, done, timeout=60.0):
    pending, t0 = set(tickets) - done, time.time()
    while pending and time.time() - t0 < timeout:
        for t in srv.poll():
            done.add(t)
            pending.discard(t)
    assert not pending


@pytest.mark.parametrize("tensor", [False, True])
def test_server_mix_equals_alone_and_oracle(tensor):
    """tensor=True: the requests whose default tile is 128 (here 4096 x 256,
    2048 x 300, 3000 x 129) run on the tensor-core kernels, the others on the
    FP32 CUDA-core kernels, all in the same resident launch."""
    shapes = [(300, 100), (64, 64), (1000, 200), (2048, 96), (150, 33), (700, 512), (4096, 256), (128, 32),
              (2048, 300), (3000, 129)]
    probs = [problem(M, N, 200 + q) for q, (M, N) in enumerate(shapes)]
    srv = hqr.Server(torch.float32, refine_iters=5, max_live=4, hbm_budget=2 << 30, tensor=tensor)
    srv.start()
    try:
        tickets, queue, done = [], list(range(len(probs))), set()
        t0 = time.time()
        while queue and time.time() - t0 < 60:
            q = queue[0]
            t = srv.submit(*probs[q][2:])
            if t is None:  # not admitted yet: wait for room
                done.update(srv.poll())
                continue
            tickets.append(t)
            queue.pop(0)
        assert not queue
        wait_all(srv, tickets, done)
    finally:
        srv.stop()
    for q, (A, b, Ad, bd, x) in enumerate(probs):
        xo = lstsq_unblocked(A.astype(np.float64), b)
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-12
        x1 = torch.zeros_like(x)
        plan = hqr.LSPlan([(Ad, bd, x1)], refine_iters=5, tensor=tensor)
        plan.run()
        assert plan.status() == 0
        assert torch.equal(x1, x), q


def test_server_burst_runs_oldest_first():
    """A burst of equal requests admitted at once, more than the GPU runs
    side by side: the server runs the oldest requests first (age classes over
    the critical-path classes) and fills idle CTAs with newer ones, so
    completion times rise with submission order instead of every request
    sharing the GPU to the end. Results do not depend on the order (bitwise
    equal to a plan of the same problem)."""
    n = 48
    probs = [problem(4096, 512, 400 + q) for q in range(n)]
    srv = hqr.Server(torch.float32, refine_iters=5, max_live=64, hbm_budget=8 << 30)
    srv.start()
    try:
        tickets = [srv.submit(*p[2:]) for p in probs]
        assert all(t is not None for t in tickets)
        when, t0 = {}, time.perf_counter()
        while len(when) < n and time.perf_counter() - t0 < 60:
            for t in srv.poll():
                when[t] = time.perf_counter() - t0
    finally:
        srv.stop()
    assert len(when) == n
    done_at = np.array([when[t] for t in tickets])
    rho = np.corrcoef(np.arange(n), done_at)[0, 1]
    assert rho > 0.5 and done_at[:8].mean() < done_at[-8:].mean(), (rho, done_at)
    for q in (0, n - 1):
        A, b, Ad, bd, x = probs[q]
        x1 = torch.zeros_like(x)
        plan = hqr.LSPlan([(Ad, bd, x1)], refine_iters=5)
        plan.run()
        assert plan.status() == 0
        assert torch.equal(x1, x), q


def test_server_fresh_servers_back_to_back():
    """Servers created one after another, each fed a burst at once: the
    device fills of a new server land before its kernel or any submission
    runs (every request completes, inbox counters match)."""
    probs = [problem(1024, 256, 500 + q) for q in range(16)]
    for rep in range(3):
        srv = hqr.Server(torch.float32, refine_iters=2, max_live=32, hbm_budget=4 << 30, task_pool=4 << 20)
        srv.start()
        try:
            tickets = [srv.submit(*p[2:]) for p in probs]
            assert all(t is not None for t in tickets)
            done, t0 = set(), time.time()
            while len(done) < len(tickets) and time.time() - t0 < 30:
                done.update(srv.poll())
            assert done == set(tickets), rep
            c = srv.counters()
            assert c["inbox_claimed"] == c["inbox_posted"] == len(tickets), c
        finally:
            srv.stop()
        del srv


def test_fp64_server_split_panels_equal_plan_and_oracle():
    """FP64 requests with tiles of 64 and 128 run split panels (one task per ib block plus the
    updates of the panel's own columns) inside the server's request graphs: every result equals
    the same problem in a plan (bitwise) and the oracle's least-squares solution (1e-12)."""
    shapes = [(300, 100), (700, 190), (2048, 300), (1500, 64)]
    probs = []
    for q, (M, N) in enumerate(shapes):
        A = inputs.gaussian(M, N, seed=600 + q)
        b = inputs.rng(600 + q, 1).standard_normal(M)
        Ad = torch.from_numpy(np.asfortranarray(A).T.copy()).cuda().t()
        probs.append((A, b, Ad, torch.from_numpy(b).cuda(), torch.zeros(N, dtype=torch.float64, device="cuda")))
    srv = hqr.Server(torch.float64, refine_iters=0, max_live=4, hbm_budget=2 << 30)
    srv.start()
    try:
        tickets, done = [], set()
        for pr in probs:
            t, t0 = None, time.time()
            while t is None and time.time() - t0 < 60:
                t = srv.submit(*pr[2:])
                if t is None:
                    done.update(srv.poll())
            assert t is not None
            tickets.append(t)
        wait_all(srv, tickets, done)
    finally:
        srv.stop()
    for q, (A, b, Ad, bd, x) in enumerate(probs):
        xo = lstsq_unblocked(A, b)
        assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-12, q
        x1 = torch.zeros_like(x)
        plan = hqr.LSPlan([(Ad, bd, x1)], refine_iters=0)
        plan.run()
        assert plan.status() == 0
        assert torch.equal(x1, x), q


def test_server_budget_admission():
    srv = hqr.Server(torch.float32, refine_iters=2, max_live=2, hbm_budget=4 << 20)
    srv.start()
    try:
        A, b, Ad, bd, x = problem(2048, 512, 300)  # workspace far above 4 MiB
        with pytest.raises(hqr.HQRError) as e:
            srv.submit(Ad, bd, x)
        assert e.value.status == hqr.ERR_BUDGET
        small = [problem(64, 32, 301 + q) for q in range(3)]
        t1 = srv.submit(*small[0][2:])
        t2 = srv.submit(*small[1][2:])
        assert t1 is not None and t2 is not None
        t3 = None
        t0 = time.time()
        while t3 is None and time.time() - t0 < 30:  # two slots: the third waits for a completion
            t3 = srv.submit(*small[2][2:])
            srv.poll()
        assert t3 is not None
    finally:
        srv.stop()
    srv.poll()
    assert srv.stats()["completed"] == 3


def test_server_idle_exit_and_restart():
    # the resident kernel leaves after ~1 s idle; a later request relaunches it
    srv = hqr.Server(torch.float32, refine_iters=3, max_live=2, hbm_budget=64 << 20)
    srv.start()
    try:
        A, b, Ad, bd, x = problem(256, 64, 310)
        time.sleep(2.5)
        t = srv.submit(Ad, bd, x)
        assert t is not None
        wait_all(srv, [t], set())
    finally:
        srv.stop()
    xo = lstsq_unblocked(A.astype(np.float64), b)
    assert np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo) <= 1e-12
