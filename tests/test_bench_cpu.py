"""CPU tests of bench.py's multi-process logic (one process per GPU; on the
CPU: world size 2 over gloo): the whole-job rate is the units of all ranks
over the slowest rank's time, and the reference arm reports from rank 0
only (the other ranks exit 0 without work)."""
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        # rank 1 is the slow one: 150 ms for the same 3 steps of 1e12 flops
        value, ms = bench.whole_job_rate(torch, dist, 100.0 + 50.0 * rank, 1e12, 3, 2, torch.device("cpu"))
        q.put((rank, value, ms))
    finally:
        dist.destroy_process_group()


def test_whole_job_rate_over_the_slowest_of_two_gloo_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    try:
        got = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for pr in procs:
            pr.join(timeout=60)
    assert [pr.exitcode for pr in procs] == [0, 0]
    for rank, value, ms in got:
        assert ms == 150.0
        assert value == pytest.approx(2 * 3 * 1e12 / 0.150 / 1e12)


def test_whole_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    value, ms = bench.whole_job_rate(torch, None, 200.0, 2e12, 5, 1, torch.device("cpu"))
    assert ms == 200.0 and value == pytest.approx(5 * 2e12 / 0.2 / 1e12)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == ""
