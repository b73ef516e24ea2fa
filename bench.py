#!/usr/bin/env python
"""Benchmark: FP64 hierarchical tile QR of a tall-skinny matrix on GB300.

Workload (one step = one whole factorization, all tasks of Alg. 1/Alg. 2):
A = 131072 x 2048 float64 with i.i.d. N(0,1) entries, tiles nb = 256 (512 x 8
tiles), inner block ib = 32, TS domains a = 4, p = 16 virtual domains, Greedy
low-level tree, Fibonacci high-level tree. Throughput uses the paper's flop
count 2 M N^2 - 2/3 N^3 (Sec. 2). A (2.1 GB) is larger than L2 (129 MB).

Prints one JSON line (rank 0). `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QR TFLOP/s and LS solves/s vs plain FP64 at FP64-oracle accuracy; p99 latency"
WORKLOAD = dict(M=131072, N=2048, nb=256, ib=32, a=4, p=16, low="greedy", high="fibonacci")
WORKLOAD_NAME = "hqr_fp64_tall_skinny_131072x2048_nb256_ib32_a4_p16_greedy_fibonacci"
SAMPLE_M = 4096  # oracle sample: the first 16 tile rows, all 2048 columns
PROFILE = os.path.join(ROOT, "profiles", "hqr_sched_fp64_tall_skinny.md")
ENGINE_SRC = os.path.join(ROOT, "paper_1110_1553_gb300", "csrc", "engine.cuh")


def qr_flops(M, N):
    return 2.0 * M * N * N - 2.0 / 3.0 * N ** 3


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def oracle_rate(M, N, wl, repeats=1):
    """CPU oracle (as it stands) on an M x N sample: (TFLOP/s, seconds)."""
    from oracle.elim_list import TREE_NAMES, hqr_elim_list
    from oracle.tile_qr import tile_qr
    from paper_1110_1553_gb300 import inputs
    names = {v: k for k, v in TREE_NAMES.items()}
    A = inputs.gaussian(M, N, seed=2)
    L = hqr_elim_list(M // wl["nb"], N // wl["nb"], wl["a"], wl["p"], names[wl["low"]], names[wl["high"]])
    times = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        tile_qr(A, wl["nb"], wl["ib"], L)
        times.append(time.perf_counter() - t0)
    return qr_flops(M, N) / 1e12 / statistics.median(times), statistics.median(times)


def host_threads():
    for var in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS"):
        if os.environ.get(var):
            return int(os.environ[var])
    return os.cpu_count() or 1


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.out = out
        else:
            self.out = ""

    def summary(self):
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power)}


def measured_dgemm_tflops(torch, dev):
    n = 8192
    a = torch.randn(n, n, dtype=torch.float64, device=dev)
    b = torch.randn(n, n, dtype=torch.float64, device=dev)
    torch.matmul(a, b)
    torch.cuda.synchronize(dev)
    best = 0.0
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b)
        e1.record()
        e1.synchronize()
        best = max(best, 2.0 * n ** 3 / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    del a, b
    return best


def ncu_traffic():
    """DRAM bytes per launch of the task kernel from the committed ncu summary,
    or None when the kernel source changed since that capture."""
    if not os.path.exists(PROFILE):
        return None, None
    txt = open(PROFILE).read()
    m_sha = re.search(r"engine_sha256:\s*([0-9a-f]{64})", txt)
    m_b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_b:
        return None, None
    cur = hashlib.sha256(open(ENGINE_SRC, "rb").read()).hexdigest()
    if cur != m_sha.group(1):
        return None, "stale"
    return float(m_b.group(1)), None


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    wl = WORKLOAD
    for _ in range(args.warmup):
        oracle_rate(SAMPLE_M, wl["N"], wl)
    rates, secs = [], []
    for _ in range(args.steps):
        r, s = oracle_rate(SAMPLE_M, wl["N"], wl)
        rates.append(r)
        secs.append(s)
    value = qr_flops(SAMPLE_M, wl["N"]) * len(secs) / sum(secs) / 1e12
    sample = "oracle tile QR of the first %d x %d rows/cols (%d x %d tiles) of the workload" % (
        SAMPLE_M, wl["N"], SAMPLE_M // wl["nb"], wl["N"] // wl["nb"])
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_NAME, **wl, "sample_rows": SAMPLE_M},
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": host_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rows", type=int, default=WORKLOAD["M"],
                    help="rows M of the tall-skinny matrix (default: the full workload; smaller values "
                         "only for profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    from paper_1110_1553_gb300 import _build, hqr, inputs
    if rank == 0:
        _build.build()
    barrier()
    hqr.load()
    wl = dict(WORKLOAD, M=args.rows)
    M, N, nb, ib = wl["M"], wl["N"], wl["nb"], wl["ib"]
    recs = hqr.elim_list(M // nb, N // nb, wl["a"], wl["p"], wl["low"], wl["high"])
    A = inputs.gaussian_torch(M, N, seed=1 + rank, device=dev)  # column-major, 2.1 GB
    t_setup = time.perf_counter()
    F = hqr.geqrf(A, nb, ib, recs)
    t_setup = time.perf_counter() - t_setup
    stream = torch.cuda.current_stream(dev)

    # accuracy property that holds at any size: Q is orthogonal, so the
    # column norms of R equal those of A
    R = F.R()
    cn_err = ((R.norm(dim=0) - A.norm(dim=0)).abs() / A.norm(dim=0)).max().item()
    del R

    for _ in range(args.warmup):
        F.refactor_async(A)
    torch.cuda.synchronize(dev)

    kernel_ms = []
    launches = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            F.refactor_async(A)
            launches += hqr.last_launches()
            kernel_ms.append(F.kernel_ms())
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    st = F.status()
    if st != 0:
        raise RuntimeError("factorization failed with status %d" % st)
    ms_total = e0.elapsed_time(e1)
    if dist is not None:
        t = torch.tensor([ms_total], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_total = t.item()
    flops = qr_flops(M, N)
    value = flops * args.steps * world / (ms_total * 1e-3) / 1e12
    kern_tflops = flops / (statistics.mean(kernel_ms) * 1e-3) / 1e12

    # end to end through the public API with host buffers: H2D of A from
    # pinned memory, the factorization, D2H of R, every step
    A_host = torch.empty((N, M), dtype=torch.float64, pin_memory=True).t()
    A_host.copy_(A)
    R_host = torch.empty((N, N), dtype=torch.float64, pin_memory=True).t()
    A_dev = torch.empty_like(A)
    k_e2e = max(1, min(args.steps, 3))
    torch.cuda.synchronize(dev)
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(k_e2e):
        A_dev.copy_(A_host, non_blocking=True)
        F.refactor_async(A_dev)
        launches_e2e = hqr.last_launches()
        R = F.R()
        R_host.copy_(R, non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = t0.elapsed_time(t1)
    e2e_value = flops * k_e2e * world / (e2e_ms * 1e-3) / 1e12
    del A_dev, A_host

    peak = measured_dgemm_tflops(torch, dev) if rank == 0 else None
    traffic, traffic_note = ncu_traffic()

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, secs = oracle_rate(SAMPLE_M, N, wl)
        cpu = {"value": rate, "unit": "TFLOP/s", "cores": host_threads(), "kind": "oracle",
               "sample": "oracle tile QR (NumPy FP64) of the first %d x %d rows/cols of the workload, "
                         "%.1f s" % (SAMPLE_M, N, secs)}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME if M == WORKLOAD["M"] else "profiling_%dx%d" % (M, N),
                   **wl, "tasks": F.ntasks,
                   "l2": "inputs larger than L2 (A is %.2f GB)" % (M * N * 8 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": M * N * 8,
                "d2h_bytes_per_step": N * N * 8, "steps": k_e2e},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": kern_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": (kern_tflops / peak) if peak else None, "traffic": traffic,
                     "kernel": "hqr::hqr_sched<double>",
                     "peak_source": "FP64 cuBLAS DGEMM 8192^3 measured in this run (best of 3); "
                                    "no FP64 entry in MEASURED_PEAKS.json",
                     "traffic_note": traffic_note},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "accuracy": {"max_rel_colnorm_err_R_vs_A": cn_err},
        "setup_s": t_setup,
    }
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
