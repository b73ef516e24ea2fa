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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QR TFLOP/s and LS solves/s vs plain FP64 at FP64-oracle accuracy; p99 latency"
WORKLOAD = dict(M=131072, N=2048, nb=256, ib=32, a=4, p=16, low="greedy", high="fibonacci")
WORKLOAD_NAME = "hqr_fp64_tall_skinny_131072x2048_nb256_ib32_a4_p16_greedy_fibonacci"
SAMPLE_M = 4096  # oracle sample: the first 16 tile rows, all 2048 columns
PROFILE = os.path.join(ROOT, "profiles", "hqr_sched_fp64_tall_skinny.md")
# the task kernels are compiled from these headers; the committed DRAM counters
# hold for the kernels built from the hashed versions only
KERNEL_SRCS = [os.path.join(ROOT, "paper_1110_1553_gb300", "csrc", f) for f in ("engine.cuh", "ptx.cuh", "tc.cuh")]


def kernel_sources_sha256():
    h = hashlib.sha256()
    for f in KERNEL_SRCS:
        h.update(open(f, "rb").read())
    return h.hexdigest()


def qr_flops(M, N):
    return 2.0 * M * N * N - 2.0 / 3.0 * N ** 3


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def whole_job_rate(torch, dist, ms_local, flops_per_step, steps, world, device):
    """Whole-job TFLOP/s over the slowest rank: every rank processed `steps`
    steps of `flops_per_step` in its own `ms_local`; the job took the maximum
    over ranks (all-reduce MAX when a process group is given). Returns
    (TFLOP/s, that maximum in ms)."""
    ms = float(ms_local)
    if dist is not None and world > 1:
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
    return flops_per_step * steps * world / (ms * 1e-3) / 1e12, ms


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


def oracle_batched(b, sample=8):
    """CPU oracle on the first `sample` batched problems: its solves/s and the
    relative error of both GPU paths' x against it."""
    import numpy as np

    from oracle.lstsq import lstsq_unblocked
    shapes, data = b["_data"]
    errs = {"mixed_tc": [], "mixed": [], "fp64": []}
    t0 = time.perf_counter()
    for q in range(sample):
        A = data[q][0].double().cpu().numpy()
        bb = data[q][1].cpu().numpy()
        xo = lstsq_unblocked(A, bb)
        for label in errs:
            x = b["_x_" + label][q].cpu().numpy()
            errs[label].append(float(np.linalg.norm(x - xo) / np.linalg.norm(xo)))
    secs = time.perf_counter() - t0
    return {"kind": "oracle", "unit": "solves/s", "value": sample / secs, "cores": host_threads(),
            "sample": "oracle least squares (unblocked Householder QR + Dot2 refinement) of the first %d "
                      "batched problems" % sample,
            "max_rel_err_vs_oracle": {k: max(v) for k, v in errs.items()}}


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
    m_sha = re.search(r"kernel_sources_sha256:\s*([0-9a-f]{64})", txt)
    m_b = re.search(r"dram_bytes_per_launch_full:\s*([0-9.eE+]+)", txt)
    if not m_sha or not m_b:
        return None, None
    cur = kernel_sources_sha256()
    if cur != m_sha.group(1):
        return None, "stale"
    return float(m_b.group(1)), None


def latency_square(torch, hqr, inputs, dev, reps=100, peak=None):
    """512 x 512 FP64 (nb 64, ib 16, flat TS a = 8): QR plus Q applied to I,
    device time per call, p50 / p99 over `reps` calls."""
    A = inputs.gaussian_torch(512, 512, seed=11, device=dev)
    recs = hqr.elim_list(8, 8, 8, 1, "flat", "flat")
    F = hqr.geqrf(A, 64, 16, recs)
    I = torch.eye(512, dtype=torch.float64, device=dev)
    Q = I.clone().t().contiguous().t()
    times = []
    for q in range(reps + 5):
        Q.copy_(I)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        F.refactor_async(A)
        F.apply_q(Q, trans=False)
        e1.record()
        e1.synchronize()
        if q >= 5:
            times.append(e0.elapsed_time(e1) * 1e3)
    times.sort()
    fl = 2 * 512 ** 3 - 2 / 3 * 512 ** 3
    fq = 4.0 * 512 * 512 * 512 - 2.0 * 512 * 512 * 512  # Q applied to I: 4 M N r - 2 N^2 r, r = N
    p50 = times[len(times) // 2]
    out = {"workload": "fp64_square_512_nb64_ib16_flat_ts", "p50_us": p50,
           "p99_us": times[min(len(times) - 1, int(0.99 * len(times)))], "qr_flops": fl, "q_flops": fq,
           "includes": "tile QR + Q applied to I (apply-Q graph), per call"}
    if peak:
        tf = (fl + fq) / (p50 * 1e-6) / 1e12
        out["roofline"] = {"bound": "latency", "achieved": tf, "peak": peak, "unit": "TFLOP/s", "frac": tf / peak,
                           "peak_source": "in-run FP64 DGEMM (context: the case is bound by its critical path)"}
    return out


def batched_buckets(torch, hqr, plan, probs, shapes, dtype, iters, tensor, peaks, reps=3):
    """The batch split by the tile size its configuration chose (32, 64, 128),
    each bucket solved alone in one launch (CUDA graph): QR TFLOP/s (paper's
    flop count over the whole solve, refinement included) against the
    bucket's roofline: the update arithmetic (FP32 FFMA, BF16x3 tensor or
    the FP64 pipe) or HBM at the updates' intensity (nb / (element size)
    flop/B)."""
    cfgs = [plan.config(q) for q in range(len(probs))]
    out = {}
    for nb in sorted({c[0] for c in cfgs}):
        idx = [q for q, c in enumerate(cfgs) if c[0] == nb]
        sub = [probs[q] for q in idx]
        sp = hqr.LSPlan(sub, refine_iters=iters, configs=[hqr.tile_config(*cfgs[q]) for q in idx], tensor=tensor)
        s = torch.cuda.Stream()
        for _ in range(3):
            sp.run(s)
            s.synchronize()
        sp.capture(s)
        sp.run(s)
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            sp.run(s)
        e1.record(s)
        e1.synchronize()
        st = sp.status(s)
        ms = e0.elapsed_time(e1) / reps
        fl = sp.info()["qr_flops"]
        tf = fl / (ms * 1e-3) / 1e12
        if dtype == torch.float64:
            hbm = peaks["hbm_gbs"] * 1e9 * nb / 8.0 / 1e12
            alu = 2 * FP64_OPS_PER_S / 1e12
            bound, pk = ("hbm", hbm) if hbm < alu else ("alu", alu)
        else:
            bound, pk = fp32_qr_bound(peaks, nb, tensor and nb == 128)
        out["nb%d" % nb] = {"problems": len(idx), "solves_per_s": len(idx) / (ms * 1e-3), "ms": ms,
                            "qr_tflops": tf, "status": st,
                            "roofline": {"bound": bound, "achieved": tf, "peak": pk, "unit": "TFLOP/s",
                                         "frac": tf / pk}}
        del sp
    return out


def batched(torch, hqr, dev, count=1024, refine=4, tune=True, peaks=None):
    """1024 uneven least-squares problems in one persistent launch: mixed
    (FP32 QR + FP64 CSNE) and plain FP64 (QR + Q^T b + back substitution)."""
    from paper_1110_1553_gb300 import workloads
    shapes = workloads.uneven_shapes(count)
    out = {"workload": "batched_uneven_%d_fp32_ls" % count, "problems": count}
    g = torch.Generator(device=dev)
    g.manual_seed(1234)
    data = [(torch.randn((n, m), dtype=torch.float32, device=dev, generator=g).t(),
             torch.randn(m, dtype=torch.float64, device=dev, generator=g)) for (m, n) in shapes]
    variants = (("mixed_tc", torch.float32, refine, True), ("mixed", torch.float32, refine, False),
                ("fp64", torch.float64, 0, False))
    for label, dtype, iters, tensor in variants:
        if tune:
            t0 = time.perf_counter()
            table = hqr.autotune(shapes, dtype, iters, reps=24, tensor=tensor)
            out[label + "_autotune_s"] = time.perf_counter() - t0
            out[label + "_autotune_classes"] = len(table)
            out[label + "_tiles_128"] = sum(1 for c in table.values() if c[0] == 128)
        probs = [(A if dtype == torch.float32 else A.double().t().contiguous().t(), b,
                  torch.zeros(n, dtype=torch.float64, device=dev)) for (A, b), (m, n) in zip(data, shapes)]
        plan = hqr.LSPlan(probs, refine_iters=iters, tensor=tensor)
        s = torch.cuda.Stream(dev)
        for _ in range(3):  # plain runs first: a split plan sets its SM share from their times
            plan.run(s)
            s.synchronize()
        plan.capture(s)
        for _ in range(2):
            plan.run(s)
        s.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(s)
        for _ in range(reps):
            plan.run(s)
        e1.record(s)
        e1.synchronize()
        st = plan.status(s)
        ms = e0.elapsed_time(e1) / reps
        info = plan.info()
        out[label] = {"solves_per_s": count / (ms * 1e-3), "ms_per_batch": ms,
                      "qr_tflops": info["qr_flops"] / (ms * 1e-3) / 1e12, "tasks": info["tasks"],
                      "refine_iters": iters, "status": st, "launches_per_batch": 3, "cuda_graph": True,
                      "tensor_cores": tensor}
        out["_x_" + label] = [p[2] for p in probs[:8]]
        if peaks is not None:
            out[label]["buckets"] = batched_buckets(torch, hqr, plan, probs, shapes, dtype, iters, tensor, peaks)
        del plan
        hqr.set_tuning({})
    out["mixed_over_fp64"] = out["mixed"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    out["mixed_tc_over_fp64"] = out["mixed_tc"]["solves_per_s"] / out["fp64"]["solves_per_s"]
    out["_data"] = (shapes, data)
    return out


def serving(torch, hqr, dev, rate=2000.0, seconds=5.0, refine=5, peaks=None, labels=("mixed_tc", "fp64"),
            stop_factor=4.0):
    """Poisson request stream at `rate` req/s for `seconds`: 90 % uneven
    batched-like shapes, 10 % 32768 x 1024 FP32 with kappa = 1e4. Mixed server
    vs plain FP64 server on the same arrivals."""
    from collections import deque

    from paper_1110_1553_gb300 import inputs, workloads
    rng = inputs.rng(5, 0)
    small_shapes = workloads.uneven_shapes(256, seed=6)
    g = torch.Generator(device=dev)
    g.manual_seed(99)
    small = [(torch.randn((n, m), dtype=torch.float32, device=dev, generator=g).t(),
              torch.randn(m, dtype=torch.float64, device=dev, generator=g)) for (m, n) in small_shapes]
    large = [(workloads.conditioned(torch, 32768, 1024, 1e4, seed=40 + q, device=dev),
              torch.randn(32768, dtype=torch.float64, device=dev, generator=g)) for q in range(4)]
    n_req = int(rate * seconds)
    gaps = rng.exponential(1.0 / rate, n_req)
    arrivals = np.cumsum(gaps)
    kinds = rng.uniform(size=n_req) < 0.1
    idx = rng.integers(0, 1 << 30, size=n_req)
    out = {"workload": "serving_poisson_%d_per_s_%gs_90pct_uneven_10pct_32768x1024_kappa1e4" % (rate, seconds),
           "offered_per_s": rate, "requests": n_req}
    for label, dtype, iters, tensor in (("mixed_tc", torch.float32, refine, True),
                                        ("fp64", torch.float64, 0, False)):
        if label not in labels:
            continue
        pool_s = small if dtype == torch.float32 else [(A.double().t().contiguous().t(), b) for A, b in small]
        pool_l = large if dtype == torch.float32 else [(A.double().t().contiguous().t(), b) for A, b in large]
        srv = hqr.Server(dtype, refine_iters=iters, max_live=2048, hbm_budget=120 << 30,
                         task_pool=16 << 20, edge_pool=64 << 20, tensor=tensor)
        srv.start()
        lat, inflight, queue = [], {}, deque()
        done_flops = 0.0
        t0 = time.perf_counter()
        i = 0
        try:
            while i < n_req or queue or inflight:
                now = time.perf_counter() - t0
                while i < n_req and arrivals[i] <= now:
                    queue.append(i)
                    i += 1
                while queue:
                    q = queue[0]
                    A, b = pool_l[idx[q] % 4] if kinds[q] else pool_s[idx[q] % 256]
                    x = torch.zeros(A.shape[1], dtype=torch.float64, device=dev)
                    t = srv.submit(A, b, x)
                    if t is None:
                        break
                    inflight[t] = (arrivals[q], qr_flops(A.shape[0], A.shape[1]))
                    queue.popleft()
                done = srv.poll()
                now = time.perf_counter() - t0
                for t in done:
                    arr, fl = inflight.pop(t)
                    lat.append(now - arr)
                    done_flops += fl
                if now > seconds * stop_factor:  # a saturated server: stop at 4x the arrival window
                    break
            wall = time.perf_counter() - t0
        finally:
            srv.stop()
        lat.sort()
        out[label] = {"completed": len(lat), "not_completed": n_req - len(lat),
                      "solves_per_s": len(lat) / wall, "wall_s": wall,
                      "p50_ms": 1e3 * lat[len(lat) // 2] if lat else None,
                      "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))] if lat else None,
                      "refine_iters": iters, "tensor_cores": tensor,
                      "qr_tflops": done_flops / wall / 1e12}
        if peaks is not None:
            pk = peaks["bf16_tflops_sustained"] / 6.0 if tensor else 2 * FP64_OPS_PER_S / 1e12
            out[label]["roofline"] = {
                "bound": "tensor" if tensor else "alu", "achieved": done_flops / wall / 1e12, "peak": pk,
                "unit": "TFLOP/s", "frac": done_flops / wall / 1e12 / pk,
                "peak_source": ("%s BF16 sustained / 6 (BF16x3)" % peaks["source"]) if tensor else
                               "FP64 pipe: 152 SMs x 2 FMA/cycle x 2.07 GHz"}
        del srv
    return out


PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
# unit-count peaks at the maximum SM clock (2.07 GHz, 152 SMs): FP32 FFMA
# 128 lanes per SM (2 flops each); FP64 pipe 2 thread-operations per cycle
# per SM (an FMA or any other FP64 operation, incl. FP32 -> FP64 conversions)
FP32_ALU_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_OPS_PER_S = 152 * 2 * 2.07e9


def pool_peaks():
    """HBM GB/s and BF16 tensor TFLOP/s (burst and sustained) measured on this
    pool's GPUs, else the machine's fallback figures; `source` says which."""
    try:
        d = json.load(open(PEAKS_FILE))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]), "source": "measured"}
    except (OSError, ValueError, KeyError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def fp32_qr_bound(peaks, nb, tensor, sustained=False):
    """Roofline of an FP32 tile QR with tiles of nb: the update arithmetic
    (BF16x3 = six BF16 products on the tensor pipe, or FP32 FFMA) against HBM
    at the updates' intensity of nb / 4 flop per byte (the killer tile kept on
    chip along a TS chain, FP32 elements). Returns (bound, peak TFLOP/s)."""
    alu = (peaks["bf16_tflops_sustained" if sustained else "bf16_tflops"] / 6.0) if tensor else FP32_ALU_TFLOPS
    hbm = peaks["hbm_gbs"] * 1e9 * nb / 4.0 / 1e12
    return ("hbm", hbm) if hbm < alu else (("tensor" if tensor else "alu"), alu)


def refine_fp64_ops(n_rows, n_cols, plain_rounds, comp_rounds):
    """FP64 pipe operations of the refinement rounds of one M x N problem:
    a plain round = r = b - A x and A^T r with one FMA and one FP32 -> FP64
    conversion per element of A (4 M N), plus the two triangular solves with
    the FP32 R (N^2 / 2 FMAs and conversions each: 2 N^2); a compensated round
    = 11 operations per element of A for each product (TwoProduct 2, TwoSum 6,
    accumulation 2, conversion 1: 22 M N) plus the solves."""
    mn, nn = float(n_rows) * n_cols, float(n_cols) * n_cols
    return plain_rounds * (4 * mn + 2 * nn) + comp_rounds * (22 * mn + 2 * nn)


def trace_phases(tr):
    """QR phase (kernel start to the end of the last packing / tile task) and
    refinement phase (the rest) of a traced least-squares plan run, in ms.
    Tasks of cancelled refinement rounds never ran and have no timestamps."""
    tr = tr[tr[:, 1] > 0]
    ops = tr[:, 3] >> np.uint64(24)
    qr = (ops <= 5) | (ops == 14)
    t0 = tr[:, 0].min()
    qr_end = tr[qr, 1].max()
    return float(qr_end - t0) * 1e-6, float(tr[:, 1].max() - qr_end) * 1e-6


GOLDEN = os.path.join(ROOT, "tests", "golden")


def serving_sustainable(torch, hqr, dev, peaks, seconds=3.0):
    """Highest offered Poisson rate (of a few) that each server sustains: at
    least 97 % of the requests completed within the window plus 50 %, with
    p50 / p99 latency at that rate."""
    out = {"criterion": "completed >= 97 %% of the offered requests within 1.5x the %g s arrival window" % seconds}
    for label, rates in (("mixed_tc", (400.0, 600.0, 750.0, 900.0)), ("fp64", (110.0, 140.0, 170.0))):
        best = None
        for rate in rates:
            r = serving(torch, hqr, dev, rate=rate, seconds=seconds, peaks=peaks, labels=(label,), stop_factor=2.0)[label]
            ok = r["completed"] >= 0.97 * int(rate * seconds) and r["wall_s"] <= 1.5 * seconds
            if ok:
                best = dict(r, offered_per_s=rate)
            else:
                break
        out[label] = best if best else {"offered_per_s": None, "note": "no tried rate was sustained"}
    return out


def square_mixed_oracle(A, b, n):
    """The committed FP64 oracle solution of the square mixed workload (written
    by tests/golden/make_square_mixed_oracle.py with oracle/ alone), if the
    fingerprints of this run's A and b match the ones it was computed for."""
    meta_f = os.path.join(GOLDEN, "square_mixed_%d_oracle.json" % n)
    x_f = os.path.join(GOLDEN, "square_mixed_%d_oracle_x.npy" % n)
    if not (os.path.exists(meta_f) and os.path.exists(x_f)):
        return None, "no committed oracle solution"
    meta = json.load(open(meta_f))
    Ah = A.cpu().numpy()
    ha = hashlib.sha256(np.asfortranarray(Ah).tobytes(order="F")).hexdigest()
    hb = hashlib.sha256(np.ascontiguousarray(b.cpu().numpy()).tobytes()).hexdigest()
    if ha != meta["sha256_A_fp32_colmajor"] or hb != meta["sha256_b_fp64"]:
        return None, "input fingerprint differs from the one the oracle solved"
    return np.load(x_f), meta["oracle"]


def square_mixed(torch, hqr, dev, peaks, n=16384, max_iter=40, tol=1e-12):
    """16384^2 FP32 least squares, A = U diag(s) V^T, s geometric 1 .. 1e-6,
    b = A x_true + 1e-8 N(0,1): FP32 tile QR with tensor-core updates
    (BF16x3) + FP64 CSNE refinement stopped at ||d|| <= tol ||x|| (at most
    max_iter rounds); x against the committed FP64 oracle solution."""
    from paper_1110_1553_gb300 import workloads
    A, b = workloads.square_mixed_problem(torch, n, device=dev)
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    nb = 128
    cfg = [hqr.tile_config(nb, nb, 16, 1, "greedy", "greedy")]
    plan = hqr.LSPlan([(A, b, x)], refine_iters=max_iter, configs=cfg, tensor=True, tol=tol)
    plan.run()
    plan.status()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    plan.run()
    e1.record()
    e1.synchronize()
    st = plan.status()
    ms = e0.elapsed_time(e1)
    info = plan.info()
    iters, last_corr, met, _, ncomp = plan.refine_info(0)
    # one traced run for the split between the QR and the refinement
    plan.trace(True)
    plan.run()
    plan.status()
    qr_ms, ref_ms = trace_phases(plan.trace())
    plan.trace(False)
    bound, qpeak = fp32_qr_bound(peaks, nb, True)
    qr_tf = info["qr_flops"] / (qr_ms * 1e-3) / 1e12
    rops = refine_fp64_ops(n, n, iters - ncomp, ncomp)
    xo, how = square_mixed_oracle(A, b, n)
    xh = x.cpu().numpy()
    err = float(np.linalg.norm(xh - xo) / np.linalg.norm(xo)) if xo is not None else None
    # independent cross-check (a library FP64 QR solve, itself accurate to about kappa * u64)
    ref = torch.linalg.lstsq(A.double(), b.unsqueeze(1), driver="gels").solution[:, 0]
    cross = ((x - ref).norm() / ref.norm()).item()
    return {"workload": "square_mixed_ls_16384_kappa1e6", "ms": ms, "solves_per_s": 1e3 / ms,
            "qr_tflops": info["qr_flops"] / (ms * 1e-3) / 1e12, "status": st,
            "refinement": {"tol": tol, "max_iter": max_iter, "iters": iters, "compensated_rounds": ncomp,
                           "converged": met, "last_rel_correction": last_corr},
            "rel_err_vs_oracle": err, "oracle": how,
            "rel_diff_vs_cusolver_fp64_qr": cross, "tasks": info["tasks"],
            "phases_ms": {"qr": qr_ms, "refinement": ref_ms, "from": "one traced run (per-task %globaltimer)"},
            "roofline": {
                "qr": {"bound": bound, "achieved": qr_tf, "peak": qpeak, "unit": "TFLOP/s", "frac": qr_tf / qpeak,
                       "tensor_peak": peaks["bf16_tflops"] / 6.0,
                       "hbm_peak": peaks["hbm_gbs"] * 1e9 * nb / 4 / 1e12,
                       "peak_source": "%s BF16 burst / 6 (BF16x3) and HBM x nb/4 flop/B" % peaks["source"]},
                "refinement": {"bound": "alu", "achieved": rops / (ref_ms * 1e-3) / 1e9, "peak": FP64_OPS_PER_S / 1e9,
                               "unit": "G FP64-ops/s", "frac": rops / (ref_ms * 1e-3) / FP64_OPS_PER_S,
                               "ops": rops, "plain_rounds": iters - ncomp, "compensated_rounds": ncomp,
                               "peak_source": "FP64 pipe: 152 SMs x 2 ops/cycle x 2.07 GHz"}}}


def list_stats(recs):
    """Records, coupling-level records and the unit-time critical path (the
    largest step) of a list."""
    steps = [int(r["step"]) for r in recs]
    return {"records": len(recs), "level2_records": int(sum(1 for r in recs if int(r["level"]) == 2)),
            "unit_time_steps": max(steps) if steps else 0}


def time_list(torch, hqr, A, nb, ib, recs, reps):
    """Factor A with the list (a first run, then `reps` timed runs back to
    back): mean task-kernel ms, status, max relative column-norm error of R."""
    F = hqr.geqrf(A, nb, ib, recs)
    F.kernel_times()
    for _ in range(reps):
        F.refactor_async(A)
    ms = F.kernel_times()
    st = F.status()
    R = F.R()
    cn = ((R.norm(dim=0) - A.norm(dim=0)).abs() / A.norm(dim=0)).max().item()
    del F, R
    torch.cuda.empty_cache()
    return statistics.mean(ms), st, cn


def list_variants(torch, hqr, A, peak, wl, headline_ms, reps=2):
    """The tall-skinny workload factored with other elimination lists on the
    same kernels (the comparisons of Sec. 5): Flat and Binary low-level trees,
    the coupling ("domino") level of Sec. 4.2, and the prior-art lists
    [SLHD10] (p = 1, TS domains of m / 16 tiles, binary tree) and [BBD+10]
    (the flat tile QR: p = 1, one TS domain)."""
    M, N, nb, ib = wl["M"], wl["N"], wl["nb"], wl["ib"]
    m, n = M // nb, N // nb
    fl = qr_flops(M, N)
    out = {"workload": "fp64_tall_skinny_%dx%d_nb%d_ib%d" % (M, N, nb, ib), "peak_tflops": peak,
           "peak_source": "FP64 cuBLAS DGEMM measured in this run", "reps": reps}
    head = hqr.elim_list(m, n, wl["a"], wl["p"], wl["low"], wl["high"])
    out["greedy_fibonacci_a4_p16"] = dict(list_stats(head), ms=headline_ms, tflops=fl / (headline_ms * 1e-3) / 1e12,
                                          frac_of_dgemm=fl / (headline_ms * 1e-3) / 1e12 / peak, headline=True)
    variants = [
        ("greedy_fibonacci_a4_p16_domino", (wl["a"], wl["p"], "greedy", "fibonacci", True)),
        ("flat_fibonacci_a4_p16", (wl["a"], wl["p"], "flat", "fibonacci", False)),
        ("binary_fibonacci_a4_p16", (wl["a"], wl["p"], "binary", "fibonacci", False)),
        ("fibonacci_fibonacci_a4_p16_domino", (wl["a"], wl["p"], "fibonacci", "fibonacci", True)),
        ("slhd10_p1_a%d_binary" % (m // 16), (m // 16, 1, "binary", "flat", False)),
        ("bbd10_flat_p1_a%d" % m, (m, 1, "flat", "flat", False)),
    ]
    for label, (a, p, low, high, domino) in variants:
        recs = hqr.elim_list(m, n, a, p, low, high, domino=domino)
        ms, st, cn = time_list(torch, hqr, A, nb, ib, recs, reps)
        tf = fl / (ms * 1e-3) / 1e12
        out[label] = dict(list_stats(recs), a=a, p=p, low=low, high=high, domino=domino, ms=ms, tflops=tf,
                          frac_of_dgemm=tf / peak, status=st, max_rel_colnorm_err=cn)
    return out


def square_fp64(torch, hqr, inputs, dev, peak, n=16384, nb=256, ib=32):
    """A large square FP64 factorization (Sec. 5's square runs): 16384^2
    N(0, 1), tiles of 256, low-level Fibonacci tree, high-level Flat tree,
    a = 4 (the paper's best square setting), p = 4; with and without the
    coupling level (Sec. 5 reports that it hurts large square matrices)."""
    A = inputs.gaussian_torch(n, n, seed=12, device=dev)
    m = n // nb
    fl = qr_flops(n, n)
    out = {"workload": "fp64_square_%d_nb%d_ib%d" % (n, nb, ib), "qr_flops": fl, "peak_tflops": peak,
           "peak_source": "FP64 cuBLAS DGEMM measured in this run"}
    for label, domino in (("fibonacci_flat_a4_p4", False), ("fibonacci_flat_a4_p4_domino", True)):
        recs = hqr.elim_list(m, m, 4, 4, "fibonacci", "flat", domino=domino)
        ms, st, cn = time_list(torch, hqr, A, nb, ib, recs, 1)
        tf = fl / (ms * 1e-3) / 1e12
        out[label] = dict(list_stats(recs), ms=ms, tflops=tf, status=st, max_rel_colnorm_err=cn,
                          roofline={"bound": "alu", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                                    "frac": tf / peak, "peak_source": "in-run FP64 DGEMM"})
    del A
    torch.cuda.empty_cache()
    return out


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
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the latency, batched, serving and square mixed-precision measurements")
    ap.add_argument("--serve-seconds", type=float, default=5.0)
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
    F.kernel_times()  # drop the warm-up runs

    launches = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(args.steps):
            F.refactor_async(A)  # back to back: no host wait inside the timed loop
            launches += hqr.last_launches()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
    # per-step device time of the task kernel (events recorded by the library
    # on the launching stream around each launch)
    kernel_ms = F.kernel_times()
    assert len(kernel_ms) == args.steps
    st = F.status()
    if st != 0:
        raise RuntimeError("factorization failed with status %d" % st)
    flops = qr_flops(M, N)
    value, ms_total = whole_job_rate(torch, dist, e0.elapsed_time(e1), flops, args.steps, world, dev)
    kern_tflops = flops / (statistics.mean(kernel_ms) * 1e-3) / 1e12

    # end to end through the public API with host buffers, pipelined as a
    # caller would run it: every step copies its A from pinned host memory,
    # factorizes it and reads R back to pinned memory; step k+1's copy runs
    # on a copy stream (into the other of two device buffers) while step k
    # factorizes
    A_host = torch.empty((N, M), dtype=torch.float64, pin_memory=True).t()
    A_host.copy_(A)
    R_host = torch.empty((N, N), dtype=torch.float64, pin_memory=True).t()
    A_dev = [torch.empty_like(A), torch.empty_like(A)]
    cs = torch.cuda.Stream(dev)
    copied = [torch.cuda.Event(), torch.cuda.Event()]
    consumed = [torch.cuda.Event(), torch.cuda.Event()]
    k_e2e = max(2, min(args.steps, 4))
    # host link alone (one copy, for context)
    h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    h0.record(stream)
    A_dev[0].copy_(A_host, non_blocking=True)
    h1.record(stream)
    torch.cuda.synchronize(dev)
    h2d_gbs = M * N * 8 / (h0.elapsed_time(h1) * 1e-3) / 1e9
    barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    cs.wait_event(t0)
    with torch.cuda.stream(cs):
        A_dev[0].copy_(A_host, non_blocking=True)
        copied[0].record(cs)
    for k in range(k_e2e):
        b = k % 2
        if k + 1 < k_e2e:
            nxt = (k + 1) % 2
            if k >= 1:
                cs.wait_event(consumed[nxt])  # step k-1 is done with that buffer
            with torch.cuda.stream(cs):
                A_dev[nxt].copy_(A_host, non_blocking=True)
                copied[nxt].record(cs)
        stream.wait_event(copied[b])
        F.refactor_async(A_dev[b])
        launches_e2e = hqr.last_launches()
        consumed[b].record(stream)
        R = F.R()
        R_host.copy_(R, non_blocking=True)
    t1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_value, _ = whole_job_rate(torch, dist, t0.elapsed_time(t1), flops, k_e2e, world, dev)
    del A_dev, A_host

    peak = measured_dgemm_tflops(torch, dev) if rank == 0 else None
    pipes = hqr.fp64_pipe_rates() if rank == 0 else (None, None)
    traffic, traffic_note = ncu_traffic()
    ntasks = F.ntasks
    del F
    torch.cuda.empty_cache()

    extras = {}
    if not args.no_extras and M == WORKLOAD["M"] and world == 1:
        peaks = pool_peaks()
        extras["list_variants"] = list_variants(torch, hqr, A, peak, wl, statistics.mean(kernel_ms))
        del A
        torch.cuda.empty_cache()
        extras["square_fp64"] = square_fp64(torch, hqr, inputs, dev, peak)
        extras["latency_square"] = latency_square(torch, hqr, inputs, dev, peak=peak)
        extras["batched"] = batched(torch, hqr, dev, peaks=peaks)
        extras["square_mixed"] = square_mixed(torch, hqr, dev, peaks)
        extras["serving"] = serving(torch, hqr, dev, seconds=args.serve_seconds, peaks=peaks)
        extras["serving_200"] = serving(torch, hqr, dev, rate=200.0, seconds=args.serve_seconds, peaks=peaks)
        extras["serving_sustainable"] = serving_sustainable(torch, hqr, dev, peaks)

    if rank != 0:
        return 0
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, secs = oracle_rate(SAMPLE_M, N, wl)
        cpu = {"value": rate, "unit": "TFLOP/s", "cores": host_threads(), "kind": "oracle",
               "sample": "oracle tile QR (NumPy FP64) of the first %d x %d rows/cols of the workload, "
                         "%.1f s" % (SAMPLE_M, N, secs)}
        if "batched" in extras:
            cpu["batched"] = oracle_batched(extras["batched"])
    for key in list(extras):
        if isinstance(extras[key], dict):
            extras[key] = {k: v for k, v in extras[key].items() if not k.startswith("_")}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_total / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME if M == WORKLOAD["M"] else "profiling_%dx%d" % (M, N),
                   **wl, "tasks": ntasks,
                   "l2": "inputs larger than L2 (A is %.2f GB)" % (M * N * 8 / 1e9),
                   "parallelism": "replicas" if world > 1 else "single"},
        "e2e": {"value": e2e_value, "unit": "TFLOP/s", "h2d_bytes_per_step": M * N * 8,
                "d2h_bytes_per_step": N * N * 8, "steps": k_e2e,
                "pipeline": "step k+1's host-to-device copy (copy stream, second buffer) overlaps step k",
                "h2d_gbs_alone": h2d_gbs},
        "gpu_launches": launches,
        "roofline": {"bound": "alu", "achieved": kern_tflops, "peak": peak, "unit": "TFLOP/s",
                     "frac": (kern_tflops / peak) if peak else None, "traffic": traffic,
                     "kernel": "hqr::hqr_sched<double>",
                     "peak_source": "FP64 cuBLAS DGEMM 8192^3 measured in this run (best of 3); "
                                    "no FP64 entry in MEASURED_PEAKS.json",
                     "fp64_pipe_tflops": {"dfma": pipes[0], "dmma": pipes[1],
                                          "from": "hqr_fp64_pipe_rates: register-only DFMA / DMMA loops"},
                     "traffic_note": traffic_note},
        "clocks": clk.summary(),
        "cpu_baseline": cpu,
        "accuracy": {"max_rel_colnorm_err_R_vs_A": cn_err},
        "extras": extras,
        "setup_s": t_setup,
    }
    print(json.dumps(line, default=lambda o: None))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
