"""Named single runs of the library's workloads, for profilers and quick
checks: each builds its seeded synthetic input, runs the operation once
(after one untimed run unless --once), prints one line and exits 0.

    python -m paper_1110_1553_gb300.cases fp64_tall_skinny --rows 16384
    python -m paper_1110_1553_gb300.cases fp32_tc_square --n 6144
    python -m paper_1110_1553_gb300.cases fp32_tc_ls --n 4096 --iters 16

Cases:
  fp64_tall_skinny  FP64 HQR of rows x 2048 (nb 256, ib 32, a 4, p 16,
                    greedy / Fibonacci), the benchmark's configuration
                    (--domino: with the coupling level of Sec. 4.2)
  fp32_tc_square    FP32 tile QR of n x n on the tensor-core kernels
                    (nb 128, a 16, greedy / greedy)
  fp32_cc_square    the same on the CUDA-core FP32 kernels (ib 16)
  fp32_tc_ls        least squares n x n, kappa 1e6, tensor-core QR + FP64
                    corrected semi-normal-equation refinement
  fp64_latency      512 x 512 FP64 QR (nb 64, ib 16, flat TS a = 8) and Q
                    applied to I, with a per-task breakdown of the
                    factorization (engine timestamps): task types, critical
                    path by measured durations, gaps along it
                    (--whole: whole panel tasks instead of split panels)
"""
import argparse
import time


def latency_breakdown(torch, hqr, inputs, dev, whole):
    """The 512 x 512 FP64 QR + Q I case with a per-task breakdown printed."""
    import numpy as np
    names = {0: "GEQRT", 1: "UNMQR", 2: "TSQRT", 3: "TSMQR", 4: "TTQRT", 5: "TTMQR"}
    if whole:
        hqr.set_panel_split(0)
    A = inputs.gaussian_torch(512, 512, seed=11, device=dev)
    recs = hqr.elim_list(8, 8, 8, 1, "flat", "flat")
    F = hqr.geqrf(A, 64, 16, recs)
    I = torch.eye(512, dtype=torch.float64, device=dev)
    Q = I.clone().t().contiguous().t()
    for _ in range(3):
        F.refactor(A)
        Q.copy_(I)
        F.apply_q(Q, trans=False)
    F.refactor(A)
    fk = F.kernel_ms()
    Q.copy_(I)
    F.apply_q(Q, trans=False)
    ak = F.kernel_ms()
    F.trace(True)
    F.refactor(A)
    tr = F.trace().astype(np.int64)
    F.trace(False)
    tasks, ptr, succ = hqr.task_graph(8, 8, 64, 16, recs, kind="factor")  # the same graph (same settings)
    hqr.set_panel_split(64)
    dur = (tr[:, 1] - tr[:, 0]) / 1e3
    for o in sorted(set(tasks[:, 0].tolist())):
        sel = tasks[:, 0] == o
        print("  %-6s count %5d mean %7.2f us" % (names[o], sel.sum(), dur[sel].mean()))
    nt = len(tr)
    bl = np.zeros(nt)
    for q in range(nt - 1, -1, -1):
        s = succ[ptr[q]:ptr[q + 1]]
        bl[q] = dur[q] + (bl[s].max() if len(s) else 0.0)
    q, gap, hops = int(np.argmax(bl)), 0.0, 0
    while True:
        s = succ[ptr[q]:ptr[q + 1]]
        if len(s) == 0:
            break
        nxt = int(s[np.argmax(bl[s])])
        gap += max(0, tr[nxt, 0] - tr[q, 1]) / 1e3
        hops += 1
        q = nxt
    makespan = (tr[:, 1].max() - tr[:, 0].min()) / 1e3
    return ("factor kernel %.3f ms (%d tasks), apply-Q kernel %.3f ms; traced makespan %.1f us, critical path "
            "by task durations %.1f us over %d hops, %.1f us of gaps along it" % (fk, len(tr), ak, makespan, bl.max(),
                                                                               hops, gap))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["fp64_tall_skinny", "fp32_tc_square", "fp32_cc_square", "fp32_tc_ls",
                                     "fp64_latency"])
    ap.add_argument("--whole", action="store_true", help="fp64_latency: whole panel tasks")
    ap.add_argument("--rows", type=int, default=131072)
    ap.add_argument("--n", type=int, default=6144)
    ap.add_argument("--iters", type=int, default=16)
    ap.add_argument("--once", action="store_true", help="no untimed first run")
    ap.add_argument("--domino", action="store_true", help="fp64_tall_skinny: list with the coupling level (Sec. 4.2)")
    a = ap.parse_args(argv)
    import torch

    from paper_1110_1553_gb300 import _build, hqr, inputs, workloads
    _build.build()
    hqr.load()
    dev = torch.device("cuda", 0)
    runs = 1 if a.once else 2
    t0 = time.perf_counter()
    if a.case == "fp64_tall_skinny":
        M, N, nb = a.rows, 2048, 256
        A = inputs.gaussian_torch(M, N, seed=1, device=dev)
        recs = hqr.elim_list(M // nb, N // nb, 4, 16, "greedy", "fibonacci", domino=a.domino)
        F = hqr.geqrf(A, nb, 32, recs)
        for _ in range(runs - 1):
            F.refactor(A)
        info = "kernel %.2f ms" % F.kernel_ms()
    elif a.case in ("fp32_tc_square", "fp32_cc_square"):
        n, tensor = a.n, a.case == "fp32_tc_square"
        g = torch.Generator(device=dev)
        g.manual_seed(3)
        A = torch.randn((n, n), dtype=torch.float32, device=dev, generator=g).t()
        recs = hqr.elim_list(n // 128, n // 128, 16, 1, "greedy", "greedy")
        F = hqr.geqrf(A, 128, 128 if tensor else 16, recs, tensor=tensor)
        for _ in range(runs - 1):
            F.refactor(A)
        info = "kernel %.2f ms" % F.kernel_ms()
    elif a.case == "fp64_latency":
        info = latency_breakdown(torch, hqr, inputs, dev, a.whole)
    else:
        n = a.n
        A = workloads.conditioned(torch, n, n, 1e6, seed=30, device=dev)
        b = A.double() @ torch.ones(n, dtype=torch.float64, device=dev)
        x = torch.zeros(n, dtype=torch.float64, device=dev)
        plan = hqr.LSPlan([(A, b, x)], refine_iters=a.iters, configs=[hqr.tile_config(128, 128, 16, 1)],
                          tensor=True)
        for _ in range(runs):
            plan.run()
        st = plan.status()
        info = "status %d, |x - 1|_max %.2e" % (st, (x - 1).abs().max().item())
    torch.cuda.synchronize()
    print("%s: %s (%.2f s)" % (a.case, info, time.perf_counter() - t0))
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
