"""Writes the FP64 oracle solution of the square mixed-precision workload
(16384 x 16384, kappa 1e6; paper_1110_1553_gb300.workloads.square_mixed_problem)
for the benchmark's accuracy check.

The matrix is generated on the GPU by the seeded workload recipe (the input
generator only: random numbers, a library QR for the Haar factors and a
library product), copied to the host and solved there by the oracle alone:
the FP64 tile QR (Alg. 1 / Alg. 2, tiles of 512, flat TS domains of 4 tiles,
greedy trees) followed by three steps of Dot2-compensated augmented-system
refinement (oracle.lstsq). The solution is stored with SHA-256 fingerprints
of the FP32 matrix and the FP64 right-hand side, so that a run whose
generator produced different bits is detected instead of compared.

Usage: python tests/golden/make_square_mixed_oracle.py OUTDIR [n]
"""
import hashlib
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)


def fingerprints(A, b):
    """SHA-256 of the column-major FP32 bytes of A and of the FP64 bytes of b."""
    ha = hashlib.sha256(np.asfortranarray(A).tobytes(order="F")).hexdigest()
    hb = hashlib.sha256(np.ascontiguousarray(b).tobytes()).hexdigest()
    return ha, hb


def main():
    import torch

    from oracle.elim_list import GREEDY, hqr_elim_list
    from oracle.lstsq import lstsq
    from paper_1110_1553_gb300 import workloads
    out = sys.argv[1]
    n = int(sys.argv[2]) if len(sys.argv) > 2 else 16384
    A, b = workloads.square_mixed_problem(torch, n, device="cuda")
    A = A.cpu().numpy()
    b = b.cpu().numpy()
    ha, hb = fingerprints(A, b)
    nb, ib = 512, 32
    t0 = time.time()
    x, _ = lstsq(A.astype(np.float64), b, nb, ib, hqr_elim_list(n // nb, n // nb, 4, 1, GREEDY, GREEDY), refine=3)
    secs = time.time() - t0
    os.makedirs(out, exist_ok=True)
    np.save(os.path.join(out, "square_mixed_%d_oracle_x.npy" % n), x)
    meta = {"workload": "square_mixed_ls_%d_kappa1e6" % n, "n": n, "sha256_A_fp32_colmajor": ha,
            "sha256_b_fp64": hb, "oracle": "oracle.lstsq: FP64 tile QR nb %d ib %d (a 4, p 1, greedy/greedy) + "
            "3 Dot2 augmented-system refinement steps" % (nb, ib), "seconds": secs,
            "host_cores": os.cpu_count(), "torch": torch.__version__, "numpy": np.__version__}
    with open(os.path.join(out, "square_mixed_%d_oracle.json" % n), "w") as f:
        json.dump(meta, f, indent=1)
    print(json.dumps(meta))


if __name__ == "__main__":
    main()
