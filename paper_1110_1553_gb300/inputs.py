"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU
oracle's checks. Random numbers only: nothing of the factorization.

Matrices follow the workloads of the paper's experiments (Sec. 5: tall-skinny
M x 4480 and square matrices), with i.i.d. N(0, 1) entries; the paper does
not state a value distribution. Generators are NumPy's Philox bit generator
(counter-based, Salmon et al. 2011) seeded by (seed, stream id), so each
named input is reproducible on any machine with the same NumPy.
"""
import numpy as np

BASE_SEED = 11101553


def rng(seed, stream=0):
    return np.random.Generator(np.random.Philox(key=[BASE_SEED + int(seed), int(stream)]))


def gaussian(M, N, seed, stream=0):
    """M x N float64 matrix of i.i.d. N(0, 1) entries (Fortran order)."""
    return np.asfortranarray(rng(seed, stream).standard_normal((M, N)))


def gaussian_torch(M, N, seed, device="cuda"):
    """M x N float64 N(0, 1) matrix generated on the device (column-major
    storage), for workloads too large to draw on the host quickly."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(BASE_SEED + int(seed))
    return torch.randn((N, M), dtype=torch.float64, device=device, generator=g).t()
