"""Seeded synthetic workloads of the benchmark (shapes and matrices only; no
factorization arithmetic). Recipes:

* tall-skinny FP64: 131072 x 2048, i.i.d. N(0, 1);
* square FP64 latency case: 512 x 512, i.i.d. N(0, 1);
* batched uneven: 1024 problems, M log-uniform in [64, 8192], N log-uniform in
  [32, 512], pairs with M < N rejected and redrawn (seed fixed), i.i.d. N(0, 1)
  FP32 entries, one FP64 N(0, 1) right-hand side each;
* square mixed-precision LS: A = U diag(s) V^T with U, V from the QR of
  Gaussian matrices (sign-fixed, Mezzadri 2007), s geometric from 1 to 1e-6,
  b = A x_true + 1e-8 N(0, 1);
* serving: Poisson arrivals, 90 % batched-like shapes, 10 % 32768 x 1024 FP32
  with geometric singular values from 1 to 1e-4 (kappa = 1e4).
"""
import numpy as np

from . import inputs


def uneven_shapes(count, seed=4, mmin=64, mmax=8192, nmin=32, nmax=512):
    rng = inputs.rng(seed, 0)
    out = []
    while len(out) < count:
        m = int(round(np.exp(rng.uniform(np.log(mmin), np.log(mmax)))))
        n = int(round(np.exp(rng.uniform(np.log(nmin), np.log(nmax)))))
        if m >= n:
            out.append((m, n))
    return out


def haar(torch, n, k, gen, device, dtype):
    """n x k matrix with orthonormal columns, Haar distributed (QR of a
    Gaussian with the signs of R's diagonal folded into Q)."""
    G = torch.randn((n, k), dtype=dtype, device=device, generator=gen)
    Q, R = torch.linalg.qr(G)
    return Q * torch.sign(torch.diagonal(R)).unsqueeze(0)


def conditioned(torch, M, N, kappa, seed, device="cuda", dtype=None):
    """A = U diag(s) V^T (M x N, column-major storage) with s geometric from 1
    to 1/kappa, generated in FP32 on the device."""
    dtype = dtype or torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(inputs.BASE_SEED + seed)
    U = haar(torch, M, N, gen, device, torch.float32)
    V = haar(torch, N, N, gen, device, torch.float32)
    s = torch.logspace(0, -np.log10(kappa), N, dtype=torch.float32, device=device)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    A = (U * s.unsqueeze(0)) @ V.t()
    torch.backends.cuda.matmul.allow_tf32 = prev
    return A.to(dtype).t().contiguous().t()


def square_mixed_problem(torch, n=16384, device="cuda"):
    """The square mixed-precision least-squares workload: A = U diag(s) V^T
    (FP32, n x n, s geometric from 1 to 1e-6, seed 30), x_true N(0, 1) and
    b = A x_true + 1e-8 N(0, 1) in FP64 (seed 31). Returns (A, b)."""
    A = conditioned(torch, n, n, 1e6, seed=30, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(31)
    xt = torch.randn(n, dtype=torch.float64, device=device, generator=g)
    b = A.double() @ xt + 1e-8 * torch.randn(n, dtype=torch.float64, device=device, generator=g)
    return A, b
