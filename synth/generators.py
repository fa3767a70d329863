"""Seeded generators for the test matrices of the paper (Section 3) and the extra workloads.

* ``randsvd``: dense A = U diag(sigma) V^T with Haar-random orthogonal U, V and
  geometrically distributed singular values sigma_i = kappa^(-(i-1)/(n-1))
  (the "mode 3" random dense matrices of Section 3), so kappa_2(A) = kappa.
* ``prolate``: symmetric Toeplitz matrix with a_0 = 2w, a_j = sin(2 pi w j)/(pi j)
  (the prolate matrices of Section 3 / Table 4).
* ``convdiff``: dense matrix of the 5-point first-order-upwind discretisation of
  -Lap(u) + beta . grad(u) on the unit square with zero Dirichlet data.
* ``batch_specs``: sizes and condition numbers of a batch of uneven systems.

Everything is FP64. No function here solves anything.
"""
from __future__ import annotations

import math

import numpy as np


def sigma_geometric(n: int, kappa: float) -> np.ndarray:
    """Singular values 1 = s_1 >= ... >= s_n = 1/kappa, geometrically spaced (randsvd mode 3)."""
    if n == 1:
        return np.ones(1)
    i = np.arange(n, dtype=np.float64)
    return kappa ** (-i / (n - 1))


def _haar(rng: np.random.Generator, n: int) -> np.ndarray:
    g = rng.standard_normal((n, n))
    q, r = np.linalg.qr(g)
    s = np.sign(np.diag(r))
    s[s == 0] = 1.0
    return q * s[None, :]


def randsvd(n: int, kappa: float, seed: int = 0) -> np.ndarray:
    """Dense FP64 randsvd matrix (numpy; intended for n up to a few thousand)."""
    rng = np.random.default_rng(seed)
    u = _haar(rng, n)
    v = _haar(rng, n)
    return (u * sigma_geometric(n, kappa)[None, :]) @ v.T


def randsvd_torch(n: int, kappa: float, seed: int = 0, device: str = "cuda"):
    """Large randsvd matrix built with torch on ``device`` (returns an FP64 torch tensor).

    The orthogonal factors come from an FP32 QR of Gaussian matrices (orthogonal to
    about 1e-5); by the multiplicative perturbation bound for singular values the
    singular values of the FP64 product U diag(sigma) V^T then equal sigma to that
    relative accuracy. The product itself is formed in FP64 so that the small
    singular values are not swamped by rounding of the entries.
    """
    import torch

    gen = torch.Generator(device=device)
    gen.manual_seed(seed)

    def haar32():
        g = torch.randn(n, n, generator=gen, device=device, dtype=torch.float32)
        q, r = torch.linalg.qr(g)
        s = torch.sign(torch.diagonal(r))
        s[s == 0] = 1.0
        return q * s[None, :]

    u = haar32().double()
    v = haar32().double()
    sig = torch.from_numpy(sigma_geometric(n, kappa)).to(device)
    a = (u * sig[None, :]) @ v.T
    del u, v
    return a.contiguous()


def prolate(n: int, w: float) -> np.ndarray:
    """Prolate Toeplitz matrix: a_0 = 2w, a_j = sin(2 pi w j) / (pi j)."""
    j = np.arange(1, n, dtype=np.float64)
    col = np.empty(n)
    col[0] = 2.0 * w
    col[1:] = np.sin(2.0 * np.pi * w * j) / (np.pi * j)
    idx = np.abs(np.arange(n)[:, None] - np.arange(n)[None, :])
    return col[idx]


def prolate_torch(n: int, w: float, device: str = "cuda"):
    """Prolate Toeplitz matrix built on ``device`` (FP64 torch tensor, same entries as ``prolate``)."""
    import torch

    j = np.arange(1, n, dtype=np.float64)
    col = np.empty(n)
    col[0] = 2.0 * w
    col[1:] = np.sin(2.0 * np.pi * w * j) / (np.pi * j)
    c = torch.from_numpy(col).to(device)
    idx = torch.arange(n, device=device)
    a = torch.empty(n, n, dtype=torch.float64, device=device)
    for r0 in range(0, n, 1024):
        r1 = min(n, r0 + 1024)
        a[r0:r1] = c[(idx[r0:r1, None] - idx[None, :]).abs()]
    return a


def convdiff(N: int = 100, peclet: float = 50.0) -> np.ndarray:
    """Dense FP64 matrix of -Lap(u) + beta.grad(u) on an N x N interior grid of the unit square.

    h = 1/(N+1), beta = (Pe, Pe)/sqrt(2) (so |beta| = Pe with unit diffusion and unit
    length), convection by first-order upwind (backward) differences, zero Dirichlet
    boundary, unknown (i, j) at index i*N + j, every row multiplied by h^2.
    """
    h = 1.0 / (N + 1)
    bx = by = peclet / math.sqrt(2.0)
    n = N * N
    a = np.zeros((n, n))
    for i in range(N):
        for j in range(N):
            r = i * N + j
            a[r, r] = 4.0 + h * (bx + by)
            if i > 0:
                a[r, r - N] = -1.0 - h * bx
            if i < N - 1:
                a[r, r + N] = -1.0
            if j > 0:
                a[r, r - 1] = -1.0 - h * by
            if j < N - 1:
                a[r, r + 1] = -1.0
    return a


def rhs_uniform(n: int, seed: int) -> np.ndarray:
    """b ~ U(0, 1)^n."""
    return np.random.default_rng(seed).random(n)


def normal_vector(n: int, seed: int) -> np.ndarray:
    """x ~ N(0, 1)^n."""
    return np.random.default_rng(seed).standard_normal(n)


def batch_specs(count: int, n_lo: int, n_hi: int, log_kappa_lo: float, log_kappa_hi: float,
                seed: int):
    """Sizes n_i ~ U{n_lo..n_hi} and condition numbers kappa_i = 10^U(lo, hi) of a batch."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, size=count)
    kap = 10.0 ** rng.uniform(log_kappa_lo, log_kappa_hi, size=count)
    return [int(v) for v in ns], [float(v) for v in kap]
