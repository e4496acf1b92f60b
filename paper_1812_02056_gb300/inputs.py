"""Seeded synthetic inputs for the blocked Cholesky / pivot-free LU workloads.

This module draws random numbers and assembles test matrices; it performs no
step of the factorization or of the solves. The CUDA path, the CPU oracle,
the tests and the benchmark all take their matrices from here, so both sides
of every parity check read the same bytes.

Workloads (all FP64, row-major, exactly symmetric where SPD):

* ``spd_gram(n, seed)``: ``A = G G^T + n I`` with ``G`` iid N(0, 1).  This
  stands in for the paper's test matrix, "symmetric with random entries and
  large values on the diagonal" (Sec. 2, timing paragraph), whose
  distribution the paper does not state.
* ``lu_diag_dominant(n, seed)``: iid U(-1, 1) plus ``n I``; strictly
  diagonally dominant by rows and columns, so every leading principal minor
  is nonzero, as Algorithm 2 requires of its input.
* ``spd_logspaced(n, seed, cond)``: ``Q diag(sigma) Q^T`` with ``sigma``
  log-spaced on ``[1, cond]`` and ``Q`` the orthogonal factor of a QR of an
  iid Gaussian matrix (columns sign-normalised so ``Q`` is unique).
* ``pascal_sym(n)`` / ``pascal_lower(n)``: the symmetric Pascal matrix
  ``P_ij = C(i+j, i)`` and the lower Pascal matrix ``C(i, j)``; the former
  equals the latter times its transpose (Vandermonde's identity), a closed
  form used to pin both implementations exactly.
* ``rhs(n, nrhs, seed)``: iid N(0, 1) right-hand sides, row-major ``n x nrhs``.
* ``batch_sizes`` / ``served_requests``: size mixes for the batched and
  served workloads.

Seeds follow ``SEED_BASE + 100 * workload_index + matrix_index``.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 1812020560

# workload indices used to derive seeds
W_SMALL = 0       # FP64 Cholesky n=512, s=32
W_N8192 = 1       # FP64/FP32 Cholesky and pivot-free LU at n=8192
W_MIXED = 2       # mixed precision at n=16384
W_BATCHED = 3     # 10,000 matrices, n in [16, 512]
W_SERVED = 4      # served request stream


def seed_for(workload: int, index: int = 0) -> int:
    return SEED_BASE + 100 * workload + index


def rng(seed: int) -> np.random.Generator:
    """Counter-based Philox stream for ``seed``."""
    return np.random.Generator(np.random.Philox(seed))


def _mirror_lower(A):
    """Make ``A`` exactly symmetric by copying its lower triangle upward."""
    if isinstance(A, np.ndarray):
        L = np.tril(A)
        return L + np.tril(A, -1).T
    import torch
    L = torch.tril(A)
    return L + torch.tril(A, -1).T


def gaussian(rows: int, cols: int, seed: int) -> np.ndarray:
    return rng(seed).standard_normal((rows, cols))


def spd_gram(n: int, seed: int, device: str | None = None):
    """``G G^T + n I`` (FP64).  ``device`` other than None/'cpu' forms the
    product with torch on that device and returns a torch tensor there."""
    G = gaussian(n, n, seed)
    if device is None or device == "cpu":
        A = _mirror_lower(G @ G.T)
        A[np.diag_indices(n)] += float(n)
        return A
    import torch
    Gd = torch.from_numpy(G).to(device)
    A = _mirror_lower(Gd @ Gd.T)
    A.diagonal().add_(float(n))
    return A


def lu_diag_dominant(n: int, seed: int) -> np.ndarray:
    """iid U(-1, 1) entries plus ``n I``."""
    A = rng(seed).uniform(-1.0, 1.0, size=(n, n))
    A[np.diag_indices(n)] += float(n)
    return A


def spd_logspaced(n: int, seed: int, cond: float = 1e4, device: str | None = None):
    """``Q diag(sigma) Q^T``, ``sigma_i = cond**(i/(n-1))``, ``Q`` from QR of an
    iid Gaussian matrix with the sign of each column fixed by ``diag(R) > 0``."""
    G = gaussian(n, n, seed)
    sigma = cond ** (np.arange(n, dtype=np.float64) / max(n - 1, 1))
    if device is None or device == "cpu":
        Q, R = np.linalg.qr(G)
        Q = Q * np.sign(np.diag(R))[None, :]
        return _mirror_lower((Q * sigma[None, :]) @ Q.T)
    import torch
    Gd = torch.from_numpy(G).to(device)
    Q, R = torch.linalg.qr(Gd)
    Q = Q * torch.sign(torch.diagonal(R))[None, :]
    s = torch.from_numpy(sigma).to(device)
    return _mirror_lower((Q * s[None, :]) @ Q.T)


def pascal_sym(n: int) -> np.ndarray:
    """Symmetric Pascal matrix ``C(i+j, i)`` (exact in FP64 for n <= 27)."""
    return np.array([[float(math.comb(i + j, i)) for j in range(n)] for i in range(n)])


def pascal_lower(n: int) -> np.ndarray:
    """Lower Pascal matrix ``C(i, j)``."""
    return np.array([[float(math.comb(i, j)) for j in range(n)] for i in range(n)])


def unit_lower_integer(n: int, seed: int, lo: int = -2, hi: int = 2) -> np.ndarray:
    """Unit-diagonal lower-triangular matrix with small integer entries."""
    L = rng(seed).integers(lo, hi + 1, size=(n, n)).astype(np.float64)
    L = np.tril(L, -1)
    L[np.diag_indices(n)] = 1.0
    return L


def small_int_spd(n: int, seed: int, lo: int = -3, hi: int = 3) -> np.ndarray:
    """``B B^T + n I`` with small integer ``B``: an SPD matrix of integers."""
    B = rng(seed).integers(lo, hi + 1, size=(n, n)).astype(np.float64)
    A = B @ B.T
    A[np.diag_indices(n)] += float(n)
    return A


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """iid N(0, 1) right-hand sides, row-major ``n x nrhs``."""
    return rng(seed).standard_normal((n, nrhs))


def batch_sizes(count: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """``count`` integer sizes uniform on ``[lo, hi]``."""
    return rng(seed).integers(lo, hi + 1, size=count).astype(np.int64)


def batch_spd(sizes, seed: int) -> list[np.ndarray]:
    """One ``G G^T + n I`` per size, matrix ``i`` seeded with ``seed + i``."""
    return [spd_gram(int(n), seed + i) for i, n in enumerate(sizes)]


def served_requests(count: int, seed: int, n_lo: int = 32, n_hi: int = 8192,
                    nrhs_hi: int = 64, rate_hz: float = 100.0):
    """Poisson arrivals: returns (arrival_s, n, nrhs) arrays; ``n`` is
    log-uniform on ``[n_lo, n_hi]`` and ``nrhs`` uniform on ``[1, nrhs_hi]``."""
    g = rng(seed)
    gaps = g.exponential(1.0 / rate_hz, size=count)
    arrival = np.cumsum(gaps)
    logn = g.uniform(math.log(n_lo), math.log(n_hi), size=count)
    n = np.clip(np.round(np.exp(logn)).astype(np.int64), n_lo, n_hi)
    nrhs = g.integers(1, nrhs_hi + 1, size=count).astype(np.int64)
    return arrival, n, nrhs


def batch_spd_device(sizes, seed: int, device, dtype=None):
    """Many SPD matrices ``G G^T + n I`` (G iid N(0, 1), drawn by torch's
    seeded Philox on ``device``), packed back to back in one flat buffer:
    returns ``(buf, offsets)`` with matrix ``i`` at
    ``buf[offsets[i] : offsets[i] + n_i * n_i]`` (row-major, ``ld = n_i``).
    Matrices of the same order are generated together."""
    import torch
    dtype = dtype or torch.float64
    sizes = np.asarray(sizes, dtype=np.int64)
    offs = np.zeros(len(sizes), dtype=np.int64)
    if len(sizes) > 1:
        offs[1:] = np.cumsum(sizes ** 2)[:-1]
    total = int((sizes ** 2).sum())
    buf = torch.empty(max(total, 1), dtype=dtype, device=device)
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    for n in np.unique(sizes):
        n = int(n)
        idx = np.nonzero(sizes == n)[0]
        for c0 in range(0, len(idx), 2048):
            part = idx[c0:c0 + 2048]
            G = torch.randn((len(part), n, n), generator=g, device=device, dtype=torch.float64)
            A = G @ G.transpose(1, 2)
            A = torch.tril(A) + torch.tril(A, -1).transpose(1, 2)
            A.diagonal(dim1=1, dim2=2).add_(float(n))
            A = A.to(dtype).reshape(len(part), n * n)
            for j, i in enumerate(part):
                buf[offs[i]:offs[i] + n * n] = A[j]
    return buf, offs
