"""Seeded synthetic inputs shaped like the paper's workloads (Sec. 6.1.1).

This module holds no step of the NMF method: it only draws matrices.  Both the
tests (for the CUDA path and the FP64 oracle) and ``bench.py`` take their
inputs from here, so each side sees identical data.

Recipes (the design notes list them with their sizes):

* ``dense_lowrank``: A = W* H* + |N(0, sigma^2)| with W* (m x r) and H* (r x n)
  uniform on [0, 1) and sigma = 0.01 (standard deviation, absolute value taken
  entrywise).  The paper's dense synthetic matrix is the noise-free product of
  two uniform factors (Sec. 6.1.1); the noise makes the residual nonzero.
* ``init_factors``: W0 (m x k) and H0 (k x n) uniform on [0, 1) -- the same
  seed gives the same H0 for every algorithm, as in Sec. 6.1.3.
* ``sparse_uniform``: CSR with entries nonzero at uniformly random positions
  (Erdos-Renyi, as the paper's sparse synthetic matrix, Sec. 6.1.1) with
  values uniform on (0, 1].
* ``dense_lowrank_torch``: the dense recipe drawn on a torch device in FP32,
  row block by row block, for sizes too large to draw on the host.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def dense_lowrank(m: int, n: int, r: int, seed: int, sigma: float = 0.01, noise: bool = True):
    """Returns (A, W*, H*) in float64."""
    g = _rng(seed)
    Ws = g.random((m, r))
    Hs = g.random((r, n))
    A = Ws @ Hs
    if noise and sigma > 0:
        A += np.abs(g.normal(0.0, sigma, size=(m, n)))
    return A, Ws, Hs


def dense_lowrank_blocked(m: int, n: int, r: int, seed: int, sigma: float = 0.01,
                          block_rows: int = 4096):
    """The dense recipe in float64 for sizes whose one-shot draw would need
    several times A's memory: W* and H* drawn first, then A filled row block
    by row block (W* H* + |N(0, sigma^2)| per block) from the same
    generator, so the extra memory is one block.  The numbers differ from
    ``dense_lowrank``'s for the same seed; the distribution is the same."""
    g = _rng(seed)
    Ws = g.random((m, r))
    Hs = g.random((r, n))
    A = np.empty((m, n))
    for r0 in range(0, m, block_rows):
        r1 = min(m, r0 + block_rows)
        np.matmul(Ws[r0:r1], Hs, out=A[r0:r1])
        if sigma > 0:
            A[r0:r1] += np.abs(g.normal(0.0, sigma, size=(r1 - r0, n)))
    return A, Ws, Hs


def init_factors(m: int, n: int, k: int, seed: int):
    """(W0, H0) uniform on [0, 1), float64; H0 is drawn first so that it does not
    depend on m."""
    g = _rng(seed + 7919)
    H0 = g.random((k, n))
    W0 = g.random((m, k))
    return W0, H0


def sparse_uniform(m: int, n: int, density: float, seed: int):
    """CSR (indptr int64, indices int32, data float64) with each row holding a
    Binomial(n, density) number of distinct, uniformly placed columns; values
    uniform on (0, 1].  Returns (indptr, indices, data)."""
    g = _rng(seed)
    counts = g.binomial(n, density, size=m).astype(np.int64)
    nnz = int(counts.sum())
    rows = np.repeat(np.arange(m, dtype=np.int64), counts)
    cols = g.integers(0, n, size=nnz, dtype=np.int64)
    key = np.unique(rows * n + cols)  # sorted by (row, col); drops rare repeats
    rows = key // n
    cols = (key % n).astype(np.int32)
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=indptr[1:])
    data = 1.0 - g.random(key.shape[0])  # (0, 1]
    return indptr, cols, data


def dense_lowrank_torch(m: int, n: int, r: int, seed: int, device, sigma: float = 0.01,
                        out=None, block_rows: int = 8192):
    """FP32 A = W* H* + |N(0, sigma^2)| drawn on ``device`` with torch's
    generator (a different stream of numbers than ``dense_lowrank``).
    Returns (A, W*, H*); ``out`` (m x n, float32) is filled when given."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    Ws = torch.rand((m, r), generator=g, device=device, dtype=torch.float32)
    Hs = torch.rand((r, n), generator=g, device=device, dtype=torch.float32)
    A = out if out is not None else torch.empty((m, n), device=device, dtype=torch.float32)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for r0 in range(0, m, block_rows):
            r1 = min(m, r0 + block_rows)
            blk = A[r0:r1]
            torch.matmul(Ws[r0:r1], Hs, out=blk)
            if sigma > 0:
                blk.add_(torch.randn((r1 - r0, n), generator=g, device=device,
                                     dtype=torch.float32).abs_().mul_(sigma))
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    return A, Ws, Hs


def init_factors_torch(m: int, n: int, k: int, seed: int, device):
    """(W0, H0) uniform on [0, 1), float32, drawn on ``device``."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed) + 7919)
    H0 = torch.rand((k, n), generator=g, device=device, dtype=torch.float32)
    W0 = torch.rand((m, k), generator=g, device=device, dtype=torch.float32)
    return W0, H0


def sparse_uniform_torch(m: int, n: int, density: float, seed: int, device):
    """CSR on ``device``: round(m n density) positions drawn uniformly with
    replacement (repeats dropped), values uniform on (0, 1].  Returns
    (rowptr int64, colidx int32, val float32)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    nnz = int(round(m * n * density))
    key = torch.randint(0, m * n, (nnz,), generator=g, device=device, dtype=torch.int64)
    key = torch.unique(key)  # sorted by (row, col)
    rows = key // n
    cols = (key % n).to(torch.int32)
    counts = torch.bincount(rows, minlength=m)
    rowptr = torch.zeros(m + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=rowptr[1:])
    val = 1.0 - torch.rand(key.shape[0], generator=g, device=device, dtype=torch.float32)
    return rowptr, cols.contiguous(), val


def _powerlaw_ranks(count: int, size: int, a: float, g, device):
    """`count` ranks in [0, size) with P(rank = i) ~ (i + 1)^-a (0 < a < 1),
    by inverse-transform sampling of the continuous density."""
    import torch

    u = torch.rand(count, generator=g, device=device, dtype=torch.float64)
    top = (size + 1.0) ** (1.0 - a) - 1.0
    x = torch.pow(1.0 + u * top, 1.0 / (1.0 - a)) - 1.0
    return torch.clamp(x.to(torch.int64), max=size - 1)


def _spread(rank, size: int, mult: int):
    """A bijection of [0, size) (multiplication by a number coprime to size),
    so that the high-degree ranks land at scattered indices."""
    return (rank * mult) % size


def _coprime(size: int, start: int) -> int:
    import math

    c = start
    while math.gcd(c, size) != 1:
        c += 1
    return c


def sparse_powerlaw_torch(m: int, n: int, nnz: int, seed: int, device, a_rows: float = 0.5,
                          a_cols: float = 0.7):
    """CSR on ``device`` with power-law row and column degrees (a stand-in for
    a web graph such as webbase-2001): `nnz` (row, column) pairs drawn with
    independent power-law ranks (row rank i with probability ~ (i+1)^-a_rows,
    column ranks with a_cols), the ranks spread over the indices by a fixed
    bijection, repeated positions dropped; values uniform on (0, 1].  Returns
    (rowptr int64, colidx int32, val float32)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    rows = _spread(_powerlaw_ranks(nnz, m, a_rows, g, device), m, _coprime(m, 2654435761 % m or 1))
    cols = _spread(_powerlaw_ranks(nnz, n, a_cols, g, device), n, _coprime(n, 40503 * 65537 % n or 1))
    key = rows * n + cols
    del rows, cols
    key = torch.unique(key)  # sorted by (row, col)
    rows = key // n
    colidx = (key % n).to(torch.int32)
    del key
    counts = torch.bincount(rows, minlength=m)
    del rows
    rowptr = torch.zeros(m + 1, dtype=torch.int64, device=device)
    torch.cumsum(counts, 0, out=rowptr[1:])
    val = 1.0 - torch.rand(colidx.shape[0], generator=g, device=device, dtype=torch.float32)
    return rowptr, colidx.contiguous(), val

