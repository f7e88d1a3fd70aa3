"""Seeded request inputs drawn directly on the GPU (for the served workload).

Same families as the numpy generators in ``workloads`` -- shifted 2D
5-point Laplacians and random banded SPD matrices, Z ~ N(0,1) -- but built
with torch on the device so that a stream of tens of thousands of requests
with up to 10^6 rows can be materialised at admission time.  Each array
comes from its own torch generator seeded with (seed, request, tag).
Nothing here performs the method's arithmetic.
"""
from __future__ import annotations

import torch


def _gen(device, seed: int, req: int, tag: int) -> torch.Generator:
    g = torch.Generator(device=device)
    g.manual_seed((seed * 1_000_003 + req * 7919 + tag) % (2**63 - 1))
    return g


def _compact(cols, vals, mask, nnz: int, device):
    """CSR arrays from per-row candidate entries (columns ascending within a
    row) keeping the entries where ``mask`` holds, in row-major order -- what
    ``cols[mask]`` gives -- without waiting for the device: the caller knows
    ``nnz`` in closed form, every kept entry goes to rowptr[row] + its rank
    among the row's kept entries, and every dropped one to a spare slot past
    the end."""
    m = cols.shape[0]
    counts = mask.sum(dim=1)
    rowptr = torch.zeros(m + 1, device=device, dtype=torch.int64)
    rowptr[1:] = torch.cumsum(counts, 0)
    rank = torch.cumsum(mask.to(torch.int64), dim=1) - 1
    pos = torch.where(mask, rowptr[:-1, None] + rank, torch.full_like(rank, nnz)).reshape(-1)
    col = torch.empty(nnz + 1, device=device, dtype=torch.int32)
    val = torch.empty(nnz + 1, device=device, dtype=torch.float64)
    col.scatter_(0, pos, cols.reshape(-1).to(torch.int32))
    val.scatter_(0, pos, vals.reshape(-1).to(torch.float64))
    return rowptr.to(torch.int32), col[:nnz], val[:nnz]


def laplace2d_csr(side: int, shift: float, device):
    """5-point Laplacian (diag 4 + shift, neighbours -1, Dirichlet) on side x side,
    row k = ix + side*iy; returns (rowptr, col, val) on the device."""
    m = side * side
    k = torch.arange(m, device=device, dtype=torch.int64)
    ix, iy = k % side, k // side
    cols = torch.stack([k - side, k - 1, k, k + 1, k + side], dim=1)
    vals = torch.tensor([-1.0, -1.0, 4.0 + shift, -1.0, -1.0], device=device, dtype=torch.float64).expand(m, 5)
    mask = torch.stack([iy > 0, ix > 0, torch.ones_like(ix, dtype=torch.bool), ix < side - 1, iy < side - 1], dim=1)
    return _compact(cols, vals.contiguous(), mask, 5 * m - 4 * side, device)


def banded_spd_csr(m: int, hb: int, gen: torch.Generator, device):
    """Upper band U(-1,1) mirrored; diagonal 1 + row |off-diagonal| sum."""
    k = torch.arange(m, device=device, dtype=torch.int64)
    d = torch.arange(1, hb + 1, device=device, dtype=torch.int64)
    up = torch.rand((m, hb), generator=gen, device=device, dtype=torch.float64) * 2.0 - 1.0
    upmask = (k[:, None] + d[None, :]) < m
    up = torch.where(upmask, up, torch.zeros_like(up))
    lo = torch.zeros_like(up)
    for dd in range(1, min(hb, m - 1) + 1):
        lo[dd:, dd - 1] = up[: m - dd, dd - 1]
    lomask = (k[:, None] - d[None, :]) >= 0
    diag = 1.0 + up.abs().sum(dim=1) + lo.abs().sum(dim=1)
    cols = torch.cat([k[:, None] - d.flip(0)[None, :], k[:, None], k[:, None] + d[None, :]], dim=1)
    vals = torch.cat([lo.flip(1), diag[:, None], up], dim=1)
    mask = torch.cat([lomask.flip(1), torch.ones((m, 1), dtype=torch.bool, device=device), upmask], dim=1)
    nnz = m + 2 * sum(m - dd for dd in range(1, min(hb, m - 1) + 1))
    return _compact(cols, vals, mask, nnz, device)


def request_inputs(kind: str, m: int, n: int, seed: int, req: int, device):
    """(A, Z, m) for one request: ``kind`` 'laplace' (side = round(sqrt(m)),
    actual m = side^2, shift 0.01) or 'banded' (half-bandwidth 8).  Z is
    column-major (an (n, m) row-major buffer viewed transposed)."""
    if kind == "laplace":
        side = max(int(round(m ** 0.5)), 2)
        A = laplace2d_csr(side, 0.01, device)
        m = side * side
    else:
        A = banded_spd_csr(m, 8, _gen(device, seed, req, 3), device)
    n = min(n, m)
    Z = torch.randn((n, m), generator=_gen(device, seed, req, 1), device=device, dtype=torch.float64).T
    return A, Z, m
