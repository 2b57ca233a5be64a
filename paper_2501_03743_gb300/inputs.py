"""Seeded synthetic workloads: SPD matrices in CSR form and right-hand sides.

This module only builds inputs.  It holds none of the solver's arithmetic and
is the one module shared by the CUDA library's tests and benchmark and by the
CPU oracle's tests.

Workloads (Section VI of the paper uses the Poisson equation on a cube with
Dirichlet boundary conditions; the other families are the synthetic
benchmark systems this library is measured on):

* ``poisson7(N)``  - 7-point finite-difference Laplacian on the N^3 interior
  nodes, lexicographic order ``row = i + N*(j + N*k)``, diagonal 6 and
  neighbours -1, boundary values eliminated (no h^2 factor).
* ``poisson27(N)`` - 27-point stencil, diagonal 26 and all 26 neighbours -1.
* ``batch_spec(count, seed)`` - a serving mix of independent systems:
  7- and 27-point stencils and variable-coefficient fields (sigma in
  {0.5, 1, 2, 3}) on grids drawn log-uniformly from 32^3 .. 160^3, each with
  1..8 right-hand sides.
* ``varcoef7(N, sigma, seed)`` - 7-point finite-volume discretisation of
  -div(k grad u) with k = exp(sigma * g), g a seeded Gaussian field smoothed
  with a Gaussian kernel of ``ell`` cells and normalised to mean 0 and
  variance 1.  Interior faces use the harmonic mean 2 k_p k_q / (k_p + k_q);
  a boundary face uses k_p, so k = 1 gives ``poisson7`` exactly.

Random numbers come from splitmix64 in counter form: the i-th draw for a seed
is the i-th output of the sequential generator started at state ``seed``,
``mix(seed + (i + 1) * 0x9E3779B97F4A7C15)``.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Draws ``offset .. offset+n-1`` of splitmix64 started at state ``seed``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int) -> np.ndarray:
    """U[-1, 1) with 53 random mantissa bits: 2 * (z >> 11) * 2^-53 - 1."""
    z = splitmix64(seed, n)
    return (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -52) - 1.0


def normal(seed: int, n: int) -> np.ndarray:
    """N(0, 1) by Box-Muller from draws 2i (radius) and 2i+1 (angle)."""
    z = splitmix64(seed, 2 * n)
    u1 = ((z[0::2] >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)  # (0, 1]
    u2 = (z[1::2] >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)          # [0, 1)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def _assemble(n: int, cols: np.ndarray, vals: np.ndarray):
    """Row-major (n, k) candidate columns (-1 = absent, sorted per row) -> CSR."""
    mask = cols >= 0
    counts = mask.sum(axis=1, dtype=np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    if rowptr[-1] >= 2 ** 31:
        raise ValueError("nnz does not fit int32 row pointers")
    col = cols[mask].astype(np.int32, copy=False)
    val = vals[mask].astype(np.float64, copy=False)
    return rowptr.astype(np.int32), col, val


def _stencil(N: int, offsets, weights):
    """Constant-coefficient stencil on the N^3 interior nodes, Dirichlet."""
    n = N ** 3
    order = sorted(range(len(offsets)), key=lambda t: offsets[t][0] * N * N + offsets[t][1] * N + offsets[t][2])
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    cols = np.empty((n, len(offsets)), dtype=np.int32)
    vals = np.empty((n, len(offsets)), dtype=np.float64)
    for c, t in enumerate(order):
        dz, dy, dx = offsets[t]
        ok = (x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N) & (z + dz >= 0) & (z + dz < N)
        cols[:, c] = np.where(ok, i + dx + N * (dy + N * dz), -1)
        vals[:, c] = weights[t]
    return _assemble(n, cols, vals)


_OFFS7 = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
_OFFS27 = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def poisson7(N: int):
    w = [6.0] + [-1.0] * 6
    return _stencil(N, _OFFS7, w)


def poisson27(N: int):
    offs = _OFFS27
    w = [26.0 if o == (0, 0, 0) else -1.0 for o in offs]
    return _stencil(N, offs, w)


def aniso7(N: int):
    """Anisotropic 7-point stencil: couplings -1, -2, -4 along x, y, z and the
    centre 14 (constant coefficients that are not all equal off the centre)."""
    w = [-(1.0 if o[2] else 2.0 if o[1] else 4.0) if o != (0, 0, 0) else 14.0 for o in _OFFS7]
    return _stencil(N, _OFFS7, w)


def smoothed_field(N: int, seed: int, ell: float = 4.0) -> np.ndarray:
    """Seeded N(0,1) noise on N^3 cells, Gaussian-smoothed (std ``ell`` cells,
    reflecting boundary, truncated at 3 std), normalised to mean 0, var 1.
    Returned flat in lexicographic order (x fastest)."""
    from scipy.ndimage import gaussian_filter

    g = normal(seed, N ** 3).reshape(N, N, N)  # [z, y, x]
    g = gaussian_filter(g, sigma=ell, mode="reflect", truncate=3.0)
    g = (g - g.mean()) / g.std()
    return g.reshape(-1)


def varcoef7(N: int, sigma: float, seed: int, ell: float = 4.0):
    """7-point finite-volume -div(k grad u), k = exp(sigma * g)."""
    n = N ** 3
    k = np.exp(sigma * smoothed_field(N, seed, ell)) if sigma != 0.0 else np.ones(n)
    i = np.arange(n, dtype=np.int64)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    offs = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 1), (0, 1, 0), (1, 0, 0)]  # (dz, dy, dx) sorted by column
    cols = np.full((n, 7), -1, dtype=np.int32)
    vals = np.zeros((n, 7), dtype=np.float64)
    diag = np.zeros(n, dtype=np.float64)
    slot = {o: c for c, o in enumerate([offs[0], offs[1], offs[2], None, offs[3], offs[4], offs[5]])}
    for o in offs:
        dz, dy, dx = o
        ok = (x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N) & (z + dz >= 0) & (z + dz < N)
        j = np.where(ok, i + dx + N * (dy + N * dz), 0)
        kq = k[j]
        face = np.where(ok, 2.0 * k * kq / (k + kq), k)
        diag += face
        c = slot[o]
        cols[:, c] = np.where(ok, j, -1)
        vals[:, c] = -face
    cols[:, 3] = i
    vals[:, 3] = diag
    return _assemble(n, cols, vals)


def matvec(rowptr, col, val, x):
    """y = A x through scipy (used only to form b = A x_true)."""
    import scipy.sparse as sp

    n = len(rowptr) - 1
    A = sp.csr_matrix((val, col, rowptr), shape=(n, n))
    return A @ x


def system(kind: str, N: int, seed: int = 0, sigma: float = 0.0, ell: float = 4.0):
    """One benchmark system: ``dict(rowptr, col, val, b, x_true, n)``.

    x_true ~ U[-1, 1) from ``seed``; b = A x_true in FP64.
    """
    if kind == "poisson7":
        rowptr, col, val = poisson7(N)
    elif kind == "poisson27":
        rowptr, col, val = poisson27(N)
    elif kind == "aniso7":
        rowptr, col, val = aniso7(N)
    elif kind == "varcoef7":
        rowptr, col, val = varcoef7(N, sigma, seed + 7919, ell)
    else:
        raise ValueError(kind)
    n = N ** 3
    x_true = uniform(seed, n)
    b = matvec(rowptr, col, val, x_true)
    return dict(rowptr=rowptr, col=col, val=val, b=b, x_true=x_true, n=n)


def closed_form_bounds(kind: str, N: int):
    """Extreme eigenvalues of A for the constant-coefficient stencils
    (tensor-product sine modes): 7-point 6 -/+ 6 cos(pi/(N+1));
    27-point 27 - (1+2c)^3 and 27 + (1+2c)^2 (2c-1), c = cos(pi/(N+1))."""
    c = np.cos(np.pi / (N + 1))
    if kind == "poisson7":
        return 6.0 - 6.0 * c, 6.0 + 6.0 * c
    if kind == "poisson27":
        return 27.0 - (1.0 + 2.0 * c) ** 3, 27.0 + (1.0 + 2.0 * c) ** 2 * (2.0 * c - 1.0)
    raise ValueError(kind)


def batch_spec(count: int, seed: int = 2025, nmin: int = 32, nmax: int = 160):
    """Seeded serving mix: ``count`` dicts (kind, N, sigma, field_seed, nrhs).

    Draws 4k..4k+3 of splitmix64(seed) pick, for system k: the kind
    (poisson7, poisson27, varcoef7 twice as likely as each), the grid edge N
    = round(nmin (nmax/nmin)^u) (log-uniform), sigma in {0.5, 1, 2, 3} and
    1..8 right-hand sides."""
    u = (uniform(seed, 4 * count) + 1.0) / 2.0  # [0, 1)
    kinds = ("poisson7", "poisson27", "varcoef7", "varcoef7")
    out = []
    for k in range(count):
        a, b, c, d = u[4 * k:4 * k + 4]
        out.append(dict(kind=kinds[int(a * 4)], N=int(round(nmin * (nmax / nmin) ** b)),
                        sigma=(0.5, 1.0, 2.0, 3.0)[int(c * 4)], field_seed=1000 + k, nrhs=1 + int(d * 8)))
    return out


def batch_csr(spec: dict):
    """CSR arrays (rowptr, col, val) of one ``batch_spec`` entry."""
    if spec["kind"] == "varcoef7":
        return varcoef7(spec["N"], spec["sigma"], spec["field_seed"])
    if spec["kind"] == "poisson27":
        return poisson27(spec["N"])
    return poisson7(spec["N"])


def stencil_torch(kind: str, N: int, device="cuda"):
    """``poisson7`` / ``poisson27`` built with torch on `device`: the same
    CSR arrays (row order, column order, values) as the numpy builders,
    as int32 / int32 / float64 tensors.  For large serving mixes."""
    import torch

    offs = _OFFS7 if kind == "poisson7" else _OFFS27
    diag = 6.0 if kind == "poisson7" else 26.0
    n = N ** 3
    order = sorted(offs, key=lambda o: o[0] * N * N + o[1] * N + o[2])
    i = torch.arange(n, dtype=torch.int64, device=device)
    x, y, z = i % N, (i // N) % N, i // (N * N)
    cols = torch.empty((n, len(order)), dtype=torch.int32, device=device)
    vals = torch.empty((n, len(order)), dtype=torch.float64, device=device)
    for c, (dz, dy, dx) in enumerate(order):
        ok = (x + dx >= 0) & (x + dx < N) & (y + dy >= 0) & (y + dy < N) & (z + dz >= 0) & (z + dz < N)
        cols[:, c] = torch.where(ok, i + dx + N * (dy + N * dz), torch.full_like(i, -1)).to(torch.int32)
        vals[:, c] = diag if (dz, dy, dx) == (0, 0, 0) else -1.0
    mask = cols >= 0
    rowptr = torch.zeros(n + 1, dtype=torch.int64, device=device)
    torch.cumsum(mask.sum(dim=1), 0, out=rowptr[1:])
    return rowptr.to(torch.int32), cols[mask], vals[mask]
