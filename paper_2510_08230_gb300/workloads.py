"""Seeded synthetic inputs (matrices and vectors) shared by the tests, the
benchmark and the CPU oracle.

This module builds inputs only.  It performs none of the operations the
library computes (no products, conversions, reductions or solves): each
generator writes down a sparsity pattern and its values directly, in CSR
form with int32 indices and ascending columns inside each row.

The workloads stand in for the SuiteSparse matrices of the paper's
evaluation (Section 6, "Performance Results and Analysis"), which are not
available here.  Generators:

* ``laplacian_1d/2d/3d`` - Dirichlet finite-difference Laplacians
  (2 / 4 / 6 on the diagonal, -1 for every grid neighbour).
* ``power_law`` - random matrix with Zipf(a) row lengths, uniform random
  distinct columns and N(0,1) values.
* ``diffusion_3d`` - 7-point variable-coefficient diffusion with log-normal
  cell coefficients and harmonic-mean face coefficients.
* ``shifted_rectangle`` / ``batched_rectangles`` - 2D 5-point Laplacian on an
  a-by-b grid plus a scalar diagonal shift (many small SPD systems).
* ``banded_spd`` - symmetric banded matrix, off-diagonals U[-1,0], diagonal
  1.1 x absolute row sum (strictly diagonally dominant, hence SPD).
* ``random_csr`` / ``random_coo`` - small irregular matrices for edge cases.
* ``uniform_vector`` - U[-1,1] vectors.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64).
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "CSR", "laplacian_1d", "laplacian_2d", "laplacian_3d", "power_law",
    "diffusion_3d", "shifted_rectangle", "batched_rectangles", "banded_spd",
    "random_csr", "random_coo", "uniform_vector", "SEED_BASE",
]

# seed = SEED_BASE + workload index (1: 64x64 Laplacian, 2: SpMV sweep,
# 3: 128^3 diffusion, 4: batched rectangles, 5: serving mix)
SEED_BASE = 2510


class CSR:
    """A CSR matrix held in host numpy arrays (int32 indices)."""

    __slots__ = ("n", "ncols", "row_ptr", "col_idx", "values", "name")

    def __init__(self, n, ncols, row_ptr, col_idx, values, name=""):
        self.n = int(n)
        self.ncols = int(ncols)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.values = np.ascontiguousarray(values)
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.col_idx.shape[0])

    def row_lengths(self) -> np.ndarray:
        return np.diff(self.row_ptr.astype(np.int64))

    def astype(self, dtype) -> "CSR":
        return CSR(self.n, self.ncols, self.row_ptr, self.col_idx,
                   self.values.astype(dtype), self.name)

    def to_dense(self) -> np.ndarray:
        """Dense copy (small matrices only; used by the pins)."""
        d = np.zeros((self.n, self.ncols), dtype=np.float64)
        rows = np.repeat(np.arange(self.n), self.row_lengths())
        np.add.at(d, (rows, self.col_idx), self.values.astype(np.float64))
        return d


def _assemble(n, ncols, cols2d, vals2d, valid2d, name):
    """Row-major compaction of an (n, k) table of candidate entries."""
    counts = valid2d.sum(axis=1, dtype=np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    col = cols2d[valid2d]
    val = vals2d[valid2d]
    return CSR(n, ncols, row_ptr.astype(np.int32), col.astype(np.int32), val,
               name)


def _stencil(dims, name):
    """Dirichlet Laplacian on a box of shape dims (x fastest)."""
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    idx = np.arange(n, dtype=np.int64)
    coord = []
    rem = idx
    for d in dims:
        coord.append(rem % d)
        rem = rem // d
    # candidate offsets in ascending column order: -s_last ... -s_0, 0, s_0 ... s_last
    offs = []
    for ax in reversed(range(len(dims))):
        offs.append((ax, -1))
    offs.append((None, 0))
    for ax in range(len(dims)):
        offs.append((ax, +1))
    k = len(offs)
    cols = np.empty((n, k), dtype=np.int64)
    valid = np.empty((n, k), dtype=bool)
    vals = np.empty((n, k), dtype=np.float64)
    diag = 2.0 * len(dims)
    for j, (ax, sgn) in enumerate(offs):
        if ax is None:
            cols[:, j] = idx
            valid[:, j] = True
            vals[:, j] = diag
        else:
            cols[:, j] = idx + sgn * strides[ax]
            valid[:, j] = (coord[ax] + sgn >= 0) & (coord[ax] + sgn < dims[ax])
            vals[:, j] = -1.0
    return _assemble(n, n, cols, vals, valid, name)


def laplacian_1d(n: int) -> CSR:
    """Tridiagonal [-1 2 -1] on n points, Dirichlet boundary."""
    return _stencil((n,), f"lap1d_{n}")


def laplacian_2d(nx: int, ny: int | None = None) -> CSR:
    """5-point Laplacian (4 / -1) on an nx-by-ny grid, Dirichlet boundary."""
    ny = nx if ny is None else ny
    return _stencil((nx, ny), f"lap2d_{nx}x{ny}")


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None) -> CSR:
    """7-point Laplacian (6 / -1) on an nx-by-ny-by-nz grid, Dirichlet."""
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    if nx * ny * nz >= 2 ** 22:
        return _stencil_3d_large(nx, ny, nz)
    return _stencil((nx, ny, nz), f"lap3d_{nx}x{ny}x{nz}")


def _stencil_3d_large(nx, ny, nz):
    """Same matrix as ``_stencil`` for 3D, built plane by plane (bounded
    temporaries for 256^3 and larger)."""
    n = nx * ny * nz
    plane = nx * ny
    # rows of one z-plane, by position in the plane (x, y)
    ix = np.arange(plane, dtype=np.int64) % nx
    iy = np.arange(plane, dtype=np.int64) // nx
    counts_xy = 1 + (ix > 0) + (ix < nx - 1) + (iy > 0) + (iy < ny - 1)
    row_len = np.empty(n, dtype=np.int64)
    for z in range(nz):
        row_len[z * plane:(z + 1) * plane] = counts_xy + (z > 0) + (z < nz - 1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(row_len, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    col = np.empty(nnz, dtype=np.int32)
    val = np.empty(nnz, dtype=np.float64)
    offs = [(-plane, None), (-nx, iy > 0), (-1, ix > 0), (0, None),
            (1, ix < nx - 1), (nx, iy < ny - 1), (plane, None)]
    loc = np.arange(plane, dtype=np.int64)
    for z in range(nz):
        base = z * plane
        cols = np.empty((plane, 7), dtype=np.int64)
        valid = np.ones((plane, 7), dtype=bool)
        vals = np.full((plane, 7), -1.0)
        for j, (o, m) in enumerate(offs):
            cols[:, j] = base + loc + o
            if m is not None:
                valid[:, j] = m
        valid[:, 0] = z > 0
        valid[:, 6] = z < nz - 1
        vals[:, 3] = 6.0
        s, e = int(row_ptr[base]), int(row_ptr[base + plane])
        col[s:e] = cols[valid]
        val[s:e] = vals[valid]
    return CSR(n, n, row_ptr.astype(np.int32), col, val,
               f"lap3d_{nx}x{ny}x{nz}")


def uniform_vector(n: int, seed: int, dtype=np.float64) -> np.ndarray:
    """U[-1, 1] entries from PCG64(seed)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=n).astype(dtype)


def _zipf_truncated(rng, a, n, lo, hi):
    """Zipf(a) draws restricted to [lo, hi] by rejection."""
    out = np.empty(n, dtype=np.int64)
    filled = 0
    while filled < n:
        z = rng.zipf(a, size=max(1024, int((n - filled) * 1.2)))
        z = z[(z >= lo) & (z <= hi)]
        take = min(z.size, n - filled)
        out[filled:filled + take] = z[:take]
        filled += take
    return out


def power_law_lengths(n: int, a: float = 1.8, mean: float = 16.0,
                      max_len: int = 4096, seed: int = SEED_BASE + 2):
    """Row lengths L_i = clamp(round(c * Z_i), 1, max_len), Z_i ~ Zipf(a)
    truncated to [1, max_len]; c found by bisection so that mean(L) is
    within 0.5 % of ``mean``; one row is forced to exactly ``max_len``."""
    rng = np.random.default_rng(seed)
    z = _zipf_truncated(rng, a, n, 1, max_len).astype(np.float64)

    def lengths(c):
        return np.clip(np.rint(c * z), 1, max_len).astype(np.int64)

    lo, hi = 0.01, 1000.0
    for _ in range(200):
        c = 0.5 * (lo + hi)
        m = lengths(c).mean()
        if abs(m - mean) <= 0.001 * mean:
            break
        if m < mean:
            lo = c
        else:
            hi = c
    L = lengths(c)
    L[int(rng.integers(0, n))] = max_len
    return L, rng


def power_law(n: int = 1 << 22, a: float = 1.8, mean: float = 16.0,
              max_len: int = 4096, seed: int = SEED_BASE + 2) -> CSR:
    """Random power-law matrix: Zipf row lengths, distinct uniformly drawn
    columns (sorted), N(0,1) values.

    Distinct columns per row come from the sorted-gap construction: draw
    L values uniformly from [0, n - L + 1) with replacement, sort them and
    add each value's rank, which gives L strictly increasing columns in
    [0, n).
    """
    max_len = min(int(max_len), int(n))
    L, rng = power_law_lengths(n, a, mean, max_len, seed)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(L, out=row_ptr[1:])
    nnz = int(row_ptr[-1])
    rows = np.repeat(np.arange(n, dtype=np.int64), L)
    span = (n - L + 1)[rows]
    draws = (rng.random(nnz) * span).astype(np.int64)
    draws = np.minimum(draws, span - 1)
    key = rows * n + draws
    key.sort(kind="stable")
    draws = key - rows * n
    del key
    rank = np.arange(nnz, dtype=np.int64) - row_ptr[rows]
    col = (draws + rank).astype(np.int32)
    del draws, rank, rows, span
    val = rng.standard_normal(nnz)
    return CSR(n, n, row_ptr.astype(np.int32), col, val,
               f"powerlaw_{n}_a{a}")


def diffusion_3d(N: int = 128, sigma: float = 1.0,
                 seed: int = SEED_BASE + 3) -> CSR:
    """7-point variable-coefficient diffusion on an N^3 grid.

    Cell coefficients k = exp(g), g ~ N(0, sigma^2) iid per cell.  The
    coefficient of the face between cells i and j is the harmonic mean
    2 k_i k_j / (k_i + k_j); the off-diagonal entry is minus it.  The
    diagonal is the sum of the interior face coefficients plus k_i for
    every boundary face of cell i (Dirichlet).
    """
    rng = np.random.default_rng(seed)
    n = N ** 3
    k = np.exp(sigma * rng.standard_normal(n))
    k3 = k.reshape(N, N, N)  # [z, y, x]
    idx = np.arange(n, dtype=np.int64).reshape(N, N, N)
    diag = np.zeros((N, N, N))
    cols = np.empty((n, 7), dtype=np.int64)
    vals = np.zeros((n, 7))
    valid = np.zeros((n, 7), dtype=bool)
    # column order: -N^2 (z-1), -N (y-1), -1 (x-1), 0, +1, +N, +N^2
    shifts = [(0, -1, -N * N), (1, -1, -N), (2, -1, -1),
              (2, +1, 1), (1, +1, N), (0, +1, N * N)]
    slots = [0, 1, 2, 4, 5, 6]
    for (axis, sgn, off), slot in zip(shifts, slots):
        nb = np.roll(k3, -sgn, axis=axis)
        face = 2.0 * k3 * nb / (k3 + nb)
        coord = np.indices((N, N, N))[axis]
        inside = (coord + sgn >= 0) & (coord + sgn < N)
        diag += np.where(inside, face, k3)
        cols[:, slot] = (idx + off).reshape(-1)
        vals[:, slot] = np.where(inside, -face, 0.0).reshape(-1)
        valid[:, slot] = inside.reshape(-1)
    cols[:, 3] = idx.reshape(-1)
    vals[:, 3] = diag.reshape(-1)
    valid[:, 3] = True
    return _assemble(n, n, cols, vals, valid, f"diffusion3d_{N}")


def convection_diffusion_2d(nx: int, c: float = 1.0) -> CSR:
    """Nonsymmetric 5-point operator on an nx-by-nx grid (x fastest):
    diffusion (4 / -1) plus first-order upwind convection in +x of
    strength c >= 0, i.e. diagonal 4 + c and west neighbour -1 - c.
    Dirichlet boundary; weakly diagonally dominant."""
    m = _stencil((nx, nx), f"convdiff2d_{nx}_c{c:g}")
    rows = np.repeat(np.arange(m.n), m.row_lengths())
    v = m.values.copy()
    v[m.col_idx == rows] += c
    v[m.col_idx == rows - 1] -= c
    m.values = v
    return m


def shifted_rectangle(a: int, b: int, shift: float) -> CSR:
    """2D 5-point Laplacian on an a-by-b grid plus shift on the diagonal."""
    m = _stencil((a, b), f"rect_{a}x{b}")
    diag_mask = m.col_idx == np.repeat(np.arange(m.n), m.row_lengths())
    m.values = m.values.copy()
    m.values[diag_mask] += shift
    return m


def batched_rectangles(count: int = 2048, seed: int = SEED_BASE + 4,
                       n_lo: int = 64, n_hi: int = 4096):
    """``count`` shifted-rectangle systems: n_target ~ U{n_lo..n_hi},
    width a ~ U{8..64}, height b = clamp(round(n_target / a), 1,
    floor(n_hi / a)), shift ~ U[0, 1].  Returns (matrices, rhs list)."""
    rng = np.random.default_rng(seed)
    mats, rhs = [], []
    for _ in range(count):
        nt = int(rng.integers(n_lo, n_hi + 1))
        a = int(rng.integers(8, 65))
        b = int(min(max(round(nt / a), 1), n_hi // a))
        s = float(rng.uniform(0.0, 1.0))
        m = shifted_rectangle(a, b, s)
        mats.append(m)
        rhs.append(rng.uniform(-1.0, 1.0, size=m.n))
    return mats, rhs


def banded_spd(n: int, half_bw: int, seed: int) -> CSR:
    """Symmetric banded matrix: off-diagonals U[-1, 0] on |i - j| <= half_bw,
    diagonal = 1.1 x absolute off-diagonal row sum."""
    rng = np.random.default_rng(seed)
    w = int(half_bw)
    upper = rng.uniform(-1.0, 0.0, size=(n, w))  # upper[i, d-1] = A[i, i+d]
    for d in range(1, w + 1):
        upper[n - d:, d - 1] = 0.0
    lower = np.zeros((n, w))  # lower[i, d-1] = A[i, i-d] = A[i-d, i]
    for d in range(1, w + 1):
        lower[d:, d - 1] = upper[:n - d, d - 1]
    idx = np.arange(n, dtype=np.int64)
    cols = np.empty((n, 2 * w + 1), dtype=np.int64)
    vals = np.empty((n, 2 * w + 1))
    valid = np.empty((n, 2 * w + 1), dtype=bool)
    for d in range(w, 0, -1):
        j = w - d
        cols[:, j] = idx - d
        vals[:, j] = lower[:, d - 1]
        valid[:, j] = idx - d >= 0
    cols[:, w] = idx
    vals[:, w] = 1.1 * (np.abs(upper).sum(axis=1) + np.abs(lower).sum(axis=1))
    valid[:, w] = True
    for d in range(1, w + 1):
        j = w + d
        cols[:, j] = idx + d
        vals[:, j] = upper[:, d - 1]
        valid[:, j] = idx + d < n
    return _assemble(n, n, cols, vals, valid, f"banded_{n}_w{w}")


def random_csr(n: int, ncols: int, density: float, seed: int,
               empty_rows: int = 0, full_rows: int = 0,
               dtype=np.float64) -> CSR:
    """Irregular small matrix: each entry present with probability
    ``density``; ``empty_rows`` rows forced empty and ``full_rows`` rows
    forced full.  Values N(0,1)."""
    rng = np.random.default_rng(seed)
    mask = rng.random((n, ncols)) < density
    if empty_rows:
        mask[rng.choice(n, size=min(empty_rows, n), replace=False)] = False
    if full_rows:
        mask[rng.choice(n, size=min(full_rows, n), replace=False)] = True
    vals = rng.standard_normal((n, ncols))
    cols = np.broadcast_to(np.arange(ncols, dtype=np.int64), (n, ncols))
    m = _assemble(n, ncols, cols, vals, mask, f"rand_{n}x{ncols}")
    m.values = m.values.astype(dtype)
    return m


def random_coo(n: int, ncols: int, nnz: int, seed: int, dup_frac: float = 0.2,
               dtype=np.float64):
    """Unsorted COO triplets with about ``dup_frac`` repeated (row, col)
    positions.  Returns (row, col, val)."""
    rng = np.random.default_rng(seed)
    base = max(1, int(nnz * (1.0 - dup_frac)))
    r = rng.integers(0, n, size=base)
    c = rng.integers(0, ncols, size=base)
    extra = nnz - base
    if extra > 0:
        pick = rng.integers(0, base, size=extra)
        r = np.concatenate([r, r[pick]])
        c = np.concatenate([c, c[pick]])
    perm = rng.permutation(r.size)
    r, c = r[perm], c[perm]
    v = rng.standard_normal(r.size).astype(dtype)
    return r.astype(np.int32), c.astype(np.int32), v


def serving_pool(count: int = 24, seed: int = SEED_BASE + 5, n_lo: float = 1e3,
                 n_hi: float = 1e6, max_nnz: int = 20_000_000):
    """Matrices for the serving mix: sizes log-uniform in [n_lo, n_hi], kind
    uniform over {2D 5-point, 3D 7-point, banded SPD with half bandwidth
    U{5..64}}.  A banded matrix whose nnz would exceed max_nnz gets fewer
    rows (its bandwidth is kept)."""
    rng = np.random.default_rng(seed)
    mats = []
    for _ in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        kind = int(rng.integers(0, 3))
        if kind == 0:
            side = max(2, int(round(n ** 0.5)))
            mats.append(laplacian_2d(side))
        elif kind == 1:
            side = max(2, int(round(n ** (1.0 / 3.0))))
            mats.append(laplacian_3d(side))
        else:
            w = int(rng.integers(5, 65))
            n = max(2 * w + 2, min(n, max_nnz // (2 * w + 1)))
            mats.append(banded_spd(n, w, int(rng.integers(0, 2 ** 31))))
    return mats


def serving_requests(pool, count: int, seed: int = SEED_BASE + 5):
    """Request parameters: (matrix index, precision 'f64' | 'ir32' 50/50,
    tol log-uniform in [1e-10, 1e-8], right-hand-side seed)."""
    rng = np.random.default_rng(seed + 1)
    out = []
    for i in range(count):
        out.append((int(rng.integers(0, len(pool))),
                    "f64" if rng.random() < 0.5 else "ir32",
                    float(10 ** rng.uniform(-10, -8)),
                    int(rng.integers(0, 2 ** 31))))
    return out
