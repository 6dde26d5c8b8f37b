"""Seeded synthetic inputs: sparse SPD stencil matrices and right-hand sides.

This module is shared by the oracle's tests and by the CUDA path's tests and
benchmark. It builds matrices only; it holds none of the factorization's
arithmetic (no ordering, no symbolic analysis, no elimination).

Every matrix is returned as the lower triangle of a symmetric matrix in
compressed sparse column form, 0-based, including the diagonal, row indices
ascending within each column, no duplicates:

    colptr : int64[n+1]
    rowind : int32[nnz]
    values : float64[nnz]

Grid points are numbered id = x + nx*(y + ny*z) (x fastest). Coefficients are
drawn once per undirected edge, so the matrix is symmetric by construction.
The stand-ins replace the SuiteSparse matrices of the paper's experiments
(Section 3.1), which are not available here.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Seeds for the five workloads: base seed + workload index (1-based).
SEED_BASE = 20240913


@dataclass
class SparseSym:
    """Lower triangle (with diagonal) of a symmetric matrix, CSC, 0-based."""

    n: int
    colptr: np.ndarray
    rowind: np.ndarray
    values: np.ndarray
    grid: tuple = (0, 0, 0)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1])


def _half_offsets(points: int):
    """Neighbour offsets (dx, dy, dz) of a stencil whose neighbour has the larger id.

    points = 5 (2D), 7 (3D face neighbours) or 27 (3D full box).
    """
    if points == 5:
        return [(1, 0, 0), (0, 1, 0)]
    if points == 7:
        return [(1, 0, 0), (0, 1, 0), (0, 0, 1)]
    if points == 27:
        offs = []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if (dz, dy, dx) > (0, 0, 0):
                        offs.append((dx, dy, dz))
        return offs
    raise ValueError(points)


def _edges(nx: int, ny: int, nz: int, points: int):
    """All undirected grid edges (i < j) of the stencil, grouped per offset."""
    x, y, z = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    x = x.transpose(2, 1, 0).ravel()  # order by id = x + nx*(y + ny*z)
    y = y.transpose(2, 1, 0).ravel()
    z = z.transpose(2, 1, 0).ravel()
    ids = np.arange(nx * ny * nz, dtype=np.int64)
    out = []
    for dx, dy, dz in _half_offsets(points):
        ok = (x + dx >= 0) & (x + dx < nx) & (y + dy >= 0) & (y + dy < ny) & (z + dz >= 0) & (z + dz < nz)
        i = ids[ok]
        j = i + dx + nx * (dy + ny * dz)
        out.append(((dx, dy, dz), i, j))
    return out


def _assemble(n: int, ei: np.ndarray, ej: np.ndarray, ew: np.ndarray, diag: np.ndarray) -> tuple:
    """CSC lower triangle from edges (ei < ej, weight ew -> A[ej, ei] = -ew) and a diagonal."""
    rows = np.concatenate([np.arange(n, dtype=np.int64), ej.astype(np.int64)])
    cols = np.concatenate([np.arange(n, dtype=np.int64), ei.astype(np.int64)])
    vals = np.concatenate([diag.astype(np.float64), -ew.astype(np.float64)])
    order = np.lexsort((rows, cols))
    rows, cols, vals = rows[order], cols[order], vals[order]
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, cols + 1, 1)
    colptr = np.cumsum(colptr)
    return colptr, rows.astype(np.int32), vals


def _rowsum(n: int, ei: np.ndarray, ej: np.ndarray, ew: np.ndarray) -> np.ndarray:
    s = np.zeros(n, dtype=np.float64)
    np.add.at(s, ei, np.abs(ew))
    np.add.at(s, ej, np.abs(ew))
    return s


def laplacian_2d(nx: int, ny: int, shift: float = 0.0) -> SparseSym:
    """2D 5-point Laplacian with Dirichlet boundary: diagonal 4 + shift, off-diagonals -1."""
    n = nx * ny
    groups = _edges(nx, ny, 1, 5)
    ei = np.concatenate([g[1] for g in groups])
    ej = np.concatenate([g[2] for g in groups])
    ew = np.ones(ei.shape[0])
    colptr, rowind, values = _assemble(n, ei, ej, ew, np.full(n, 4.0 + shift))
    return SparseSym(n, colptr, rowind, values, (nx, ny, 1), f"lap2d_{nx}x{ny}")


def diffusion_3d_7pt(nx: int, ny: int, nz: int, seed: int, lo: float = 1e-2, hi: float = 1e2,
                     shift: float = 1e-6) -> SparseSym:
    """3D 7-point variable-coefficient diffusion.

    Edge coefficient c ~ log-uniform[lo, hi]; A_ij = -c; A_ii = sum_j |A_ij| + shift,
    the sum over in-grid neighbours only (a Neumann-type graph Laplacian plus a shift).
    """
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    groups = _edges(nx, ny, nz, 7)
    ei = np.concatenate([g[1] for g in groups])
    ej = np.concatenate([g[2] for g in groups])
    ew = np.exp(rng.uniform(np.log(lo), np.log(hi), size=ei.shape[0]))
    diag = _rowsum(n, ei, ej, ew) + shift
    colptr, rowind, values = _assemble(n, ei, ej, ew, diag)
    return SparseSym(n, colptr, rowind, values, (nx, ny, nz), f"diff7_{nx}x{ny}x{nz}")


def stencil_3d_27pt(nx: int, ny: int, nz: int, seed: int, wlo: float = 0.5, whi: float = 1.5,
                    dominance: float = 1.01) -> SparseSym:
    """3D 27-point stencil: weights w ~ U[wlo, whi], A_ij = -w, A_ii = dominance * row sum."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    groups = _edges(nx, ny, nz, 27)
    ei = np.concatenate([g[1] for g in groups])
    ej = np.concatenate([g[2] for g in groups])
    ew = rng.uniform(wlo, whi, size=ei.shape[0])
    diag = dominance * _rowsum(n, ei, ej, ew)
    colptr, rowind, values = _assemble(n, ei, ej, ew, diag)
    return SparseSym(n, colptr, rowind, values, (nx, ny, nz), f"st27_{nx}x{ny}x{nz}")


def anisotropic_3d_7pt(nx: int, ny: int, nz: int, seed: int, axis=(1.0, 1.0, 100.0),
                       lo: float = 0.1, hi: float = 10.0, shift: float = 1e-8) -> SparseSym:
    """3D 7-point anisotropic diffusion: c = axis[d] * log-uniform[lo, hi]; diagonal = row sum + shift."""
    rng = np.random.default_rng(seed)
    n = nx * ny * nz
    groups = _edges(nx, ny, nz, 7)
    eis, ejs, ews = [], [], []
    for (dx, dy, dz), i, j in groups:
        d = 0 if dx else (1 if dy else 2)
        eis.append(i)
        ejs.append(j)
        ews.append(axis[d] * np.exp(rng.uniform(np.log(lo), np.log(hi), size=i.shape[0])))
    ei, ej, ew = np.concatenate(eis), np.concatenate(ejs), np.concatenate(ews)
    diag = _rowsum(n, ei, ej, ew) + shift
    colptr, rowind, values = _assemble(n, ei, ej, ew, diag)
    return SparseSym(n, colptr, rowind, values, (nx, ny, nz), f"aniso7_{nx}x{ny}x{nz}")


def batch_laplacians_2d(count: int, seed: int, side_lo: int = 32, side_hi: int = 256,
                        shift_lo: float = 1e-3, shift_hi: float = 1e-1) -> list:
    """Independent 2D 5-point Laplacians, side ~ U{side_lo..side_hi}, shift ~ U[shift_lo, shift_hi]."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(side_lo, side_hi + 1, size=count)
    shifts = rng.uniform(shift_lo, shift_hi, size=count)
    return [laplacian_2d(int(s), int(s), float(sh)) for s, sh in zip(sides, shifts)]


def random_spd(n: int, density: float, seed: int) -> SparseSym:
    """Random sparse symmetric diagonally dominant matrix (for brute-force checks on small n)."""
    rng = np.random.default_rng(seed)
    mask = np.triu(rng.random((n, n)) < density, 1)
    ei, ej = np.nonzero(mask)
    ew = rng.uniform(0.1, 1.0, size=ei.shape[0])
    diag = _rowsum(n, ei, ej, ew) + rng.uniform(0.5, 1.5, size=n)
    colptr, rowind, values = _assemble(n, ei.astype(np.int64), ej.astype(np.int64), ew, diag)
    return SparseSym(n, colptr, rowind, values, (0, 0, 0), f"rand{n}")


def from_lower_pattern(n: int, entries, diag: float | None = None, seed: int = 0) -> SparseSym:
    """Matrix with a given strictly-lower pattern [(i, j), i > j], diagonally dominant values."""
    rng = np.random.default_rng(seed)
    ej = np.array([e[0] for e in entries], dtype=np.int64)  # row (larger)
    ei = np.array([e[1] for e in entries], dtype=np.int64)  # column (smaller)
    ew = rng.uniform(0.1, 1.0, size=ei.shape[0])
    d = _rowsum(n, ei, ej, ew) + 1.0 if diag is None else np.full(n, diag)
    colptr, rowind, values = _assemble(n, ei, ej, ew, d)
    return SparseSym(n, colptr, rowind, values, (0, 0, 0), "pattern")


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """Right-hand sides, uniform[-1, 1], column-major n x nrhs (Fortran order)."""
    rng = np.random.default_rng(seed + 7919)
    return np.asfortranarray(rng.uniform(-1.0, 1.0, size=(n, nrhs)))


# The five workloads, with their full sizes. `scale` shrinks grid sides for tests.
def workload(idx: int, scale: float = 1.0):
    """Return (matrix or list of matrices, nrhs) for workload idx in 1..5."""
    seed = SEED_BASE + idx

    def s(v):
        return max(4, int(round(v * scale)))

    if idx == 1:
        return laplacian_2d(s(64), s(64)), 1
    if idx == 2:
        return diffusion_3d_7pt(s(48), s(48), s(48), seed), 4
    if idx == 3:
        return stencil_3d_27pt(s(80), s(80), s(80), seed), 16
    if idx == 4:
        count = max(2, int(round(256 * scale)))
        return batch_laplacians_2d(count, seed, side_lo=s(32), side_hi=s(256)), 1
    if idx == 5:
        return anisotropic_3d_7pt(s(128), s(128), s(128), seed), 64
    raise ValueError(idx)


def dense_from_lower(A: SparseSym) -> np.ndarray:
    """Dense symmetric matrix (small n only)."""
    M = np.zeros((A.n, A.n))
    for j in range(A.n):
        for p in range(A.colptr[j], A.colptr[j + 1]):
            i = A.rowind[p]
            M[i, j] = A.values[p]
            M[j, i] = A.values[p]
    return M
