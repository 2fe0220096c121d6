"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module holds no arithmetic of the eigensolver itself.  It builds the test matrices of
the paper's experiments (Section 4.1, Table 1: 5-point / 7-point finite-difference Laplacians
on regular grids with Dirichlet boundaries) and the Anderson-disordered 3-D Laplacian
(7-point Laplacian plus a seeded uniform random diagonal), all in CSR form with sorted
columns and lexicographic row ordering (x fastest).

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-based:

    mix(z)      = the SplitMix64 output function (xor-shift 30/27/31, two multiplies)
    key(s, t)   = mix(s ^ (t * 0xD1B54A32D192ED03) + 0x9E3779B97F4A7C15)
    draw(s,t,k) = mix(key(s, t) + (k + 1) * 0x9E3779B97F4A7C15)        (mod 2**64)

i.e. draw(s, t, k) is the (k+1)-th output of a SplitMix64 generator seeded with key(s, t),
and key(s, t) is the first output of one seeded with s ^ (t * 0xD1B54A32D192ED03).
A uniform double in [0, 1) is (x >> 11) * 2**-53; a Rademacher sign is +1 when the top bit
of x is 0 and -1 otherwise.  The oracle and the CUDA kernels each carry their own
implementation of the same definition; stream numbers are fixed below.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
STREAM_MUL = np.uint64(0xD1B54A32D192ED03)

# Stream tags (the `t` argument of draw()).
STREAM_ANDERSON = 1     # Anderson disorder, k = row index
STREAM_KPM = 2          # KPM Rademacher probes, k = probe * n + row
STREAM_LANCZOS = 3      # Lanczos start vectors, k = restart_index * n + row
STREAM_BOUNDS = 4       # start vector of the spectral-bounds Lanczos run, k = row
STREAM_LANDOS = 5       # start vectors of the Lanczos density runs, k = vector * n + row

_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64_sequence(seed: int, count: int) -> np.ndarray:
    """First `count` outputs of a plain SplitMix64 generator seeded with `seed`."""
    k = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(np.uint64(seed) + k * GOLDEN)


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = np.uint64(seed) ^ (np.uint64(stream) * STREAM_MUL)
        return _mix(np.array([s + GOLDEN], dtype=np.uint64))[0]


def draw(seed: int, stream: int, k: np.ndarray) -> np.ndarray:
    """Counter-based SplitMix64 draws for indices k (uint64 array)."""
    key = stream_key(seed, stream)
    k = np.asarray(k, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return _mix(key + (k + np.uint64(1)) * GOLDEN)


def to_unit(x: np.ndarray) -> np.ndarray:
    """Uniform double in [0, 1) from the top 53 bits."""
    return (np.asarray(x, dtype=np.uint64) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def to_sign(x: np.ndarray) -> np.ndarray:
    """Rademacher sign from the top bit: +1.0 or -1.0."""
    return np.where((np.asarray(x, dtype=np.uint64) >> np.uint64(63)) == 0, 1.0, -1.0)


def rademacher_block(n: int, nvec: int, seed: int) -> np.ndarray:
    """The KPM probe block V (n x nvec, column-major meaning probe l is V[:, l])."""
    k = np.arange(n * nvec, dtype=np.uint64)
    return to_sign(draw(seed, STREAM_KPM, k)).reshape(nvec, n).T.copy()


class CSR:
    """Symmetric sparse matrix in CSR form (int64 row_ptr, int32 col_idx, float64 val)."""

    def __init__(self, n, row_ptr, col_idx, val, name=""):
        self.n = int(n)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        self.name = name

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        a = np.zeros((self.n, self.n))
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        a[rows, self.col_idx] = self.val
        return a

    def __repr__(self):
        return f"CSR({self.name!r}, n={self.n}, nnz={self.nnz})"


def _grid_csr(dims, diag_extra=None, name=""):
    """Finite-difference Laplacian on a grid with Dirichlet boundaries (no wrap).

    dims = (nx,) (1-D), (nx, ny) or (nx, ny, nz); row r = i + nx*(j + ny*k).
    Diagonal 2*len(dims), off-diagonals -1 to each in-grid neighbour.
    """
    dims = tuple(int(d) for d in dims)
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx.copy()
    for d in dims:
        coords.append(rem % d)
        rem //= d
    strides = [1]
    for d in dims[:-1]:
        strides.append(strides[-1] * d)
    # neighbour offsets in increasing column order: -s_last, ..., -s_0, 0, +s_0, ..., +s_last
    offs = []
    for a in reversed(range(len(dims))):
        offs.append((a, -1))
    offs.append((None, 0))
    for a in range(len(dims)):
        offs.append((a, +1))
    cols = np.full((n, len(offs)), -1, dtype=np.int64)
    vals = np.zeros((n, len(offs)))
    for t, (axis, sgn) in enumerate(offs):
        if axis is None:
            cols[:, t] = idx
            vals[:, t] = 2.0 * len(dims)
            if diag_extra is not None:
                vals[:, t] += diag_extra
            continue
        c = coords[axis]
        ok = (c > 0) if sgn < 0 else (c < dims[axis] - 1)
        cols[ok, t] = idx[ok] + sgn * strides[axis]
        vals[ok, t] = -1.0
    mask = cols >= 0
    counts = mask.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr, cols[mask].astype(np.int32), vals[mask], name=name)


def laplacian_2d(nx: int, ny: int | None = None) -> CSR:
    ny = nx if ny is None else ny
    return _grid_csr((nx, ny), name=f"lap2d_{nx}x{ny}")


def laplacian_3d(nx: int, ny: int | None = None, nz: int | None = None) -> CSR:
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    return _grid_csr((nx, ny, nz), name=f"lap3d_{nx}x{ny}x{nz}")


def mass_matrix_2d(nx: int) -> CSR:
    """Linear finite-element mass matrix on an nx x nx grid, M (x) M with the 1-D mass matrix
    M = tridiag(1, 4, 1) / 6 (SPD, condition number below 3): the B of a generalized pencil
    (A, B) with A = laplacian_2d(nx).  Rows ordered like laplacian_2d (x fastest), columns
    sorted; entry ((y, x), (y', x')) = M[x, x'] M[y, y']."""
    k = np.arange(nx, dtype=np.int64)
    # 1-D entries (i, j, M[i, j])
    i1 = np.concatenate([k, k[1:], k[:-1]])
    j1 = np.concatenate([k, k[:-1], k[1:]])
    v1 = np.concatenate([np.full(nx, 4.0 / 6.0), np.full(2 * (nx - 1), 1.0 / 6.0)])
    # 2-D entries: y-part along the first axis, x-part along the second
    rows = (i1[:, None] * nx + i1[None, :]).ravel()
    cols = (j1[:, None] * nx + j1[None, :]).ravel()
    vals = (v1[None, :] * v1[:, None]).ravel()
    order = np.lexsort((cols, rows))
    n = nx * nx
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return CSR(n, row_ptr, cols[order].astype(np.int32), vals[order], name=f"mass2d_{nx}")


def anderson_diagonal(n: int, W: float, seed: int) -> np.ndarray:
    """Uniform[-W/2, W/2] disorder, one SplitMix64 draw per row."""
    u = to_unit(draw(seed, STREAM_ANDERSON, np.arange(n, dtype=np.uint64)))
    return W * (u - 0.5)


def anderson_3d(nx: int, W: float, seed: int = 0) -> CSR:
    """Anderson model: 7-point Laplacian with diagonal 6 + U[-W/2, W/2] (seeded)."""
    n = nx ** 3
    return _grid_csr((nx, nx, nx), diag_extra=anderson_diagonal(n, W, seed),
                     name=f"anderson3d_{nx}_W{W:g}_s{seed}")


def start_vector(n: int, seed: int, stream: int, index: int = 0) -> np.ndarray:
    """Uniform(-1, 1) vector number `index` of a stream (not normalised)."""
    k = np.arange(n, dtype=np.uint64) + np.uint64(index) * np.uint64(n)
    return 2.0 * to_unit(draw(seed, stream, k)) - 1.0


def workload(name: str) -> dict:
    """The named synthetic workloads (sizes of the paper's and the benchmark's cases)."""
    if name == "lap2d_100":
        return dict(matrix=lambda: laplacian_2d(100), xi=0.40, eta=0.48, kpm_deg=80,
                    kpm_nvec=20, nslices=1)
    if name == "lap3d_100":
        return dict(matrix=lambda: laplacian_3d(100), xi=0.20, eta=0.60, kpm_deg=120,
                    kpm_nvec=40, nslices=10)
    if name == "anderson3d_80":
        return dict(matrix=lambda: anderson_3d(80, 4.0, 0), xi=-1.0, eta=1.0, kpm_deg=120,
                    kpm_nvec=40, nslices=16)
    if name == "anderson3d_200":
        return dict(matrix=lambda: anderson_3d(200, 2.0, 0), kpm_deg=300, kpm_nvec=64)
    raise KeyError(name)
