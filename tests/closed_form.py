"""Closed-form spectra of the Dirichlet finite-difference Laplacians (test-side helper).

The 1-D second-difference matrix tridiag(-1, 2, -1) of order N has eigenvalues
2 - 2 cos(i pi/(N+1)), i = 1..N; the 2-D / 3-D grid Laplacians are Kronecker sums of it,
so their eigenvalues are the sums over the axes.
"""
import numpy as np


def lap1d_eigs(nx):
    return 2.0 - 2.0 * np.cos(np.arange(1, nx + 1) * np.pi / (nx + 1))


def lap_eigs(dim, nx):
    f = lap1d_eigs(nx)
    if dim == 2:
        e = f[:, None] + f[None, :]
    else:
        e = f[:, None, None] + f[None, :, None] + f[None, None, :]
    return np.sort(e.ravel())


def count_in(e, a, b, right_closed=True):
    return int(np.count_nonzero((e >= a) & ((e <= b) if right_closed else (e < b))))


def nnz_formula(dim, nx):
    return nx ** 2 + 4 * nx * (nx - 1) if dim == 2 else nx ** 3 + 6 * nx ** 2 * (nx - 1)
