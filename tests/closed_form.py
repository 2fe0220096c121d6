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


def pencil_eigs(nx):
    """Eigenvalues of the pencil (laplacian_2d(nx), mass_matrix_2d(nx)): A = T (x) I + I (x) T and
    B = M (x) M with M = tridiag(1, 4, 1) / 6 share the sine eigenvectors, so
    lambda_ij = (t_i + t_j) / (m_i m_j) with t_i = 2 - 2 cos(i pi/(nx+1)), m_i = (4 + 2 cos(i pi/(nx+1))) / 6."""
    k = np.arange(1, nx + 1)
    t = 2.0 - 2.0 * np.cos(k * np.pi / (nx + 1))
    m = (4.0 + 2.0 * np.cos(k * np.pi / (nx + 1))) / 6.0
    return np.sort(((t[:, None] + t[None, :]) / (m[:, None] * m[None, :])).ravel())
