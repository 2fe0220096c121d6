"""Python access to the plain FP64 CPU oracle (oracle/evsl_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers.  The CUDA path never imports this package, and this package
imports nothing from the CUDA path.  Each wrapper names the paper passage the C function
follows (arXiv:1802.05215, Sections 2.1-2.5 and Algorithm 2).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "evsl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

DAMP_NONE, DAMP_JACKSON, DAMP_SIGMA = 0, 1, 2


_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_libs = {}
_threads = 1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FMA contraction), once plain and once with OpenMP.
    The loops the OpenMP build runs in parallel (SpMV rows, elementwise updates, independent
    dot products) carry no reduction, so both builds give bitwise the same results; the
    OpenMP one only serves the multi-core CPU baseline."""
    for lib, extra in ((_LIB, []), (_LIB_OMP, ["-fopenmp"])):
        if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", *extra,
                                   "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, lib)
    return _LIB


def set_threads(n: int) -> int:
    """Run the oracle on n host threads (n <= 1: the plain single-threaded build).  Returns the
    previous setting."""
    global _threads, _lib
    prev = _threads
    _threads = max(1, int(n))
    _lib = None
    if _threads > 1:
        build()
        gomp = C.CDLL("libgomp.so.1", mode=C.RTLD_GLOBAL)
        gomp.omp_set_num_threads(_threads)
    return prev


def threads() -> int:
    return _threads


def _load():
    global _lib
    if _lib is None:
        build()
        path = _LIB_OMP if _threads > 1 else _LIB
        if path in _libs:
            _lib = _libs[path]
            return _lib
        _lib = C.CDLL(path)
        _libs[path] = _lib
        d, i32, i64, u64 = C.c_double, C.c_int, C.c_int64, C.c_uint64
        P = C.c_void_p
        _lib.orc_draw.restype = u64
        _lib.orc_draw.argtypes = [u64, u64, u64]
        _lib.orc_splitmix64_next.restype = u64
        _lib.orc_splitmix64_next.argtypes = [P]
        _lib.orc_spmv.argtypes = [i64, P, P, P, P, P]
        _lib.orc_syev.restype = i32
        _lib.orc_syev.argtypes = [i32, P, P, P]
        _lib.orc_bounds.restype = i32
        _lib.orc_bounds.argtypes = [i64, P, P, P, i32, u64, P, P]
        _lib.orc_kpm_moments.restype = i32
        _lib.orc_kpm_moments.argtypes = [i64, P, P, P, i32, i32, u64, d, d, P]
        _lib.orc_kpm_probe_moments.restype = i32
        _lib.orc_kpm_probe_moments.argtypes = [i64, P, P, P, i32, i64, i32, u64, d, d, P]
        _lib.orc_kpm_moments_doubling.restype = i32
        _lib.orc_kpm_moments_doubling.argtypes = [i64, P, P, P, i32, i32, u64, d, d, P]
        _lib.orc_jackson.argtypes = [i32, P]
        _lib.orc_dos_count.restype = d
        _lib.orc_dos_count.argtypes = [P, i32, d, d, d]
        _lib.orc_slicer.restype = i32
        _lib.orc_slicer.argtypes = [P, i32, d, d, d, d, i32, i32, P, P]
        _lib.orc_filter_build.restype = i32
        _lib.orc_filter_build.argtypes = [d, d, d, d, d, d, i32, i32, P, P, P, P, i32, P]
        _lib.orc_filter_apply.argtypes = [i64, P, P, P, d, d, i32, P, i32, P, P]
        _lib.orc_reorth_cgs.restype = i32
        _lib.orc_reorth_cgs.argtypes = [i64, P, P, i32]
        _lib.orc_cheblantr.restype = i32
        _lib.orc_cheblantr.argtypes = [i64, P, P, P, d, d, i32, d, d, i32, P, d,
                                       i32, i32, i32, d, d, u64, i32, P, P, P, P, P]
        _lib.orc_landos.restype = i32
        _lib.orc_landos.argtypes = [i64, P, P, P, i32, i32, u64, P, P, P]
        _lib.orc_slicer_landos.restype = i32
        _lib.orc_slicer_landos.argtypes = [P, P, P, i32, i32, i64, d, d, i32, P, P]
        _lib.orc_lspol.restype = i32
        _lib.orc_lspol.argtypes = [d, d, d, i32, P, P]
        _lib.orc_lspol_isqrt.restype = i32
        _lib.orc_lspol_isqrt.argtypes = [d, d, d, i32, P, P]
        _lib.orc_cheblantr_gen.restype = i32
        _lib.orc_cheblantr_gen.argtypes = [i64, P, P, P, P, P, P, d, d, i32, P, d, d, i32, d, d, i32, P, d,
                                           i32, i32, i32, d, d, u64, i32, P, P, P, P, P]
        _lib.orc_landos_gen.restype = i32
        _lib.orc_landos_gen.argtypes = [i64, P, P, P, P, P, P, d, d, i32, P, i32, P, i32, i32, u64, P, P, P]
        _lib.orc_kpm_moments_gen.restype = i32
        _lib.orc_kpm_moments_gen.argtypes = [i64, P, P, P, P, P, P, d, d, i32, P, i32, P, i32, i32, u64, d, d, P]
        _lib.orc_polyB_apply.restype = None
        _lib.orc_polyB_apply.argtypes = [i64, P, P, P, d, d, i32, P, P, P]
        _lib.orc_bounds_gen.restype = i32
        _lib.orc_bounds_gen.argtypes = [i64, P, P, P, P, P, P, d, d, i32, P, i32, u64, P, P]
        _lib.orc_cheblannr_gen.restype = i32
        _lib.orc_cheblannr_gen.argtypes = [i64, P, P, P, P, P, P, d, d, i32, P, d, d, i32, d, d, i32, P,
                                           d, i32, i32, d, d, u64, i32, P, P, P, P, P]
        _lib.orc_chebsi.restype = i32
        _lib.orc_chebsi.argtypes = [i64, P, P, P, d, d, i32, d, d, i32, P, d, i32, i32, d, u64,
                                    i32, P, P, P, P, P]
        _lib.orc_cheblannr.restype = i32
        _lib.orc_cheblannr.argtypes = [i64, P, P, P, d, d, i32, d, d, i32, P, d,
                                       i32, i32, d, d, u64, i32, P, P, P, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p)


def _csr_args(A):
    return (A.n, _p(A.row_ptr), _p(A.col_idx), _p(A.val))


def draw(seed: int, stream: int, k: int) -> int:
    return int(_load().orc_draw(seed, stream, k))


def splitmix64_sequence(seed: int, count: int) -> list[int]:
    st = C.c_uint64(seed)
    lib = _load()
    return [int(lib.orc_splitmix64_next(C.byref(st))) for _ in range(count)]


def spmv(A, x: np.ndarray) -> np.ndarray:
    """y = A x (CSR, Sec. 3.1)."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(A.n)
    _load().orc_spmv(*_csr_args(A), _p(x), _p(y))
    return y


def syev(Amat: np.ndarray):
    """Eigenvalues (ascending) and eigenvectors of a dense symmetric matrix
    (Householder tridiagonalisation + implicit symmetric QR)."""
    n = Amat.shape[0]
    a = np.asfortranarray(Amat, dtype=np.float64)
    w = np.empty(n)
    z = np.empty((n, n), order="F")
    st = _load().orc_syev(n, _p(a), _p(w), _p(z))
    if st != 0:
        raise RuntimeError("oracle syev did not converge")
    return w, z


def bounds(A, steps: int = 80, seed: int = 0):
    """Spectral bounds by a short Lanczos run (Sec. 2.2.1, LanTrbounds)."""
    lo, hi = C.c_double(), C.c_double()
    st = _load().orc_bounds(*_csr_args(A), steps, seed, C.byref(lo), C.byref(hi))
    if st != 0:
        raise RuntimeError("oracle bounds failed")
    return lo.value, hi.value


def kpm_moments_doubling(A, degree: int, nvec: int, seed: int, lmin: float, lmax: float) -> np.ndarray:
    """KPM moments from ceil(degree/2) recurrence steps (doubling identities)."""
    mu = np.empty(degree + 1)
    _load().orc_kpm_moments_doubling(*_csr_args(A), degree, nvec, seed, lmin, lmax, _p(mu))
    return mu


def kpm_moments(A, degree: int, nvec: int, seed: int, lmin: float, lmax: float) -> np.ndarray:
    """KPM moments mu_0..mu_degree with Rademacher probes (Sec. 2.1)."""
    mu = np.empty(degree + 1)
    _load().orc_kpm_moments(*_csr_args(A), degree, nvec, seed, lmin, lmax, _p(mu))
    return mu


def kpm_probe_moments(A, degree: int, first: int, nprobe: int, seed: int, lmin: float,
                      lmax: float) -> np.ndarray:
    """Per-probe KPM sums v_l^T T_k(Ahat) v_l for probes first..first+nprobe-1 (Sec. 2.1, the
    estimator's terms before averaging): an nprobe x (degree + 1) array."""
    out = np.empty((nprobe, degree + 1))
    _load().orc_kpm_probe_moments(*_csr_args(A), degree, first, nprobe, seed, lmin, lmax, _p(out))
    return out


def jackson(M: int) -> np.ndarray:
    g = np.empty(M + 1)
    _load().orc_jackson(M, _p(g))
    return g


def dos_count(mu: np.ndarray, lmin: float, lmax: float, t: float) -> float:
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    return float(_load().orc_dos_count(_p(mu), len(mu) - 1, lmin, lmax, t))


def slicer(mu, lmin, lmax, xi, eta, nslices, npts=None):
    """DOS-balanced slice ends (Eq. (2.2), spslicer)."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    npts = npts or max(2001, 100 * nslices)
    sli = np.empty(nslices + 1)
    est = np.empty(nslices)
    st = _load().orc_slicer(_p(mu), len(mu) - 1, lmin, lmax, xi, eta, nslices, npts,
                            _p(sli), _p(est))
    if st != 0:
        raise ValueError("oracle slicer: bad arguments")
    return sli, est


def filter_build(a, b, lmin, lmax, tau=0.8, damping=DAMP_JACKSON, maxdeg=10000, tau_ext=0.4):
    """Chebyshev delta filter for [a, b] (Sec. 2.2.1).  Returns a dict."""
    cap = maxdeg + 1
    coef = np.empty(cap)
    deg, gam, bar, bnd = C.c_int(), C.c_double(), C.c_double(), C.c_int()
    st = _load().orc_filter_build(a, b, lmin, lmax, tau, tau_ext, damping, maxdeg, C.byref(deg),
                                  C.byref(gam), C.byref(bar), _p(coef), cap, C.byref(bnd))
    if st not in (0, -2):
        raise ValueError(f"oracle filter_build failed ({st})")
    return dict(deg=deg.value, gamma=gam.value, bar=bar.value, coef=coef[:deg.value + 1].copy(),
                boundary=bnd.value, lmin=lmin, lmax=lmax, a=a, b=b, reached_max=(st == -2))


def filter_apply(A, lmin, lmax, coef, X: np.ndarray) -> np.ndarray:
    """Y = rho(Ahat) X for each column of X (Eq. (2.4))."""
    X = np.asfortranarray(X.reshape(A.n, -1), dtype=np.float64)
    nvec = X.shape[1]
    Y = np.empty_like(X, order="F")
    coef = np.ascontiguousarray(coef, dtype=np.float64)
    _load().orc_filter_apply(*_csr_args(A), lmin, lmax, len(coef) - 1, _p(coef), nvec,
                             _p(X), _p(Y))
    return Y


def reorth(z: np.ndarray, B: np.ndarray) -> int:
    """Full reorthogonalisation of z (in place) against the columns of B (n x k, Fortran
    order): CGS with the DGKS test, at most two passes (Sec. 2.3).  Returns the passes."""
    assert z.flags.c_contiguous and B.flags.f_contiguous and z.dtype == B.dtype == np.float64
    return int(_load().orc_reorth_cgs(len(z), _p(z), _p(B), B.shape[1]))


def landos(A, m, nvec, seed=0):
    """Lanczos / Gaussian-quadrature density: nodes, weights (nvec x m) and steps used."""
    nodes = np.zeros((nvec, m))
    weights = np.zeros((nvec, m))
    mused = np.zeros(nvec, dtype=np.int32)
    _load().orc_landos(*_csr_args(A), m, nvec, seed, _p(nodes), _p(weights), _p(mused))
    return dict(nodes=nodes, weights=weights, mused=mused)


def landos_count(d, n, t):
    """Cumulative count N(t) = (n / nvec) sum of the weights of the nodes <= t."""
    nvec = d["nodes"].shape[0]
    tot = 0.0
    for l in range(nvec):
        k = int(d["mused"][l])
        tot += d["weights"][l, :k][d["nodes"][l, :k] <= t].sum()
    return n * tot / nvec


def slicer_landos(d, n, xi, eta, ns):
    """Slices of [xi, eta] with equal quadrature counts (spslicer2 reading)."""
    m = d["nodes"].shape[1]
    nvec = d["nodes"].shape[0]
    sli = np.zeros(ns + 1)
    est = np.zeros(ns)
    nodes = np.ascontiguousarray(d["nodes"])
    weights = np.ascontiguousarray(d["weights"])
    mused = np.ascontiguousarray(d["mused"], dtype=np.int32)
    st = _load().orc_slicer_landos(_p(nodes), _p(weights), mused.ctypes.data_as(C.c_void_p), m, nvec, n,
                                   xi, eta, ns, _p(sli), _p(est))
    if st != 0:
        raise ValueError("no quadrature node in [xi, eta]")
    return sli, est


def lspol(bmin, bmax, eps=1e-13, maxdeg=200):
    """Chebyshev interpolant p(t) ~ 1/t on [bmin, bmax] (the polynomial B^{-1}); returns a dict."""
    coef = np.zeros(maxdeg + 1)
    deg = C.c_int()
    st = _load().orc_lspol(bmin, bmax, eps, maxdeg, C.byref(deg), _p(coef))
    return dict(status=st, deg=deg.value, coef=coef[:deg.value + 1].copy(), bmin=bmin, bmax=bmax)


def lspol_isqrt(bmin, bmax, eps=1e-13, maxdeg=200):
    """Chebyshev interpolant q(t) ~ t^{-1/2} on [bmin, bmax] (the polynomial B^{-1/2}); a dict."""
    coef = np.zeros(maxdeg + 1)
    deg = C.c_int()
    st = _load().orc_lspol_isqrt(bmin, bmax, eps, maxdeg, C.byref(deg), _p(coef))
    return dict(status=st, deg=deg.value, coef=coef[:deg.value + 1].copy(), bmin=bmin, bmax=bmax)


def kpm_moments_gen(A, B, lp, lq, M, nvec, seed, lmin, lmax):
    """KPM moments mu_0..M of the pencil (A, B): p(B) ~ B^{-1} from lp, q(B) ~ B^{-1/2} from lq
    (both on the same [bmin, bmax])."""
    mu = np.zeros(M + 1)
    _load().orc_kpm_moments_gen(*_csr_args(A), *_csr_args(B)[1:], lp["bmin"], lp["bmax"], lp["deg"], _p(lp["coef"]),
                                lq["deg"], _p(lq["coef"]), M, nvec, seed, lmin, lmax, _p(mu))
    return mu


def landos_gen(A, B, lp, lq, m, nvec, seed=0):
    """Lanczos quadrature density of the pencil (A, B) (the density of B^{-1/2} A B^{-1/2}): dict of
    nodes, weights (nvec x m) and mused, as landos."""
    nodes = np.zeros((nvec, m))
    weights = np.zeros((nvec, m))
    mused = np.zeros(nvec, dtype=np.int32)
    _load().orc_landos_gen(*_csr_args(A), *_csr_args(B)[1:], lp["bmin"], lp["bmax"], lp["deg"], _p(lp["coef"]),
                           lq["deg"], _p(lq["coef"]), m, nvec, seed, _p(nodes), _p(weights), _p(mused))
    return dict(nodes=nodes, weights=weights, mused=mused)


def poly_solve(B, lp, x):
    """p(B) x for an lspol dict."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty_like(x)
    _load().orc_polyB_apply(*_csr_args(B), lp["bmin"], lp["bmax"], lp["deg"], _p(lp["coef"]), _p(x), _p(y))
    return y


def bounds_gen(A, B, lp, steps=80, seed=0):
    """Spectral bounds of the pencil (A, B) by B-Lanczos on B^{-1} A."""
    lo, hi = C.c_double(), C.c_double()
    _load().orc_bounds_gen(*_csr_args(A), *_csr_args(B)[1:], lp["bmin"], lp["bmax"], lp["deg"], _p(lp["coef"]),
                           steps, seed, C.byref(lo), C.byref(hi))
    return lo.value, hi.value


def cheblannr_gen(A, B, lp, a, b, pol, m=200, ncycle=10, tol=1e-8, tau1=1e-10, seed=0, cap=None,
                  right_closed=True):
    """Filtered non-restart Lanczos for A x = lambda B x (B-orthonormal eigenvectors)."""
    cap = cap or m
    lam = np.empty(cap)
    res = np.empty(cap)
    X = np.empty((A.n, cap), order="F")
    nev = C.c_int()
    stats = np.zeros(4, dtype=np.int64)
    coef = np.ascontiguousarray(pol["coef"], dtype=np.float64)
    st = _load().orc_cheblannr_gen(*_csr_args(A), *_csr_args(B)[1:], lp["bmin"], lp["bmax"], lp["deg"],
                                   _p(lp["coef"]), a, b, int(right_closed), pol["lmin"], pol["lmax"],
                                   len(coef) - 1, _p(coef), pol["bar"], m, ncycle, tol, tau1, seed, cap,
                                   C.byref(nev), _p(lam), _p(X), _p(res), _p(stats))
    k = nev.value
    return dict(status=st, nev=k, lam=lam[:k].copy(), Y=X[:, :k].copy(), res=res[:k].copy(),
                niter=int(stats[0]), nmv=int(stats[1]))


def cheblantr_gen(A, B, lp, a, b, pol, m=100, maxit=0, ncycle=10, tol=1e-8, tau1=1e-10, seed=0, cap=None,
                  right_closed=True):
    """Filtered thick-restart Lanczos with locking for A x = lambda B x (B-orthonormal
    eigenvectors); stats as cheblantr (npass = 0)."""
    cap = cap or (m + 64)
    maxit = maxit or 20 * m
    lam = np.empty(cap)
    res = np.empty(cap)
    X = np.empty((A.n, cap), order="F")
    nev = C.c_int()
    stats = np.zeros(4, dtype=np.int64)
    coef = np.ascontiguousarray(pol["coef"], dtype=np.float64)
    st = _load().orc_cheblantr_gen(*_csr_args(A), *_csr_args(B)[1:], lp["bmin"], lp["bmax"], lp["deg"],
                                   _p(lp["coef"]), a, b, int(right_closed), pol["lmin"], pol["lmax"],
                                   len(coef) - 1, _p(coef), pol["bar"], m, maxit, ncycle, tol, tau1, seed, cap,
                                   C.byref(nev), _p(lam), _p(X), _p(res), _p(stats))
    k = nev.value
    return dict(status=st, nev=k, lam=lam[:k].copy(), Y=X[:, :k].copy(), res=res[:k].copy(),
                niter=int(stats[0]), nmv=int(stats[1]), nrestart=int(stats[2]))


def chebsi(A, a, b, pol, nv, maxit=100, tol=1e-8, seed=0, cap=None, right_closed=True):
    """Polynomial filtered subspace iteration (ChebSI) with a block of nv vectors.  Returns a
    dict (niter = filter passes that fed a Rayleigh-Ritz step, nmv = all filter matvecs)."""
    cap = cap or nv
    lam = np.empty(cap)
    res = np.empty(cap)
    Y = np.empty((A.n, cap), order="F")
    nev = C.c_int()
    stats = np.zeros(4, dtype=np.int64)
    coef = np.ascontiguousarray(pol["coef"], dtype=np.float64)
    st = _load().orc_chebsi(*_csr_args(A), a, b, int(right_closed), pol["lmin"], pol["lmax"],
                            len(coef) - 1, _p(coef), pol["bar"], nv, maxit, tol, seed, cap, C.byref(nev),
                            _p(lam), _p(Y), _p(res), _p(stats))
    k = nev.value
    order = np.argsort(lam[:k])
    return dict(status=st, nev=k, lam=lam[:k][order].copy(), Y=Y[:, :k][:, order].copy(),
                res=res[:k][order].copy(), niter=int(stats[0]), nmv=int(stats[1]), npass=int(stats[3]))


def cheblannr(A, a, b, pol, m=200, ncycle=10, tol=1e-8, tau1=1e-10, seed=0, cap=None,
              right_closed=True):
    """Filtered non-restart Lanczos (ChebLanNr) with a basis of at most m vectors.  Returns a
    dict (niter, nmv, extractions, npass in place of the restart statistics)."""
    cap = cap or m
    lam = np.empty(cap)
    res = np.empty(cap)
    Y = np.empty((A.n, cap), order="F")
    nev = C.c_int()
    stats = np.zeros(4, dtype=np.int64)
    coef = np.ascontiguousarray(pol["coef"], dtype=np.float64)
    st = _load().orc_cheblannr(*_csr_args(A), a, b, int(right_closed), pol["lmin"], pol["lmax"],
                               len(coef) - 1, _p(coef), pol["bar"], m, ncycle, tol, tau1, seed, cap,
                               C.byref(nev), _p(lam), _p(Y), _p(res), _p(stats))
    k = nev.value
    return dict(status=st, nev=k, lam=lam[:k].copy(), Y=Y[:, :k].copy(), res=res[:k].copy(),
                niter=int(stats[0]), nmv=int(stats[1]), extractions=int(stats[2]),
                npass=int(stats[3]))


def cheblantr(A, a, b, pol, m=100, maxit=None, ncycle=10, tol=1e-8, tau1=1e-10, seed=0,
              cap=None, right_closed=True):
    """Filtered thick-restart Lanczos with locking (Algorithm 2).  Returns a dict."""
    cap = cap or (m + 64)
    maxit = maxit or 20 * m
    lam = np.empty(cap)
    res = np.empty(cap)
    Y = np.empty((A.n, cap), order="F")
    nev = C.c_int()
    stats = np.zeros(4, dtype=np.int64)
    coef = np.ascontiguousarray(pol["coef"], dtype=np.float64)
    st = _load().orc_cheblantr(*_csr_args(A), a, b, int(right_closed), pol["lmin"], pol["lmax"],
                               len(coef) - 1, _p(coef), pol["bar"], m, maxit, ncycle, tol, tau1,
                               seed, cap, C.byref(nev), _p(lam), _p(Y), _p(res), _p(stats))
    k = nev.value
    return dict(status=st, nev=k, lam=lam[:k].copy(), Y=Y[:, :k].copy(), res=res[:k].copy(),
                niter=int(stats[0]), nmv=int(stats[1]), nrestart=int(stats[2]),
                npass=int(stats[3]))
