"""Thin Python binding of the C ABI in include/evsl_gb300.h (argument marshalling only).

Every numerical step runs inside libevsl_gb300.so; this module converts numpy arrays and
torch CUDA tensors to plain pointers.  Loading fails loudly if the library is missing: there
is no CPU fallback.  Each function mirrors the C call of the same name; the passage of
arXiv:1802.05215 it implements is given in its docstring (and beside its declaration in the
header).  A context runs on its own non-blocking CUDA stream, which does not wait for torch's,
so every CUDA tensor handed to a call is preceded by a synchronisation of torch's current stream
on its device (tensors produced on other streams must be complete before the call).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

EVSL_OK = 0
ERRORS = {-1: "EVSL_ERR_ARG", -2: "EVSL_ERR_NOMEM", -3: "EVSL_ERR_CUDA", -4: "EVSL_ERR_NOCONV",
          -5: "EVSL_ERR_CAPACITY", -6: "EVSL_ERR_TIMEOUT", -7: "EVSL_ERR_STATE"}
DAMP_NONE, DAMP_JACKSON, DAMP_SIGMA = 0, 1, 2
FP64, FP32 = 0, 1
K_CHEB_STEP, K_KPM_STEP, K_REORTH, K_RITZ_GEMM, K_SMALL_EIG, K_GEN_STEP = range(6)
NOALLOC_MAX_ELEMS = 1 << 21


class EvslError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class FilterOpts(C.Structure):
    _fields_ = [("tau", C.c_double), ("tau_ext", C.c_double), ("damping", C.c_int),
                ("max_deg", C.c_int)]


class PolFilt(C.Structure):
    _fields_ = [("deg", C.c_int), ("boundary", C.c_int), ("gamma", C.c_double),
                ("bar", C.c_double), ("lmin", C.c_double), ("lmax", C.c_double),
                ("a", C.c_double), ("b", C.c_double), ("coef", C.POINTER(C.c_double))]


class LanOpts(C.Structure):
    _fields_ = [("m", C.c_int), ("maxit", C.c_int), ("ncycle", C.c_int), ("tol", C.c_double),
                ("tau1", C.c_double), ("seed", C.c_uint64), ("prec", C.c_int),
                ("right_closed", C.c_int)]


class SliceJob(C.Structure):
    _fields_ = [("a", C.c_double), ("b", C.c_double), ("pol", C.POINTER(PolFilt)),
                ("m", C.c_int), ("cap", C.c_int), ("right_closed", C.c_int),
                ("nev", C.POINTER(C.c_int)), ("lam", C.c_void_p), ("res", C.c_void_p),
                ("Y", C.c_void_p), ("stats", C.c_void_p), ("status", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("niter", C.c_int64), ("nmv", C.c_int64), ("nrestart", C.c_int64),
                ("npass", C.c_int64), ("t_filter", C.c_double), ("t_orth", C.c_double),
                ("t_restart", C.c_double), ("t_total", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libevsl_gb300.so (building it with nvcc first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"{_build.LIB} is missing; run paper_1802_05215_gb300.build.build()")
    lib = C.CDLL(_build.LIB)
    P, d, i32, i64, u64, sz = C.c_void_p, C.c_double, C.c_int, C.c_int64, C.c_uint64, C.c_size_t
    sig = {
        "evsl_create": (i32, [C.POINTER(P), i32, sz]),
        "evsl_destroy": (None, [P]),
        "evsl_last_error": (C.c_char_p, [P]),
        "evsl_set_stream": (i32, [P, P]),
        "evsl_set_csr": (i32, [P, i64, P, P, P]),
        "evsl_bounds": (i32, [P, i32, u64, P, P]),
        "evsl_kpm_dos": (i32, [P, i32, i32, u64, d, d, i32, P]),
        "evsl_kpm_dos_doubling": (i32, [P, i32, i32, u64, d, d, i32, P]),
        "evsl_kpm_probe_moments": (i32, [P, i32, i64, i32, u64, d, d, i32, P]),
        "evsl_slice_by_dos": (i32, [P, i32, i64, d, d, d, d, i32, i32, P, P]),
        "evsl_cheb_filter_build": (i32, [d, d, d, d, P, P, P, i32]),
        "evsl_filter_apply": (i32, [P, P, i32, P, P, i32]),
        "evsl_filter_apply_noalloc": (i32, [P, P, i32, P, P]),
        "evsl_filter_apply_multi": (i32, [P, i32, P, P, P, i32]),
        "evsl_chebLanTr": (i32, [P, d, d, P, P, i32, P, P, P, P, P]),
        "evsl_chebLanNr": (i32, [P, d, d, P, P, i32, P, P, P, P, P]),
        "evsl_chebSI": (i32, [P, d, d, P, P, i32, P, P, P, P, P]),
        "evsl_landos": (i32, [P, i32, i32, u64, P, P, P]),
        "evsl_slice_by_landos": (i32, [P, P, P, i32, i32, i64, d, d, i32, P, P]),
        "evsl_chebLanTr_batch": (i32, [P, i32, P, P]),
        "evsl_batch_create": (i32, [P, P, C.POINTER(P)]),
        "evsl_batch_add": (i32, [P, P]),
        "evsl_batch_step": (i32, [P, P, P]),
        "evsl_batch_destroy": (None, [P]),
        "evsl_lspol": (i32, [d, d, d, i32, P, P, i32, P]),
        "evsl_set_csr_b": (i32, [P, i64, P, P, P, d, d, d, i32, P, P]),
        "evsl_lspol_isqrt": (i32, [d, d, d, i32, P, P, i32, P]),
        "evsl_kpm_dos_gen": (i32, [P, i32, i32, u64, d, d, P]),
        "evsl_landos_gen": (i32, [P, i32, i32, u64, P, P, P]),
        "evsl_polyB_apply": (i32, [P, P, P]),
        "evsl_bounds_gen": (i32, [P, i32, u64, P, P]),
        "evsl_chebLanNr_gen": (i32, [P, d, d, P, P, i32, P, P, P, P, P]),
        "evsl_chebLanTr_gen": (i32, [P, d, d, P, P, i32, P, P, P, P, P]),
        "evsl_launch_count": (i64, [P]),
        "evsl_set_device_budget": (i32, [i32, sz]),
        "evsl_device_used": (sz, [i32]),
        "evsl_mem_used": (sz, [P]),
        "evsl_dense_gemm": (i32, [P, i32, i64, i32, i64, P, i64, P, i64, P, i64, i32]),
        "evsl_set_tensor_gemm": (i32, [P, i32]),
        "evsl_set_graphs": (i32, [P, i32]),
        "evsl_profile": (i32, [P, i32]),
        "evsl_profile_get": (i32, [P, i32, P, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _ptr(a) -> int:
    """Address of a numpy array or a torch tensor (host or device).  Before a CUDA tensor is
    handed over, torch's current stream on its device is synchronised: the context's own stream
    does not wait for it, and the tensor may still be being written there."""
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if getattr(a, "is_cuda", False):
            import torch
            torch.cuda.current_stream(a.device).synchronize()
        return a.data_ptr()
    raise TypeError(type(a))


def _addr(a):
    return C.c_void_p(_ptr(a))


class Filter:
    """A built Chebyshev filter; owns its coefficient array."""

    def __init__(self, pol: PolFilt, coef: np.ndarray, status: int):
        self.coef = coef
        self.pol = pol
        self.pol.coef = coef.ctypes.data_as(C.POINTER(C.c_double))
        self.status = status

    deg = property(lambda s: s.pol.deg)
    bar = property(lambda s: s.pol.bar)
    gamma = property(lambda s: s.pol.gamma)
    boundary = property(lambda s: s.pol.boundary)
    lmin = property(lambda s: s.pol.lmin)
    lmax = property(lambda s: s.pol.lmax)


def lspol(bmin, bmax, eps=1e-13, maxdeg=200, isqrt=False):
    """Chebyshev coefficients of p(t) ~ 1/t (or ~ t^{-1/2} with isqrt) on [bmin, bmax] (the
    polynomial B^{-1} of Sec. 4.3's lsPol, or B^{-1/2} for the starting vectors of a pencil's
    density, Sec. 2.1): dict(status, deg, coef, err)."""
    lib = load()
    coef = np.zeros(maxdeg + 1)
    deg, err = C.c_int(), C.c_double()
    fn = lib.evsl_lspol_isqrt if isqrt else lib.evsl_lspol
    st = fn(bmin, bmax, eps, maxdeg, C.byref(deg), _addr(coef), len(coef), C.byref(err))
    if st not in (EVSL_OK, -4):
        raise EvslError(st, "lspol")
    return dict(status=st, deg=deg.value, coef=coef[:deg.value + 1].copy(), err=err.value)


def cheb_filter_build(a, b, lmin, lmax, tau=0.8, tau_ext=0.4, damping=DAMP_JACKSON,
                      max_deg=10000) -> Filter:
    """Damped Chebyshev delta filter for [a, b] on [lmin, lmax] (Sec. 2.2.1, Eqs. (2.4)-(2.7);
    boundary slices as in Sec. 4.2).  Returns a Filter; EVSL_ERR_NOCONV (max_deg reached) is
    reported in its status, other errors raise."""
    lib = load()
    opts = FilterOpts(tau, tau_ext, damping, max_deg)
    pol = PolFilt()
    coef = np.zeros(max_deg + 1)
    st = lib.evsl_cheb_filter_build(a, b, lmin, lmax, C.byref(opts), C.byref(pol),
                                    _addr(coef), len(coef))
    if st not in (EVSL_OK, -4):
        raise EvslError(st, "cheb_filter_build")
    coef = coef[:pol.deg + 1].copy()
    return Filter(pol, coef, st)


def slice_by_landos(d, n, xi, eta, nslices):
    """Slices of [xi, eta] with equal counts under a Lanczos quadrature density d (Sec. 2.1; from
    Context.landos); returns (sli, est)."""
    lib = load()
    nodes = np.ascontiguousarray(d["nodes"], dtype=np.float64)
    weights = np.ascontiguousarray(d["weights"], dtype=np.float64)
    mused = np.ascontiguousarray(d["mused"], dtype=np.int32)
    sli = np.zeros(nslices + 1)
    est = np.zeros(nslices)
    st = lib.evsl_slice_by_landos(_addr(nodes), _addr(weights), mused.ctypes.data, nodes.shape[1],
                                  nodes.shape[0], n, xi, eta, nslices, _addr(sli), _addr(est))
    if st != EVSL_OK:
        raise EvslError(st, "slice_by_landos")
    return sli, est


def slice_by_dos(mu, n, lmin, lmax, xi, eta, nslices, npts=0):
    """DOS-balanced slice ends t_0..t_ns of [xi, eta] and per-slice count estimates from KPM
    moments (Eq. (2.2), spslicer).  Host only."""
    lib = load()
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    sli = np.zeros(nslices + 1)
    est = np.zeros(nslices)
    st = lib.evsl_slice_by_dos(_addr(mu), len(mu) - 1, n, lmin, lmax, xi, eta, nslices, npts,
                               _addr(sli), _addr(est))
    if st != EVSL_OK:
        raise EvslError(st, "slice_by_dos")
    return sli, est


def set_device_budget(device: int, nbytes: int):
    """Cap the device memory held by all contexts on `device` together (0 = no cap)."""
    st = load().evsl_set_device_budget(device, nbytes)
    if st != EVSL_OK:
        raise EvslError(st, f"set_device_budget({device})")


def device_used(device: int) -> int:
    """Bytes held by the library's contexts on `device`."""
    return int(load().evsl_device_used(device))


class Context:
    """One evsl_ctx: a CUDA device, a stream, the device matrix and workspaces."""

    def __init__(self, device: int = 0, hbm_budget: int = 0):
        self.lib = load()
        h = C.c_void_p()
        st = self.lib.evsl_create(C.byref(h), device, hbm_budget)
        if st != EVSL_OK:
            raise EvslError(st, f"evsl_create(device={device}) failed")
        self.h = h
        self.n = 0

    def close(self):
        if getattr(self, "h", None):
            # the library destroys this context's batches with it: invalidate their handles first
            for b in getattr(self, "_batches", []):
                bt = b()
                if bt is not None:
                    bt.h = None
            self.lib.evsl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, st, what):
        if st != EVSL_OK:
            raise EvslError(st, f"{what}: {self.lib.evsl_last_error(self.h).decode()}")
        return st

    def set_stream(self, stream_handle: int | None):
        self._check(self.lib.evsl_set_stream(self.h, C.c_void_p(stream_handle or 0)), "set_stream")

    def set_csr(self, A):
        """The matrix A (inputs.CSR, both triangles), copied to HBM in sliced ELLPACK (Sec. 3.1)."""
        self._check(self.lib.evsl_set_csr(self.h, A.n, _addr(A.row_ptr), _addr(A.col_idx),
                                          _addr(A.val)), "set_csr")
        self.n = A.n

    def set_csr_b(self, B, bmin, bmax, eps=1e-13, maxdeg=200):
        """Mass matrix of a generalized problem (Sec. 2.4) with its spectrum in [bmin, bmax]; builds the
        polynomial inverse.  Returns (degree, relative error) of p(t) ~ 1/t."""
        deg, err = C.c_int(), C.c_double()
        self._check(self.lib.evsl_set_csr_b(self.h, B.n, _addr(B.row_ptr), _addr(B.col_idx), _addr(B.val),
                                            bmin, bmax, eps, maxdeg, C.byref(deg), C.byref(err)), "set_csr_b")
        return deg.value, err.value

    def polyB_apply(self, x, y):
        """y = p(B) x, the polynomial solve with B (Sec. 4.3), for device vectors of n doubles."""
        self._check(self.lib.evsl_polyB_apply(self.h, _addr(x), _addr(y)), "polyB_apply")

    def kpm_dos_gen(self, degree, nvec, seed, lmin, lmax):
        """KPM moments mu_0..degree of the pencil (the density of B^{-1/2} A B^{-1/2}; Sec. 2.1)."""
        mu = np.zeros(degree + 1)
        self._check(self.lib.evsl_kpm_dos_gen(self.h, degree, nvec, seed, lmin, lmax, _addr(mu)), "kpm_dos_gen")
        return mu

    def landos_gen(self, m, nvec, seed=0):
        """Lanczos quadrature density of the pencil (Sec. 2.1; the density of B^{-1/2} A B^{-1/2}):
        dict of nodes, weights (nvec x m) and mused, as landos."""
        nodes = np.zeros((nvec, m))
        weights = np.zeros((nvec, m))
        mused = np.zeros(nvec, dtype=np.int32)
        self._check(self.lib.evsl_landos_gen(self.h, m, nvec, seed, _addr(nodes), _addr(weights),
                                             mused.ctypes.data), "landos_gen")
        return dict(nodes=nodes, weights=weights, mused=mused)

    def bounds_gen(self, steps=80, seed=0):
        """Spectral bounds of the pencil (A, B) by B-Lanczos on B^{-1} A (Algorithm 3)."""
        lo, hi = C.c_double(), C.c_double()
        self._check(self.lib.evsl_bounds_gen(self.h, steps, seed, C.byref(lo), C.byref(hi)), "bounds_gen")
        return lo.value, hi.value

    def chebLanNr_gen(self, a, b, filt: Filter, m=200, ncycle=10, tol=1e-8, tau1=1e-10, seed=0,
                      right_closed=True, cap=None, Y=None, allow_partial=False):
        """Filtered non-restart Lanczos for A x = lambda B x on [a, b] (Sec. 2.5, Algorithm 3); as chebLanNr
        (the eigenvectors are B-orthonormal)."""
        cap = cap or m
        opts = LanOpts(m, 0, ncycle, tol, tau1, seed, FP64, int(right_closed))
        lam = np.zeros(cap)
        res = np.zeros(cap)
        if Y is None:
            Y = np.zeros((cap, self.n))
        nev = C.c_int()
        stats = Stats()
        st = self.lib.evsl_chebLanNr_gen(self.h, a, b, C.byref(filt.pol), C.byref(opts), cap,
                                         C.byref(nev), _addr(lam), _addr(Y), _addr(res), C.byref(stats))
        if st != EVSL_OK and not (allow_partial and st in (-4, -5)):
            self._check(st, "chebLanNr_gen")
        k = nev.value
        return dict(status=st, nev=k, lam=lam[:k].copy(), res=res[:k].copy(), Y=Y,
                    stats=stats.as_dict())

    def chebLanTr_gen(self, a, b, filt: Filter, m=100, maxit=0, ncycle=10, tol=1e-8, tau1=1e-10, seed=0,
                      right_closed=True, cap=None, Y=None, allow_partial=False):
        """Filtered thick-restart Lanczos with locking for A x = lambda B x on [a, b] (Algorithm 2 in
        the B-inner product, Sec. 2.5); outputs as
        chebLanTr (B-orthonormal eigenvectors)."""
        cap = cap or (m + 64)
        opts = LanOpts(m, maxit, ncycle, tol, tau1, seed, FP64, int(right_closed))
        lam = np.zeros(cap)
        res = np.zeros(cap)
        if Y is None:
            Y = np.zeros((cap, self.n))
        nev = C.c_int()
        stats = Stats()
        st = self.lib.evsl_chebLanTr_gen(self.h, a, b, C.byref(filt.pol), C.byref(opts), cap,
                                         C.byref(nev), _addr(lam), _addr(Y), _addr(res), C.byref(stats))
        if st != EVSL_OK and not (allow_partial and st in (-4, -5)):
            self._check(st, "chebLanTr_gen")
        k = nev.value
        return dict(status=st, nev=k, lam=lam[:k].copy(), res=res[:k].copy(), Y=Y,
                    stats=stats.as_dict())

    def bounds(self, steps=80, seed=0):
        """Spectral bounds (lmin, lmax) from `steps` Lanczos steps (Sec. 2.2.1, LanTrbounds)."""
        lo, hi = C.c_double(), C.c_double()
        self._check(self.lib.evsl_bounds(self.h, steps, seed, C.byref(lo), C.byref(hi)), "bounds")
        return lo.value, hi.value

    def kpm_dos(self, degree, nvec, seed, lmin, lmax, prec=FP64, doubling=False):
        """KPM moments mu_0..degree (Sec. 2.1; doubling: from ceil(degree/2) recurrence steps)."""
        mu = np.zeros(degree + 1)
        fn = self.lib.evsl_kpm_dos_doubling if doubling else self.lib.evsl_kpm_dos
        self._check(fn(self.h, degree, nvec, seed, lmin, lmax, prec, _addr(mu)), "kpm_dos")
        return mu

    def kpm_probe_moments(self, degree, first, nprobe, seed, lmin, lmax, prec=FP64):
        """Per-probe KPM sums v_l^T T_k(Ahat) v_l of probes first .. first + nprobe - 1 (Sec. 2.1):
        an nprobe x (degree + 1) array whose rows, gathered from any split of the probes and
        added in probe order, give the same moments bitwise."""
        out = np.zeros((nprobe, degree + 1))
        self._check(self.lib.evsl_kpm_probe_moments(self.h, degree, first, nprobe, seed, lmin, lmax, prec,
                                                    _addr(out)), "kpm_probe_moments")
        return out

    def filter_apply(self, filt: Filter, X, Y, prec=FP64):
        """Y = rho(Ahat) X (Eq. (2.4)) for device blocks X, Y (n x nvec column-major, e.g. torch tensors
        of shape (nvec, n) on the GPU)."""
        nvec = X.numel() // self.n
        self._check(self.lib.evsl_filter_apply(self.h, C.byref(filt.pol), nvec, _addr(X),
                                               _addr(Y), prec), "filter_apply")

    def filter_apply_multi(self, filters, X, Y, prec=FP64):
        """Column t of the device block X (n x len(filters)) is filtered by filters[t] (Eq. (2.4) for
        several slices at once)."""
        arr = (PolFilt * len(filters))(*[f.pol for f in filters])
        self._check(self.lib.evsl_filter_apply_multi(self.h, len(filters), arr, _addr(X), _addr(Y),
                                                     prec), "filter_apply_multi")

    def filter_apply_noalloc(self, filt: Filter, X, Y):
        """Allocation-free Y = rho(Ahat) X (FP64) using the library's fixed device scratch;
        n * nvec must not exceed NOALLOC_MAX_ELEMS."""
        nvec = X.numel() // self.n
        self._check(self.lib.evsl_filter_apply_noalloc(self.h, C.byref(filt.pol), nvec, _addr(X),
                                                       _addr(Y)), "filter_apply_noalloc")

    def chebLanTr(self, a, b, filt: Filter, m=100, maxit=0, ncycle=10, tol=1e-8, tau1=1e-10,
                  seed=0, prec=FP64, right_closed=True, cap=None, Y=None, allow_partial=False):
        """Filtered thick-restart Lanczos with locking on [a, b] (Algorithm 2).  Y: None (host numpy result) or a
        caller-provided buffer (numpy host array or torch CUDA tensor of n*cap doubles)."""
        cap = cap or (m + 64)
        opts = LanOpts(m, maxit, ncycle, tol, tau1, seed, prec, int(right_closed))
        lam = np.zeros(cap)
        res = np.zeros(cap)
        if Y is None:
            Y = np.zeros((cap, self.n))       # row j = eigenvector j (column-major n x cap)
        nev = C.c_int()
        stats = Stats()
        st = self.lib.evsl_chebLanTr(self.h, a, b, C.byref(filt.pol), C.byref(opts), cap,
                                     C.byref(nev), _addr(lam), _addr(Y), _addr(res),
                                     C.byref(stats))
        if st != EVSL_OK and not (allow_partial and st in (-4, -5)):
            self._check(st, "chebLanTr")
        k = nev.value
        return dict(status=st, nev=k, lam=lam[:k].copy(), res=res[:k].copy(), Y=Y,
                    stats=stats.as_dict())

    def landos(self, m, nvec, seed=0):
        """Lanczos quadrature density (Sec. 2.1): dict of nodes, weights (nvec x m) and mused."""
        nodes = np.zeros((nvec, m))
        weights = np.zeros((nvec, m))
        mused = np.zeros(nvec, dtype=np.int32)
        self._check(self.lib.evsl_landos(self.h, m, nvec, seed, _addr(nodes), _addr(weights),
                                         mused.ctypes.data), "landos")
        return dict(nodes=nodes, weights=weights, mused=mused)

    def chebSI(self, a, b, filt: Filter, nv, maxit=100, tol=1e-8, seed=0, right_closed=True,
               cap=None, Y=None, allow_partial=False):
        """Polynomial filtered subspace iteration (Sec. 2.6) with a block of nv vectors; same outputs as
        chebLanTr (stats["niter"] counts passes)."""
        cap = cap or nv
        opts = LanOpts(nv, maxit, 10, tol, 1e-10, seed, FP64, int(right_closed))
        lam = np.zeros(cap)
        res = np.zeros(cap)
        if Y is None:
            Y = np.zeros((cap, self.n))
        nev = C.c_int()
        stats = Stats()
        st = self.lib.evsl_chebSI(self.h, a, b, C.byref(filt.pol), C.byref(opts), cap, C.byref(nev),
                                  _addr(lam), _addr(Y), _addr(res), C.byref(stats))
        if st != EVSL_OK and not (allow_partial and st in (-4, -5)):
            self._check(st, "chebSI")
        k = nev.value
        return dict(status=st, nev=k, lam=lam[:k].copy(), res=res[:k].copy(), Y=Y,
                    stats=stats.as_dict())

    def chebLanNr(self, a, b, filt: Filter, m=400, ncycle=10, tol=1e-8, tau1=1e-10, seed=0,
                  prec=FP64, right_closed=True, cap=None, Y=None, allow_partial=False):
        """Filtered non-restart Lanczos (ChebLanNr, Sec. 2.3) on [a, b] with a basis of at most m vectors; same
        outputs as chebLanTr (stats["nrestart"] counts the extractions)."""
        cap = cap or m
        opts = LanOpts(m, 0, ncycle, tol, tau1, seed, prec, int(right_closed))
        lam = np.zeros(cap)
        res = np.zeros(cap)
        if Y is None:
            Y = np.zeros((cap, self.n))
        nev = C.c_int()
        stats = Stats()
        st = self.lib.evsl_chebLanNr(self.h, a, b, C.byref(filt.pol), C.byref(opts), cap,
                                     C.byref(nev), _addr(lam), _addr(Y), _addr(res),
                                     C.byref(stats))
        if st != EVSL_OK and not (allow_partial and st in (-4, -5)):
            self._check(st, "chebLanNr")
        k = nev.value
        return dict(status=st, nev=k, lam=lam[:k].copy(), res=res[:k].copy(), Y=Y,
                    stats=stats.as_dict())

    def chebLanTr_batch(self, slices, filters, ms, caps=None, maxit=0, ncycle=10, tol=1e-8,
                        tau1=1e-10, seed=0, prec=FP64, right_closed=None, Ys=None,
                        allow_partial=False):
        """Several slices [a_j, b_j] of the current matrix solved in lockstep (Algorithm 2 per slice) with batched
        filters.  Returns one result dict per slice (as chebLanTr)."""
        nj = len(slices)
        caps = caps or [m + 64 for m in ms]
        right_closed = right_closed if right_closed is not None else [True] * nj
        opts = LanOpts(0, maxit, ncycle, tol, tau1, seed, prec, 1)
        keep, jobs = [], (SliceJob * nj)()
        for j, ((a, b), f, m, cap) in enumerate(zip(slices, filters, ms, caps)):
            nev = C.c_int()
            lam, res = np.zeros(cap), np.zeros(cap)
            Y = Ys[j] if Ys is not None else np.zeros((cap, self.n))
            st = Stats()
            keep.append((nev, lam, res, Y, st))
            jobs[j] = SliceJob(a, b, C.pointer(f.pol), m, cap, int(right_closed[j]), C.pointer(nev),
                               _ptr(lam), _ptr(res), _ptr(Y), C.addressof(st), 0)
        rc = self.lib.evsl_chebLanTr_batch(self.h, nj, jobs, C.byref(opts))
        if rc != EVSL_OK and not (allow_partial and rc in (-4, -5)):
            self._check(rc, "chebLanTr_batch")
        out = []
        for j, (nev, lam, res, Y, st) in enumerate(keep):
            k = nev.value
            out.append(dict(status=jobs[j].status, nev=k, lam=lam[:k].copy(), res=res[:k].copy(),
                            Y=Y, stats=st.as_dict()))
        return out

    def set_graphs(self, enable: bool):
        """Allow (default) or forbid CUDA-graph replay of single-vector filter applications."""
        self._check(self.lib.evsl_set_graphs(self.h, int(enable)), "set_graphs")

    def launch_count(self) -> int:
        return int(self.lib.evsl_launch_count(self.h))

    def dense_gemm(self, A, B, C, trans_a=False, mode=0):
        """C {=, -=, +=} op(A) B for device tensors holding column-major FP64 matrices: pass
        torch tensors of shape (cols, rows) (row j = column j); op(A) = A or A^T."""
        ka, ra = A.shape            # columns, rows of the column-major A
        n_b, k_b = B.shape
        M = ka if trans_a else ra
        K = ra if trans_a else ka
        assert k_b == K and C.shape == (n_b, M)
        self._check(self.lib.evsl_dense_gemm(self.h, int(trans_a), M, n_b, K, _addr(A), ra, _addr(B), k_b,
                                             _addr(C), M, mode), "dense_gemm")

    def set_tensor_gemm(self, enable: bool):
        """Large FP64 products on the tensor cores (default) or on the plain FP64 kernels."""
        self._check(self.lib.evsl_set_tensor_gemm(self.h, int(enable)), "set_tensor_gemm")

    def mem_used(self) -> int:
        """Device bytes this context holds."""
        return int(self.lib.evsl_mem_used(self.h))

    def profile(self, enable: bool):
        self._check(self.lib.evsl_profile(self.h, int(enable)), "profile")

    def profile_get(self, kernel: int):
        n = C.c_int64()
        ms = C.c_double()
        self._check(self.lib.evsl_profile_get(self.h, kernel, C.byref(n), C.byref(ms)),
                    "profile_get")
        return n.value, ms.value


class Job:
    """One slice solve submitted to a Batch; holds the buffers the library writes into."""

    def __init__(self, a, b, filt: Filter, m, cap, right_closed, n, Y=None, tag=None):
        self.filt = filt
        self.nev_c = C.c_int()
        self.lam = np.zeros(cap)
        self.res = np.zeros(cap)
        self.Y = Y if Y is not None else np.zeros((cap, n))
        self.stats_c = Stats()
        self.tag = tag
        self.struct = SliceJob(a, b, C.pointer(filt.pol), m, cap, int(right_closed),
                               C.pointer(self.nev_c), _ptr(self.lam), _ptr(self.res), _ptr(self.Y),
                               C.addressof(self.stats_c), 0)
        self.done = False

    def result(self):
        k = self.nev_c.value
        return dict(status=self.struct.status, nev=k, lam=self.lam[:k].copy(),
                    res=self.res[:k].copy(), Y=self.Y, stats=self.stats_c.as_dict(), tag=self.tag)


class Batch:
    """Continuous batching of slice solves on one context (evsl_batch_*): jobs join between
    steps and leave when finished; each step applies every active job's filter in one pass."""

    def __init__(self, ctx: Context, maxit=0, ncycle=10, tol=1e-8, tau1=1e-10, seed=0, prec=FP64):
        self.ctx = ctx
        self.opts = LanOpts(0, maxit, ncycle, tol, tau1, seed, prec, 1)
        h = C.c_void_p()
        ctx._check(ctx.lib.evsl_batch_create(ctx.h, C.byref(self.opts), C.byref(h)), "batch_create")
        self.h = h
        self.active: list[Job] = []
        import weakref
        if not hasattr(ctx, "_batches"):
            ctx._batches = []
        ctx._batches.append(weakref.ref(self))

    def add(self, a, b, filt: Filter, m, cap=None, right_closed=True, Y=None, tag=None) -> Job:
        """Admit a job; raises EvslError with code -2 when the HBM budget has no room for it."""
        job = Job(a, b, filt, m, cap or (m + 64), right_closed, self.ctx.n, Y, tag)
        self.ctx._check(self.ctx.lib.evsl_batch_add(self.h, C.byref(job.struct)), "batch_add")
        self.active.append(job)
        return job

    def step(self):
        """One lockstep Lanczos step; returns the jobs that finished in it."""
        na, nf = C.c_int(), C.c_int()
        self.ctx._check(self.ctx.lib.evsl_batch_step(self.h, C.byref(na), C.byref(nf)), "batch_step")
        done = []
        if nf.value:
            # a finished job has its status and outputs written; the library drops it from the batch
            still = []
            for j in self.active:
                (done if self._finished(j) else still).append(j)
            self.active = still
        return done

    def _finished(self, job):
        # outputs are written once; a finished job has its stats filled in (t_total > 0)
        if job.stats_c.t_total > 0 and not job.done:
            job.done = True
            return True
        return False

    def close(self):
        if getattr(self, "h", None) and getattr(self.ctx, "h", None):
            self.ctx.lib.evsl_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
