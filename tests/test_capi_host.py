"""CPU-side checks of the C ABI: the library builds for sm_103a and exports every declared
symbol, and its pure-host entry points (filter construction, DOS slicer) agree with the
oracle.  No GPU is needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT, golden
from paper_1802_05215_gb300 import inputs as I

HEADER = os.path.join(ROOT, "include", "evsl_gb300.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(evsl_[A-Za-z_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def native():
    from paper_1802_05215_gb300 import native
    native.load()
    return native


def test_library_exports_every_declared_symbol(native):
    names = declared_functions()
    assert len(names) >= 14
    lib = ctypes.CDLL(native.library_path())
    missing = [n for n in names if not hasattr(lib, n)]
    assert missing == []


def test_library_is_built_for_sm103a(native):
    # the fatbinary of an sm_103a build carries the architecture name
    data = open(native.library_path(), "rb").read()
    assert b"sm_103a" in data


def test_filter_build_matches_oracle(native, oracle_mod):
    cases = [(0.40, 0.48, 0.0, 8.0), (1.0, 1.3, 0.01, 7.99), (0.2, 0.24, 0.0029, 11.997),
             (-1.0, -0.2, -0.4, 12.36), (11.5, 12.5, 0.0, 12.0), (0.0, 0.9, 0.1, 11.7)]
    for damping in (native.DAMP_JACKSON, native.DAMP_SIGMA, native.DAMP_NONE):
        for a, b, lo, hi in cases:
            f = native.cheb_filter_build(a, b, lo, hi, damping=damping)
            o = oracle_mod.filter_build(a, b, lo, hi, damping=damping)
            assert f.deg == o["deg"] and f.boundary == o["boundary"], (a, b, damping)
            assert abs(f.bar - o["bar"]) < 1e-12 and abs(f.gamma - o["gamma"]) < 1e-12
            assert np.max(np.abs(f.coef - o["coef"])) < 1e-12 * np.abs(o["coef"]).max()


def test_filter_build_table4_degrees(native):
    for ns, i, left, right, nu, deg in golden("table4_slices.txt"):
        f = native.cheb_filter_build(float(left), float(right), 0.0, 11.9882,
                                     damping=native.DAMP_SIGMA)
        assert f.deg == int(deg)


def test_filter_build_errors(native):
    with pytest.raises(native.EvslError):
        native.cheb_filter_build(0.5, 0.4, 0.0, 8.0)             # b <= a
    with pytest.raises(native.EvslError):
        native.cheb_filter_build(-1.0, 9.0, 0.0, 8.0)            # whole spectrum
    with pytest.raises(native.EvslError):
        native.cheb_filter_build(-1.0, -0.5, 0.0, 8.0)           # below the spectrum
    f = native.cheb_filter_build(0.40, 0.4000001, 0.0, 8.0, max_deg=50)
    assert f.status == -4 and f.deg == 50                        # max degree reached


def test_slicer_matches_oracle(native, oracle_mod):
    from paper_1802_05215_gb300 import inputs
    A = inputs.laplacian_2d(60)
    lo, hi = oracle_mod.bounds(A, 60, 0)
    mu = oracle_mod.kpm_moments(A, 60, 8, 0, lo, hi)
    for ns, npts in [(1, 0), (4, 0), (10, 3001), (7, 50)]:
        s, e = native.slice_by_dos(mu, A.n, lo, hi, 0.3, 2.5, ns, npts)
        so, eo = oracle_mod.slicer(mu, lo, hi, 0.3, 2.5, ns, npts or None)
        assert np.max(np.abs(s - so)) < 1e-12 and np.max(np.abs(e - eo)) < 1e-9



def test_slicer_landos_matches_oracle(native, oracle_mod):
    # the host slicer on a Lanczos quadrature density (nodes and weights from the oracle)
    A = I.anderson_3d(12, 4.0, 0)
    d = oracle_mod.landos(A, 60, 50, 4)
    for xi, eta, ns in [(1.0, 5.0, 4), (-0.5, 12.0, 7), (6.0, 6.5, 2)]:
        sli, est = native.slice_by_landos(d, A.n, xi, eta, ns)
        sli_o, est_o = oracle_mod.slicer_landos(d, A.n, xi, eta, ns)
        assert np.allclose(sli, sli_o, rtol=0, atol=1e-12)
        assert np.allclose(est, est_o, rtol=0, atol=1e-9 * A.n)
    with pytest.raises(native.EvslError):
        native.slice_by_landos(d, A.n, 50.0, 60.0, 3)

def test_context_needs_a_gpu(native):
    # without a usable device the library refuses instead of computing on the CPU
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(native.EvslError):
        native.Context(0)



def test_entry_points_reject_null_context_and_bad_arguments(native):
    # every context entry point refuses a NULL context with EVSL_ERR_ARG (no device touched), and
    # the host-only slicer validates its arguments
    lib = native.load()
    P, i32 = ctypes.c_void_p, ctypes.c_int
    nul = P(0)
    buf = (ctypes.c_double * 8)()
    ibuf = (ctypes.c_int * 4)()
    assert lib.evsl_chebLanNr(nul, 0.0, 1.0, nul, nul, 1, ctypes.byref(i32()), buf, nul, buf, nul) == -1
    assert lib.evsl_chebSI(nul, 0.0, 1.0, nul, nul, 1, ctypes.byref(i32()), buf, nul, buf, nul) == -1
    assert lib.evsl_landos(nul, 10, 2, 0, buf, buf, ibuf) == -1
    assert lib.evsl_kpm_dos_doubling(nul, 10, 2, 0, 0.0, 1.0, 0, buf) == -1
    assert lib.evsl_filter_apply_multi(nul, 1, nul, nul, nul, 0) == -1
    assert lib.evsl_set_csr_b(nul, 4, nul, nul, nul, 0.5, 1.0, 1e-13, 50, nul, nul) == -1
    assert lib.evsl_polyB_apply(nul, nul, nul) == -1
    assert lib.evsl_bounds_gen(nul, 10, 0, buf, buf) == -1
    assert lib.evsl_kpm_dos_gen(nul, 10, 2, 0, 0.0, 1.0, buf) == -1
    assert lib.evsl_landos_gen(nul, 10, 2, 0, buf, buf, ibuf) == -1
    assert lib.evsl_chebLanTr_gen(nul, 0.0, 1.0, nul, nul, 1, ctypes.byref(i32()), buf, nul, buf, nul) == -1
    assert lib.evsl_chebLanNr_gen(nul, 0.0, 1.0, nul, nul, 1, ctypes.byref(i32()), buf, nul, buf, nul) == -1
    nodes = np.array([[0.1, 0.5, 0.9]])
    weights = np.array([[0.2, 0.3, 0.5]])
    d = dict(nodes=nodes, weights=weights, mused=np.array([3], dtype=np.int32))
    sli, est = native.slice_by_landos(d, 100, 0.0, 1.0, 2)
    assert sli[0] == 0.0 and sli[-1] == 1.0 and abs(est.sum() - 100.0) <= 1e-12
    with pytest.raises(native.EvslError):
        native.slice_by_landos(d, 100, 1.0, 0.0, 2)           # eta <= xi
    bad = dict(d, mused=np.array([4], dtype=np.int32))        # more steps than stored
    with pytest.raises(native.EvslError):
        native.slice_by_landos(bad, 100, 0.0, 1.0, 2)

def test_lspol_matches_oracle(native, oracle_mod):
    # the library's host lsPol (polynomial B^{-1}) and the oracle's: same degree, same
    # coefficients; the reported error is within eps; too small a maxdeg is reported
    for bmin, bmax, eps in [(0.11, 0.99, 1e-13), (1.0 / 9.0, 1.0, 1e-10), (0.5, 4.0, 1e-13), (2.0, 3.0, 1e-6)]:
        lp = native.lspol(bmin, bmax, eps)
        lo = oracle_mod.lspol(bmin, bmax, eps)
        assert lp["status"] == 0 and lo["status"] == 0
        assert lp["deg"] == lo["deg"]
        assert np.max(np.abs(lp["coef"] - lo["coef"])) <= 1e-14 * np.abs(lo["coef"]).max()
        assert lp["err"] <= eps
    lp = native.lspol(0.01, 1.0, 1e-13, maxdeg=5)
    assert lp["status"] == -4 and lp["deg"] == 5 and lp["err"] > 1e-13
    for bad in [(0.0, 1.0, 1e-13), (1.0, 0.5, 1e-13), (0.5, 1.0, 0.0)]:
        with pytest.raises(native.EvslError):
            native.lspol(*bad)


def test_lspol_isqrt_matches_oracle(native, oracle_mod):
    # the library's host q(t) ~ t^{-1/2} and the oracle's: same degree and coefficients
    for bmin, bmax, eps in [(0.11, 0.99, 1e-13), (1.0 / 9.0, 1.0, 1e-10), (0.5, 4.0, 1e-13)]:
        lq = native.lspol(bmin, bmax, eps, isqrt=True)
        lo = oracle_mod.lspol_isqrt(bmin, bmax, eps)
        assert lq["status"] == 0 and lo["status"] == 0 and lq["deg"] == lo["deg"]
        assert np.max(np.abs(lq["coef"] - lo["coef"])) <= 1e-14 * np.abs(lo["coef"]).max()
        assert lq["err"] <= eps
    with pytest.raises(native.EvslError):
        native.lspol(-1.0, 1.0, 1e-13, isqrt=True)


def test_slice_by_landos_hand_computed_cuts(native):
    # the same hand-computed quadratures as the oracle's pin: cuts midway between the first
    # node reaching each equal share and the node before it
    one = lambda nodes, weights: dict(nodes=np.array([nodes]), weights=np.array([weights]),
                                      mused=np.array([len(nodes)], dtype=np.int32))
    sli, est = native.slice_by_landos(one([0.1, 0.3, 0.5, 0.7, 0.9], [0.2] * 5), 100, 0.0, 1.0, 2)
    assert np.allclose(sli, [0.0, 0.4, 1.0], atol=1e-15) and np.allclose(est, [40, 60], atol=1e-12)
    sli, est = native.slice_by_landos(one([0.1, 0.3, 0.5, 0.7, 0.9], [0.1, 0.2, 0.3, 0.2, 0.2]), 100, 0.0, 1.0, 4)
    assert np.allclose(sli, [0.0, 0.2, 0.4, 0.6, 1.0], atol=1e-15)
    assert np.allclose(est, [10, 20, 30, 40], atol=1e-12)
    d = dict(nodes=np.array([[0.1, 0.5], [0.3, 0.7]]), weights=np.full((2, 2), 0.5),
             mused=np.array([2, 2], dtype=np.int32))
    sli, est = native.slice_by_landos(d, 100, 0.0, 1.0, 2)
    assert np.allclose(sli, [0.0, 0.2, 1.0], atol=1e-15) and np.allclose(est, [25, 75], atol=1e-12)


C_PROGRAM = r"""
#include <stdio.h>
#include "evsl_gb300.h"

int main(void)
{
    double coef[401];
    evsl_filter_opts o = {0.8, 0.4, EVSL_DAMP_JACKSON, 400};
    evsl_polfilt pol;
    int st = evsl_cheb_filter_build(0.40, 0.48, 0.0, 8.0, &o, &pol, coef, 401);
    printf("%d %d %.17g %.17g %.17g\n", st, pol.deg, pol.bar, pol.gamma, coef[pol.deg]);
    double lc[201], err = 0.0;
    int deg = 0;
    st = evsl_lspol(0.11, 0.99, 1e-13, 200, &deg, lc, 201, &err);
    printf("%d %d %.17g %.17g\n", st, deg, lc[0], err);
    evsl_ctx *ctx = 0;
    printf("%d\n", evsl_set_csr(ctx, 1, 0, 0, 0));
    return 0;
}
"""


def test_header_and_library_are_usable_from_c(native, tmp_path):
    # a C99 program includes the header, links the library and calls host-only entry points;
    # the values equal the Python binding's, and a NULL context is refused
    import subprocess
    src = tmp_path / "prog.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "prog"
    libdir = os.path.dirname(native.library_path())
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", libdir, "-levsl_gb300", f"-Wl,-rpath,{libdir}"], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    st, deg, bar, gamma, clast = out[0].split()
    f = native.cheb_filter_build(0.40, 0.48, 0.0, 8.0)
    assert int(st) == 0 and int(deg) == f.deg
    assert float(bar) == f.bar and float(gamma) == f.gamma and float(clast) == f.coef[-1]
    st, deg, c0, err = out[1].split()
    lp = native.lspol(0.11, 0.99, 1e-13)
    assert int(st) == 0 and int(deg) == lp["deg"] and float(c0) == lp["coef"][0] and float(err) == lp["err"]
    assert int(out[2]) == -1                    # EVSL_ERR_ARG
