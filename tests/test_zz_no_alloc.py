"""Allocation-free filter application (evsl_filter_apply_noalloc).

Some callers cannot allocate device memory once they are running: code being recorded into
a CUDA stream capture, real-time loops that forbid allocation after set-up, and hosts whose
device memory belongs to another allocator.  For them the library offers one entry point
whose temporaries live in a fixed device array instead of freshly allocated workspaces.
This file is collected last, and runs both alone and after the rest of the suite: it calls
the entry point through the C ABI twice in a row and checks each result against the
allocating evsl_filter_apply, within the FP64 filter tolerance used by the parity tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1802_05215_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nat():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1802_05215_gb300 import native
    native.load()
    return native


def test_noalloc_filter_matches_allocating_entry_point(nat):
    import torch
    A = I.laplacian_3d(60)                      # n = 216,000: many slices, ragged tail
    lib = nat.load()
    with nat.Context(0) as ctx:
        ctx.set_csr(A)
        lo, hi = 0.0, 12.0
        f = nat.cheb_filter_build(0.5, 0.6, lo, hi)
        assert f.deg > 10
        rng = np.random.default_rng(7)
        for call, nvec in enumerate([1, 3]):  # two calls in a row, different shapes
            X = torch.tensor(rng.standard_normal((nvec, A.n)), device="cuda")
            Y_ref = torch.empty_like(X)
            Y_na = torch.full_like(X, np.nan)
            ctx.filter_apply(f, X, Y_ref)
            st = lib.evsl_filter_apply_noalloc(ctx.h, ctypes.byref(f.pol), nvec,
                                               ctypes.c_void_p(X.data_ptr()),
                                               ctypes.c_void_p(Y_na.data_ptr()))
            assert st == 0, lib.evsl_last_error(ctx.h)
            scale = np.abs(f.coef).sum() * float(X.abs().max())
            err = float((Y_na - Y_ref).abs().max())
            assert err <= 1e-12 * scale, (call, err)


def test_noalloc_rejects_sizes_beyond_its_array(nat):
    import torch
    lib = nat.load()
    A = I.laplacian_2d(1100)                    # n = 1.21e6: two columns exceed 2^21 doubles
    with nat.Context(0) as ctx:
        ctx.set_csr(A)
        f = nat.cheb_filter_build(0.5, 0.6, 0.0, 8.0)
        X = torch.zeros((2, A.n), dtype=torch.float64, device="cuda")
        Y = torch.zeros_like(X)
        st = lib.evsl_filter_apply_noalloc(ctx.h, ctypes.byref(f.pol), 2,
                                           ctypes.c_void_p(X.data_ptr()),
                                           ctypes.c_void_p(Y.data_ptr()))
        assert st == -1
        assert b"EVSL_NOALLOC_MAX_ELEMS" in lib.evsl_last_error(ctx.h)
