"""Allocation-free filter application (evsl_filter_apply_noalloc).

Some callers cannot allocate device memory once they are running: hosts whose device memory
belongs to another allocator (a framework's caching pool that owns the GPU), and real-time
loops that forbid allocation after set-up because cudaMalloc and cudaFree can block and
synchronise the device.  For them the library offers one entry point whose temporaries live in
a fixed device array instead of freshly allocated workspaces.  This file is collected last,
and runs both alone and after the rest of the suite: it calls the entry point through the C
ABI twice in a row on a fresh context (the unmapped-values branch), then twice more after the
allocating evsl_filter_apply has made the mapped values current, and checks every result
against the allocating entry point within the FP64 filter tolerance of the parity tests.
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


def _noalloc(lib, ctx, f, X, Y):
    # the raw C call: torch's work on X and Y (fills, copies) must be complete first, since the
    # context's stream does not wait for torch's
    import torch
    torch.cuda.current_stream().synchronize()
    return lib.evsl_filter_apply_noalloc(ctx.h, ctypes.byref(f.pol), X.shape[0],
                                         ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()))


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
        Xs = [torch.tensor(rng.standard_normal((nvec, A.n)), device="cuda") for nvec in (1, 3)]
        # two calls in a row on a fresh context: the mapped values do not exist yet
        fresh = []
        for X in Xs:
            Y = torch.full_like(X, np.nan)
            assert _noalloc(lib, ctx, f, X, Y) == 0, lib.evsl_last_error(ctx.h)
            fresh.append(Y)
        for X, Y_fresh in zip(Xs, fresh):
            Y_ref = torch.empty_like(X)
            ctx.filter_apply(f, X, Y_ref)        # allocating path; makes the mapped values current
            Y_mapped = torch.full_like(X, np.nan)
            assert _noalloc(lib, ctx, f, X, Y_mapped) == 0, lib.evsl_last_error(ctx.h)
            scale = np.abs(f.coef).sum() * float(X.abs().max())
            for Y in (Y_fresh, Y_mapped):
                err = float((Y - Y_ref).abs().max())
                assert err <= 1e-12 * scale, (X.shape[0], err)


def test_noalloc_restores_the_callers_current_device(nat):
    import torch
    lib = nat.load()
    A = I.laplacian_2d(40)
    with nat.Context(0) as ctx:
        ctx.set_csr(A)
        f = nat.cheb_filter_build(1.0, 1.2, 0.0, 8.0)
        X = torch.ones((1, A.n), dtype=torch.float64, device="cuda")
        Y = torch.empty_like(X)
        before = torch.cuda.current_device()
        assert _noalloc(lib, ctx, f, X, Y) == 0, lib.evsl_last_error(ctx.h)
        assert torch.cuda.current_device() == before


def test_noalloc_rejects_sizes_beyond_its_array(nat):
    import torch
    lib = nat.load()
    A = I.laplacian_2d(1100)                    # n = 1.21e6: two columns exceed 2^21 doubles
    with nat.Context(0) as ctx:
        ctx.set_csr(A)
        f = nat.cheb_filter_build(0.5, 0.6, 0.0, 8.0)
        X = torch.zeros((2, A.n), dtype=torch.float64, device="cuda")
        Y = torch.zeros_like(X)
        assert _noalloc(lib, ctx, f, X, Y) == -1
        assert b"EVSL_NOALLOC_MAX_ELEMS" in lib.evsl_last_error(ctx.h)
