"""Small fixed workloads for profiling single kernels with ncu (a few launches, < 1 GB).

    python -m paper_1802_05215_gb300.profile_cases cheb      # filter step: FP64 then FP32
    python -m paper_1802_05215_gb300.profile_cases steptime  # live per-launch time of the filter step
    python -m paper_1802_05215_gb300.profile_cases gemv      # Gram-Schmidt GEMV-T / GEMV-N
    python -m paper_1802_05215_gb300.profile_cases kpm       # KPM moment step, FP64 then FP32
    python -m paper_1802_05215_gb300.profile_cases multi     # 16-slice batched filter step, FP32
    python -m paper_1802_05215_gb300.profile_cases gen       # generalized step: solves with p(B)
    python -m paper_1802_05215_gb300.profile_cases gemm      # tensor-core FP64 GEMM, Ritz shape
    python -m paper_1802_05215_gb300.profile_cases kpm160    # FP32 KPM step, Anderson 160^3, 64 probes

Each case but `gen`, `gemm` and `kpm160` runs on the 100^3 7-point Laplacian (n = 1e6, nnz = 6.94e6); `gen` uses the
1000^2 linear-element mass matrix (n = 1e6, nnz = 8.99e6).  Each prints the number of kernels
the library launched.
"""
from __future__ import annotations

import sys


def _ctx():
    from . import inputs, native
    A = inputs.laplacian_3d(100)
    ctx = native.Context(0)
    ctx.set_csr(A)
    return native, A, ctx


def cheb():
    """Six-degree filter on one vector: 6 launches of the fused step in FP64, then 6 in FP32."""
    import torch
    native, A, ctx = _ctx()
    f = native.cheb_filter_build(0.40, 0.428, 0.0, 12.0)
    f.pol.deg = 6
    X = torch.randn(1, A.n, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    ctx.filter_apply(f, X, Y, prec=native.FP64)
    ctx.filter_apply(f, X, Y, prec=native.FP32)
    torch.cuda.synchronize()
    return ctx


def steptime():
    """Live per-launch time of the fused filter step, FP64 then FP32: ten applications of the
    degree-217 filter of [0.349, 0.391] (one slice of the 100^3 benchmark) after two warm-up ones,
    timed by the library's CUDA events on its own stream; prints time, algorithmic GB/s and the
    fraction of the measured copy peak."""
    import json
    import os
    import torch
    native, A, ctx = _ctx()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    try:
        peak = json.load(open(os.path.join(root, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, KeyError, ValueError):
        peak = 6800.0
    lo, hi = ctx.bounds(80, 0)
    f = native.cheb_filter_build(0.34906336788172704, 0.39063876503853284, lo, hi)
    X = torch.randn(1, A.n, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    for prec, b in [(native.FP64, 8), (native.FP32, 4)]:
        for _ in range(2):
            ctx.filter_apply(f, X, Y, prec=prec)
        ctx.profile(True)
        for _ in range(10):
            ctx.filter_apply(f, X, Y, prec=prec)
        nl, ms = ctx.profile_get(native.K_CHEB_STEP)
        ctx.profile(False)
        alg = A.nnz * (b + 4) + 8 * (A.n + 1) + 5 * A.n * b
        us = ms / nl * 1e3
        print(f"steptime {'fp64' if b == 8 else 'fp32'}: degree {f.deg}, {nl} launches, {us:.3f} us per launch = "
              f"{alg / us / 1e3:.1f} GB/s algorithmic = {alg / us / 1e3 / peak:.4f} of {peak} GB/s", flush=True)
    return ctx


def gemv():
    """400 bounds-Lanczos steps: the last projections run against ~400 basis columns (3.2 GB)."""
    native, A, ctx = _ctx()
    ctx.bounds(400, 0)
    return ctx


def kpm():
    """KPM degree 4 with 40 probes, FP64 then FP32."""
    native, A, ctx = _ctx()
    ctx.kpm_dos(4, 40, 0, 0.0, 12.0, prec=native.FP64)
    ctx.kpm_dos(4, 40, 0, 0.0, 12.0, prec=native.FP32)
    return ctx


def multi():
    """16 slice filters of [0.2, 0.6] batched (one block launch per degree), FP32."""
    import numpy as np
    import torch
    native, A, ctx = _ctx()
    cuts = np.linspace(0.2, 0.6, 17)
    fs = [native.cheb_filter_build(cuts[i], cuts[i + 1], 0.0, 12.0) for i in range(16)]
    for f in fs:
        f.pol.deg = min(f.pol.deg, 6)
    X = torch.randn(16, A.n, dtype=torch.float64, device="cuda")
    Y = torch.empty_like(X)
    ctx.filter_apply_multi(fs, X, Y, prec=native.FP32)
    torch.cuda.synchronize()
    return ctx


def gen():
    """Two solves y = p(B) x with the lsPol polynomial on [0.11, 1] (which holds the spectrum of
    the 1000^2 mass matrix M (x) M, M = tridiag(1, 4, 1)/6): 2 x deg(p) launches of k_gen_step,
    each solve one MODE 0 launch and then MODE 1 launches."""
    import torch
    from . import inputs, native
    B = inputs.mass_matrix_2d(1000)
    ctx = native.Context(0)
    deg, _ = ctx.set_csr_b(B, 0.11, 1.0, 1e-13)
    x = torch.randn(B.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    ctx.polyB_apply(x, y)
    ctx.polyB_apply(x, y)
    torch.cuda.synchronize()
    print(f"gen: p(B) degree {deg}")
    return ctx


def kpm160():
    """KPM degree 4 with 64 probes in FP32 on the Anderson model 160^3 (W = 2, n = 4.1e6): the
    probe-block shape of the 200^3 benchmark (every lane of a row active) at about 3 GB."""
    from . import inputs, native
    A = inputs.anderson_3d(160, 2.0, 0)
    ctx = native.Context(0)
    ctx.set_csr(A)
    lo, hi = ctx.bounds(40, 0)
    ctx.kpm_dos(4, 64, 0, lo, hi, prec=native.FP32)
    return ctx


def gemm():
    """The restart's Ritz-vector product Y = Q S in the shape of a 100^3 slice scaled to
    n = 100,000 rows (k = 1320 basis vectors, l = 720 candidates): one untimed and three timed
    products on the tensor cores (digit splitting included), then three with the FP64 kernel;
    prints the FP64-equivalent rate 2 n k l / time of each."""
    import torch
    from . import native
    n, k, l = 100_000, 1320, 720
    g = torch.Generator(device="cuda").manual_seed(0)
    Q = torch.randn(k, n, dtype=torch.float64, device="cuda", generator=g) / n ** 0.5
    S = torch.randn(l, k, dtype=torch.float64, device="cuda", generator=g) / k ** 0.5
    Y = torch.empty(l, n, dtype=torch.float64, device="cuda")
    ctx = native.Context(0)
    for tc in (True, False):
        ctx.set_tensor_gemm(tc)
        ctx.dense_gemm(Q, S, Y)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(3):
            ctx.dense_gemm(Q, S, Y)
        e1.record()
        torch.cuda.synchronize()
        s = e0.elapsed_time(e1) * 1e-3 / 3
        print(f"gemm {'tensor-core' if tc else 'fp64 kernel'}: n={n} k={k} l={l}: {s * 1e3:.2f} ms = "
              f"{2 * n * k * l / s / 1e12:.2f} TFLOP/s (FP64-equivalent)")
    return ctx


CASES = {"cheb": cheb, "steptime": steptime, "gemv": gemv, "kpm": kpm, "multi": multi, "gen": gen, "gemm": gemm, "kpm160": kpm160}

if __name__ == "__main__":
    name = sys.argv[1] if len(sys.argv) > 1 else "cheb"
    ctx = CASES[name]()
    if ctx is not None:
        print(f"{name}: ok, launches={ctx.launch_count()}")
