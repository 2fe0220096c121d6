"""The FP64-accurate tensor-core GEMM (evsl_dense_gemm: Ozaki digit splitting on tcgen05).

References are exact: each checked entry is the correctly rounded value of sum_k a_ik b_kj,
obtained from Dekker's error-free products and math.fsum, independent of any GPU code.  The
bound is 2^-51 sum_k |a_ik| |b_kj|, which FP64 summation itself only meets for short sums; the
tensor-core result is also compared with the plain FP64 kernel of the library (it must be at
least as accurate on every sampled entry, up to one unit of the bound's rounding).
"""
import math

import numpy as np
import pytest

from closed_form import lap_eigs
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


def _two_prod(a, b):
    """Dekker's error-free product: a * b = p + e exactly (no overflow)."""
    def split(x):
        c = 134217729.0 * x
        hi = c - (c - x)
        return hi, x - hi
    p = a * b
    ah, al = split(a)
    bh, bl = split(b)
    e = al * bl - (((p - ah * bh) - al * bh) - ah * bl)
    return p, e


def _exact(a, b):
    p, e = _two_prod(a, b)
    return math.fsum(np.concatenate([p, e])), float(np.sum(np.abs(a * b)))


def _check(Am, Bm, C, trans_a, rows, cols):
    """Max over sampled (i, j) of |C_ij - exact| / sum|a||b| (Am, Bm as numpy column-major
    arrays given row-major as (cols, rows))."""
    worst = 0.0
    for i, j in zip(rows, cols):
        a = Am[i] if trans_a else Am[:, i]
        ex, bound = _exact(a, Bm[j])
        if bound:
            worst = max(worst, abs(C[j, i] - ex) / bound)
    return worst


@pytest.mark.parametrize("trans_a,M,N,K", [(False, 300, 61, 1000), (False, 129, 48, 31), (True, 97, 130, 2000),
                                           (False, 1000, 17, 448), (True, 256, 96, 449)])
def test_dense_gemm_matches_exact_dot_products(nat, trans_a, M, N, K):
    # ragged M (not a multiple of 128), N (not of 48), K (not of 32), K across several
    # 448-long exact chunks; rows of A with exponents spread over 2^+-40
    import torch
    rng = np.random.default_rng(M + N + K)
    if trans_a:
        A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-40, 40, (M, 1)))   # M columns of length K
    else:
        A = rng.standard_normal((K, M)) * np.exp2(rng.integers(-40, 40, (1, M)))   # K columns of length M
    B = rng.standard_normal((N, K)) * np.exp(rng.uniform(-3, 3, (N, K)))
    At, Bt = torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda")
    with nat.Context(0) as ctx:
        Ct = torch.full((N, M), np.nan, dtype=torch.float64, device="cuda")
        ctx.dense_gemm(At, Bt, Ct, trans_a=trans_a)
        C = Ct.cpu().numpy()
        ctx.set_tensor_gemm(False)
        Cf = torch.full((N, M), np.nan, dtype=torch.float64, device="cuda")
        ctx.dense_gemm(At, Bt, Cf, trans_a=trans_a)
        C64 = Cf.cpu().numpy()
    assert np.all(np.isfinite(C))
    samp = rng.integers(0, M, 200), rng.integers(0, N, 200)
    err_tc = _check(A, B, C, trans_a, *samp)
    err_64 = _check(A, B, C64, trans_a, *samp)
    assert err_tc <= 2.0 ** -51, err_tc
    assert err_tc <= err_64 + 2.0 ** -60, (err_tc, err_64)


@pytest.mark.parametrize("signs", ["positive", "random"])
def test_dense_gemm_chunk_sums_at_the_exactness_bound(nat, signs):
    # every element has all nine digits (nearly) at their maximum; with positive signs each
    # diagonal's FP32 sums reach 9 * 63^2 * 448 ~ 1.6e7 (just below 2^24) in every chunk, so
    # the result equals the exact product only if the accumulation of integer products is
    # exact; random signs add cancellation
    import torch
    rng = np.random.default_rng(3)
    M, N, K = 256, 96, 1344
    top = 2.0 - 2.0 ** -52
    pick = (lambda shape: np.ones(shape)) if signs == "positive" else (lambda shape: rng.choice([-1.0, 1.0], shape))
    A = top * pick((K, M))
    B = top * pick((N, K))
    with nat.Context(0) as ctx:
        Ct = torch.empty((N, M), dtype=torch.float64, device="cuda")
        ctx.dense_gemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), Ct)
        C = Ct.cpu().numpy()
    # exact: (sum of signs) * top^2, a multiple of top^2 with |sum| <= K
    ssum = (np.sign(A).T @ np.sign(B).T)             # M x N integers, exact in FP64
    exact = ssum * top * top
    rel = np.abs(C - exact.T) / (K * top * top)
    assert rel.max() <= 2.0 ** -52, rel.max()


@pytest.mark.parametrize("mode", [1, 2])
def test_dense_gemm_subtract_and_add_modes(nat, mode):
    import torch
    rng = np.random.default_rng(mode)
    M, N, K = 200, 50, 600
    A = torch.tensor(rng.standard_normal((K, M)), device="cuda")
    B = torch.tensor(rng.standard_normal((N, K)), device="cuda")
    C0 = torch.tensor(rng.standard_normal((N, M)), device="cuda")
    with nat.Context(0) as ctx:
        P = torch.empty_like(C0)
        ctx.dense_gemm(A, B, P)
        C = C0.clone()
        ctx.dense_gemm(A, B, C, mode=mode)
    want = C0 - P if mode == 1 else C0 + P
    assert torch.allclose(C, want, rtol=0, atol=1e-13 * float(P.abs().max()))


def test_dense_gemm_tall_ritz_shape_and_transposed_panels(nat):
    # the Ritz-vector shape (a tall basis times a small block; K spans three chunks and the rows
    # two panels of the 2 GiB digit workspace) and a transposed product whose contraction is
    # split into two panels
    import torch
    rng = np.random.default_rng(11)
    n, k, l = 200_000, 1000, 72
    Q = torch.tensor(rng.standard_normal((k, n)) / np.sqrt(n), device="cuda")
    S = torch.tensor(rng.standard_normal((l, k)) / np.sqrt(k), device="cuda")
    with nat.Context(0) as ctx:
        Y = torch.empty((l, n), dtype=torch.float64, device="cuda")
        ctx.dense_gemm(Q, S, Y)
        samp = rng.integers(0, n, 100), rng.integers(0, l, 100)
        err = _check(Q.cpu().numpy(), S.cpu().numpy(), Y.cpu().numpy(), False, *samp)
        assert err <= 2.0 ** -51, err
        p, q, K = 1500, 1500, 50_000                   # (p + q) * 9 * 2 * K > 2 GiB
        W = torch.tensor(rng.standard_normal((p, K)), device="cuda")
        Z = torch.tensor(rng.standard_normal((q, K)), device="cuda")
        G = torch.empty((q, p), dtype=torch.float64, device="cuda")
        ctx.dense_gemm(W, Z, G, trans_a=True)
        samp = rng.integers(0, p, 40), rng.integers(0, q, 40)
        err = _check(W.cpu().numpy(), Z.cpu().numpy(), G.cpu().numpy(), True, *samp)
        assert err <= 2.0 ** -51, err


def test_solver_results_agree_with_and_without_tensor_core_gemm(nat):
    # a slice large enough that the restart's Ritz-vector product runs on the tensor cores
    # (2 n k l >= 1e9): the same count and eigenvalues as with the FP64 kernel, and both equal
    # the closed form
    A = I.laplacian_3d(30)
    e = lap_eigs(3, 30)
    a, b = 1.0, 1.25
    ex = e[(e >= a) & (e <= b)]
    assert len(ex) > 150
    out = []
    for tc in (True, False):
        with nat.Context(0) as ctx:
            ctx.set_tensor_gemm(tc)
            ctx.set_csr(A)
            lo, hi = ctx.bounds(80, 0)
            f = nat.cheb_filter_build(a, b, lo, hi)
            m = 2 * len(ex) + 40
            assert 2.0 * A.n * len(ex) * m >= 1e9
            out.append(ctx.chebLanTr(a, b, f, m=m))
    for r in out:
        assert r["status"] == 0 and r["nev"] == len(ex)
        assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.abs(ex))
        assert r["res"].max() <= 1e-8
    assert np.max(np.abs(out[0]["lam"] - out[1]["lam"])) <= 1e-11


def test_dense_gemm_largest_polish_shapes_3300(nat):
    # the largest products the FP32-filter polish forms: a Gram projection C = W^T Z of two
    # n x 3300 blocks (3300 x 3300 result, contraction split into panels) and a Ritz-vector product
    # Y = Q S with Q of n x 3300 and S of 3300 x 3300 (rows split into panels).  Sampled entries
    # against exact dot products; the whole result against cuBLAS DGEMM,
    # ||C - C_dgemm||_F <= 1e-15 ||W||_F ||Z||_F.  The operands are made by torch kernels that may
    # still be running on torch's stream when the call is made: the binding orders them
    import torch
    rng = np.random.default_rng(17)
    g = torch.Generator(device="cuda").manual_seed(17)
    n, k = 40_000, 3300

    def block(rows, cols, spread):
        X = torch.randn((cols, rows), generator=g, dtype=torch.float64, device="cuda")
        return X * torch.exp2(torch.randint(-spread, spread + 1, (cols, 1), generator=g, device="cuda").double())

    with nat.Context(0) as ctx:
        W, Z = block(n, k, 20), block(n, k, 20)           # 3300 columns of length n each
        C = torch.empty((k, k), dtype=torch.float64, device="cuda")
        ctx.dense_gemm(W, Z, C, trans_a=True)
        ref = Z @ W.T
        assert torch.linalg.norm(C - ref) <= 1e-15 * torch.linalg.norm(W) * torch.linalg.norm(Z)
        i, j = rng.integers(0, k, 60), rng.integers(0, k, 60)
        Wi, Zj = W[torch.tensor(i)].cpu().numpy(), Z[torch.tensor(j)].cpu().numpy()
        Cij = C[torch.tensor(j), torch.tensor(i)].cpu().numpy()
        worst = max(abs(Cij[t] - _exact(Wi[t], Zj[t])[0]) / _exact(Wi[t], Zj[t])[1] for t in range(60))
        assert worst <= 2.0 ** -51, worst
        del W, Z, C, ref

        Q = block(n, k, 0) / np.sqrt(n)                     # k columns of length n
        S = block(k, k, 0) / np.sqrt(k)                     # k columns of length k
        Y = torch.empty((k, n), dtype=torch.float64, device="cuda")
        ctx.dense_gemm(Q, S, Y)
        ref = S @ Q
        assert torch.linalg.norm(Y - ref) <= 1e-15 * torch.linalg.norm(Q) * torch.linalg.norm(S)
        r, c = rng.integers(0, n, 60), rng.integers(0, k, 60)
        Qr, Sc = Q[:, torch.tensor(r)].cpu().numpy(), S[torch.tensor(c)].cpu().numpy()
        Yrc = Y[torch.tensor(c), torch.tensor(r)].cpu().numpy()
        worst = max(abs(Yrc[t] - _exact(Qr[:, t], Sc[t])[0]) / _exact(Qr[:, t], Sc[t])[1] for t in range(60))
        assert worst <= 2.0 ** -51, worst
