"""GPU parity of the generalized path A x = lambda B x (B^{-1} by the lsPol polynomial): the
polynomial solve, the pencil's Lanczos bounds and the filtered non-restart Lanczos against the
FP64 oracle and against the closed form of the pencil (laplacian_2d(nx), mass_matrix_2d(nx)).

n = 400 and 1369 span 13 and 43 slices of 32 rows with a ragged last slice.  Tolerances:
p(B) x within 1e-12 sum_j |c_j| ||x||_inf of the oracle (the same recurrence rounded in another
order) and B p(B) x = x to 1e-12; converged bounds within 1e-8 lambda_max; eigenpairs with the exact
count, eigenvalues within 1e-9 relative, ||A x - lambda B x|| <= 1e-8 bmax lmax and
||X^T B X - I|| <= 1e-10.
"""
import numpy as np
import pytest

from closed_form import pencil_eigs
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


@pytest.fixture(scope="module")
def ctx(nat):
    c = nat.Context(0)
    yield c
    c.close()


def _pencil(ctx, oracle_mod, nx):
    A, B = I.laplacian_2d(nx), I.mass_matrix_2d(nx)
    blo, bhi = oracle_mod.bounds(B, 80, 0)
    lp = oracle_mod.lspol(blo, bhi, 1e-13)
    ctx.set_csr(A)
    deg, err = ctx.set_csr_b(B, blo, bhi, 1e-13)
    assert deg == lp["deg"] and err <= 1e-13
    return A, B, lp


@pytest.mark.parametrize("nx", [20, 37])
def test_polyB_apply_matches_oracle(ctx, oracle_mod, nx):
    import torch
    A, B, lp = _pencil(ctx, oracle_mod, nx)
    x = np.random.default_rng(nx).standard_normal(B.n)
    xd = torch.tensor(x, device="cuda")
    yd = torch.empty_like(xd)
    ctx.polyB_apply(xd, yd)
    y = yd.cpu().numpy()
    yo = oracle_mod.poly_solve(B, lp, x)
    assert np.max(np.abs(y - yo)) <= 1e-12 * np.abs(lp["coef"]).sum() * np.abs(x).max()
    assert np.linalg.norm(B.to_dense() @ y - x) <= 1e-12 * np.linalg.norm(x)


def test_bounds_gen_matches_oracle_and_encloses(ctx, oracle_mod):
    # 200 steps converge both ends, so both bounds agree with the oracle's to rounding; after 80
    # steps the lowest Ritz value is still moving (its bound shifts by ~1e-6 under a change of
    # rounding order), so there only the converged upper end is compared and the lower one must
    # enclose the spectrum.  The upper bound may sit ~1e-13 relative below lambda_max: p(B) is
    # B^{-1} to 1e-13.
    A, B, lp = _pencil(ctx, oracle_mod, 20)
    lam = pencil_eigs(20)
    lo, hi = ctx.bounds_gen(200, 0)
    olo, ohi = oracle_mod.bounds_gen(A, B, lp, 200, 0)
    assert abs(lo - olo) <= 1e-8 * lam[-1] and abs(hi - ohi) <= 1e-8 * lam[-1]
    lo, hi = ctx.bounds_gen(80, 0)
    olo, ohi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    assert abs(hi - ohi) <= 1e-8 * lam[-1]
    assert lo <= lam[0] and hi >= lam[-1] - 1e-9 * lam[-1]


@pytest.mark.parametrize("a,b", [(2.0, 3.0), (10.0, 11.0), (40.0, 42.0)])
def test_cheblannr_gen_matches_closed_form_and_oracle(ctx, nat, oracle_mod, a, b):
    nx = 20
    A, B, lp = _pencil(ctx, oracle_mod, nx)
    lam = pencil_eigs(nx)
    lo, hi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    f = nat.cheb_filter_build(a, b, lo, hi)
    ex = lam[(lam >= a) & (lam <= b)]
    m = max(6 * len(ex), 200)
    r = ctx.chebLanNr_gen(a, b, f, m=m)
    assert r["status"] == 0 and r["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1.0, ex))
    X, Ad, Bd = r["Y"][:r["nev"]].T, A.to_dense(), B.to_dense()
    R = Ad @ X - (Bd @ X) * r["lam"]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-8 * lp["bmax"] * hi
    assert np.max(np.abs(X.T @ Bd @ X - np.eye(r["nev"]))) <= 1e-10
    assert r["stats"]["nmv"] == f.deg * r["stats"]["niter"]
    ro = oracle_mod.cheblannr_gen(A, B, lp, a, b, oracle_mod.filter_build(a, b, lo, hi), m=m)
    assert ro["status"] == 0 and ro["nev"] == r["nev"]
    assert abs(ro["niter"] - r["stats"]["niter"]) <= 10
    assert np.all(np.abs(ro["lam"] - r["lam"]) <= 1e-9 * np.maximum(1.0, ex))


def test_generalized_state_errors(nat, oracle_mod):
    # no B, B of another order, and an lsPol degree limit are reported, not computed around
    c = nat.Context(0)
    try:
        A = I.laplacian_2d(12)
        c.set_csr(A)
        f = nat.cheb_filter_build(2.0, 3.0, 0.0, 80.0)
        with pytest.raises(nat.EvslError):
            c.chebLanNr_gen(2.0, 3.0, f, m=50)
        c.set_csr_b(I.mass_matrix_2d(11), 0.1, 1.0)
        with pytest.raises(nat.EvslError):
            c.bounds_gen(20, 0)
        with pytest.raises(nat.EvslError):
            c.set_csr_b(I.mass_matrix_2d(12), 0.1, 1.0, maxdeg=4)
        c.set_csr_b(I.mass_matrix_2d(12), 0.1, 1.0)
        lo, hi = c.bounds_gen(40, 0)
        assert lo < pencil_eigs(12)[0] + 1e-9 and hi > 0.9 * pencil_eigs(12)[-1]
    finally:
        c.close()


def test_cheblannr_gen_graph_replay_bitwise_equals_direct(ctx, nat, oracle_mod):
    # the filter's CUDA graph (captured once, replayed every step) and direct launches run the
    # same kernels with the same arguments: identical eigenpairs; the profiler sees
    # deg (deg(p) + 1) generalized steps per Lanczos step either way
    A, B, lp = _pencil(ctx, oracle_mod, 20)
    lo, hi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    f = nat.cheb_filter_build(10.0, 11.0, lo, hi)
    out = []
    for graphs in (True, False):
        ctx.set_graphs(graphs)
        ctx.profile(True)
        r = ctx.chebLanNr_gen(10.0, 11.0, f, m=200)
        nl, ms = ctx.profile_get(nat.K_GEN_STEP)
        ctx.profile(False)
        assert nl == f.deg * (lp["deg"] + 1) * r["stats"]["niter"] and ms > 0
        out.append(r)
    ctx.set_graphs(True)
    assert out[0]["nev"] == out[1]["nev"] > 0
    assert np.array_equal(out[0]["lam"], out[1]["lam"]) and np.array_equal(out[0]["res"], out[1]["res"])
    assert np.array_equal(out[0]["Y"][:out[0]["nev"]], out[1]["Y"][:out[1]["nev"]])


def test_kpm_gen_matches_oracle_and_slices(ctx, nat, oracle_mod):
    # the pencil's KPM moments against the oracle's (same probes, p and q from the same interval),
    # mu_0 = n, and the DOS slicer on them gives the oracle's slices
    A, B, lp = _pencil(ctx, oracle_mod, 20)
    lq = oracle_mod.lspol_isqrt(lp["bmin"], lp["bmax"], 1e-13)
    lo, hi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    for M, nv, seed in [(50, 7, 0), (1, 1, 3), (0, 2, 1)]:
        mu = ctx.kpm_dos_gen(M, nv, seed, lo, hi)
        mo = oracle_mod.kpm_moments_gen(A, B, lp, lq, M, nv, seed, lo, hi)
        assert abs(mu[0] - A.n) <= 1e-12 * A.n
        assert np.max(np.abs(mu - mo)) <= 1e-11 * A.n
    mu = ctx.kpm_dos_gen(60, 10, 0, lo, hi)
    mo = oracle_mod.kpm_moments_gen(A, B, lp, lq, 60, 10, 0, lo, hi)
    s, e = nat.slice_by_dos(mu, A.n, lo, hi, 1.0, 60.0, 5, 0)
    so, eo = oracle_mod.slicer(mo, lo, hi, 1.0, 60.0, 5, None)
    assert np.max(np.abs(s - so)) <= 1e-8 * (hi - lo) and np.max(np.abs(e - eo)) <= 1e-6 * A.n


def test_kpm_gen_scaled_identity_equals_standard_kpm(ctx, nat, oracle_mod):
    # B = 2I: the pencil's moments on [lmin/2, lmax/2] are the standard moments on [lmin, lmax]
    A = I.anderson_3d(9, 3.0, 1)
    n = A.n
    B2 = I.CSR(n, np.arange(n + 1), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    ctx.set_csr(A)
    ctx.set_csr_b(B2, 1.5, 2.5, 1e-13)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    mg = ctx.kpm_dos_gen(40, 3, 7, lo / 2, hi / 2)
    ms = ctx.kpm_dos(40, 3, 7, lo, hi)
    assert np.max(np.abs(mg - ms)) <= 1e-12 * n


@pytest.mark.parametrize("a,b,m", [(2.0, 3.0, 40), (10.0, 11.0, 40), (40.0, 42.0, 30)])
def test_cheblantr_gen_restarts_match_closed_form_and_oracle(ctx, nat, oracle_mod, a, b, m):
    # thick restart with locking for the pencil, with bases small enough to need several
    # cycles: exact count and eigenvalues, residuals, B-orthonormality; the oracle's run finds the
    # same eigenvalues
    nx = 20
    A, B, lp = _pencil(ctx, oracle_mod, nx)
    lam = pencil_eigs(nx)
    lo, hi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    f = nat.cheb_filter_build(a, b, lo, hi)
    ex = lam[(lam >= a) & (lam <= b)]
    r = ctx.chebLanTr_gen(a, b, f, m=m)
    assert r["status"] == 0 and r["nev"] == len(ex) and r["stats"]["nrestart"] >= 3
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1.0, ex))
    X, Ad, Bd = r["Y"][:r["nev"]].T, A.to_dense(), B.to_dense()
    assert np.max(np.linalg.norm(Ad @ X - (Bd @ X) * r["lam"], axis=0)) <= 1e-8 * lp["bmax"] * hi
    assert np.max(np.abs(X.T @ Bd @ X - np.eye(r["nev"]))) <= 1e-10
    assert r["stats"]["nmv"] == f.deg * r["stats"]["niter"]
    ro = oracle_mod.cheblantr_gen(A, B, lp, a, b, oracle_mod.filter_build(a, b, lo, hi), m=m)
    assert ro["status"] == 0 and ro["nev"] == r["nev"]
    assert np.all(np.abs(ro["lam"] - r["lam"]) <= 1e-9 * np.maximum(1.0, ex))


def test_cheblantr_gen_noncommuting_pencil_matches_dense_eigensolver(ctx, nat, oracle_mod):
    # Anderson A with B = 0.4 I + 0.05 L (3-D Laplacian): B's eigenvectors are not A's; the
    # eigenvalues in two slices against scipy's dense generalized eigensolver
    import scipy.linalg as sl
    nx = 7
    A = I.anderson_3d(nx, 3.0, 0)
    n = A.n
    Bd = 0.4 * np.eye(n) + 0.05 * I.laplacian_3d(nx).to_dense()
    rows, cols = np.nonzero(Bd)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    B = I.CSR(n, rp, cols.astype(np.int32), Bd[rows, cols])
    w = sl.eigh(A.to_dense(), Bd, eigvals_only=True)
    ctx.set_csr(A)
    ctx.set_csr_b(B, 0.39, 1.01, 1e-13)
    lo, hi = ctx.bounds_gen(80, 0)
    # converged bounds match the extreme eigenvalues up to p(B)'s 1e-13 accuracy
    assert lo <= w[0] + 1e-12 * abs(w[-1]) and hi >= w[-1] - 1e-9 * abs(w[-1])
    for a, b in [(2.0, 4.0), (8.0, 9.0)]:
        ex = w[(w >= a) & (w <= b)]
        f = nat.cheb_filter_build(a, b, lo, hi)
        r = ctx.chebLanTr_gen(a, b, f, m=max(2 * len(ex), 40))
        assert r["status"] == 0 and r["nev"] == len(ex)
        assert np.max(np.abs(r["lam"] - ex)) <= 1e-9 * max(1.0, np.abs(ex).max())
        X = r["Y"][:r["nev"]].T
        assert np.max(np.abs(X.T @ Bd @ X - np.eye(r["nev"]))) <= 1e-10


def test_landos_gen_matches_oracle_and_slices(nat, oracle_mod):
    # the pencil's Lanczos quadrature density against the oracle's (same start vectors, p and q
    # from the same interval), and the quadrature slicer on it gives the oracle's slices
    A, B = I.laplacian_2d(20), I.mass_matrix_2d(20)
    blo, bhi = oracle_mod.bounds(B, 80, 0)
    lp, lq = oracle_mod.lspol(blo, bhi, 1e-13), oracle_mod.lspol_isqrt(blo, bhi, 1e-13)
    with nat.Context(0) as ctx:
        ctx.set_csr(A)
        ctx.set_csr_b(B, blo, bhi, 1e-13)
        d = ctx.landos_gen(30, 6, 2)
    do = oracle_mod.landos_gen(A, B, lp, lq, 30, 6, 2)
    assert np.array_equal(d["mused"], do["mused"])
    lam = pencil_eigs(20)
    assert np.max(np.abs(d["nodes"] - do["nodes"])) <= 1e-9 * lam[-1]
    assert np.max(np.abs(d["weights"] - do["weights"])) <= 1e-9
    s, e = nat.slice_by_landos(d, A.n, 10.0, 60.0, 4)
    so, eo = oracle_mod.slicer_landos(do, A.n, 10.0, 60.0, 4)
    assert np.allclose(s, so, atol=1e-9 * lam[-1])
