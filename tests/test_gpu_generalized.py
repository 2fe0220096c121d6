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
