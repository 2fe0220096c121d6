"""GPU parity: the sm_103a kernels behind the C ABI against the FP64 CPU oracle.

Sizes are chosen so that the oracle finishes in seconds while the GPU path spans many
32-row slices and reduction chunks with a ragged tail (n not a multiple of 32).
Tolerances: KPM moments |mu_gpu - mu_oracle| <= 1e-12 n (FP64) / 1e-5 n (FP32), n being the
largest any moment can be (|v^T T_k(Ahat) v| <= ||v||^2 = n); filter outputs relative to
sum_j |c_j| ||x||_inf; eigenpairs: exact count, eigenvalues within 1e-9 relative, residual
||Ax - lambda x|| / ||A|| <= 1e-8, ||Y^T Y - I|| <= 1e-10, eigenspaces by projectors.
"""
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


@pytest.fixture(scope="module")
def ctx(nat):
    c = nat.Context(0)
    yield c
    c.close()


def _dense_residuals(A, lam, Y):
    D = A.to_dense()
    normA = np.abs(np.linalg.eigvalsh(D)).max()
    return np.linalg.norm(D @ Y - Y * lam, axis=0) / normA


# ------------------------------------------------------------------------------ KPM
@pytest.mark.parametrize("mat", ["lap2d_45", "anderson_13", "lap3d_9"])
def test_kpm_fp64_matches_oracle(ctx, oracle_mod, mat):
    A = {"lap2d_45": lambda: I.laplacian_2d(45), "anderson_13": lambda: I.anderson_3d(13, 4.0, 1),
         "lap3d_9": lambda: I.laplacian_3d(9)}[mat]()
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 60, 0)
    for M, nv, seed in [(50, 7, 0), (1, 1, 5), (0, 3, 2)]:
        mu = ctx.kpm_dos(M, nv, seed, lo, hi)
        mo = oracle_mod.kpm_moments(A, M, nv, seed, lo, hi)
        assert mu[0] == A.n
        assert np.max(np.abs(mu - mo)) <= 1e-12 * A.n


def test_kpm_fp32_matches_oracle(ctx, nat, oracle_mod):
    A = I.anderson_3d(14, 4.0, 0)
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 60, 0)
    mu = ctx.kpm_dos(80, 9, 1, lo, hi, prec=nat.FP32)
    mo = oracle_mod.kpm_moments(A, 80, 9, 1, lo, hi)
    assert np.max(np.abs(mu - mo)) <= 1e-5 * A.n



@pytest.mark.parametrize("prec,tol", [(0, 1e-11), (1, 2e-5)])
def test_kpm_doubling_matches_oracle(ctx, nat, oracle_mod, prec, tol):
    # the doubled moments (half the recurrence steps) against the oracle's doubled and direct
    # moments, same probes; odd and even degrees
    A = I.anderson_3d(12, 4.0, 0)
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    for M in (31, 40):
        mu = ctx.kpm_dos(M, 9, 3, lo, hi, prec=prec, doubling=True)
        ref = oracle_mod.kpm_moments_doubling(A, M, 9, 3, lo, hi)
        direct = oracle_mod.kpm_moments(A, M, 9, 3, lo, hi)
        assert mu[0] == A.n
        assert np.max(np.abs(mu - ref)) <= tol * A.n
        assert np.max(np.abs(mu - direct)) <= tol * A.n

def test_kpm_is_deterministic(ctx):
    A = I.laplacian_3d(20)
    ctx.set_csr(A)
    m1 = ctx.kpm_dos(40, 5, 9, 0.0, 12.0)
    m2 = ctx.kpm_dos(40, 5, 9, 0.0, 12.0)
    assert np.array_equal(m1, m2)


def test_kpm_config_2d_100(ctx, oracle_mod):
    # 100 x 100 Laplacian, degree 80, 20 probes, seed 0
    A = I.laplacian_2d(100)
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    mu = ctx.kpm_dos(80, 20, 0, lo, hi)
    mo = oracle_mod.kpm_moments(A, 80, 20, 0, lo, hi)
    assert np.max(np.abs(mu - mo)) <= 1e-12 * A.n


def test_kpm_full_size_3d_100(ctx, nat, oracle_mod):
    # n = 1e6, degree 120: 40 probes on the GPU; probes are independent of nvec, so the first
    # two are checked against the oracle one by one, and the full set against the closed-form
    # trace statistics and the FP32 run.
    A = I.laplacian_3d(100)
    ctx.set_csr(A)
    lo, hi = 0.0, 12.0
    mu40 = ctx.kpm_dos(120, 40, 0, lo, hi)
    mu2 = ctx.kpm_dos(120, 2, 0, lo, hi)
    mo2 = oracle_mod.kpm_moments(A, 120, 2, 0, lo, hi)
    assert np.max(np.abs(mu2 - mo2)) <= 1e-12 * A.n
    assert mu40[0] == A.n
    e = lap_eigs(3, 100)
    lh = (e - 6.0) / 6.0
    for k in range(0, 121, 10):
        tk = np.cos(k * np.arccos(np.clip(lh, -1, 1)))
        sig = np.sqrt(2.0 * np.sum(tk * tk) / 40)
        assert abs(mu40[k] - tk.sum()) <= 6 * sig + 1e-6
    m32 = ctx.kpm_dos(120, 40, 0, lo, hi, prec=nat.FP32)
    assert np.max(np.abs(m32 - mu40)) <= 1e-5 * A.n


# ------------------------------------------------------------------------------ filter
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_filter_apply_matches_oracle(ctx, nat, oracle_mod, prec, tol):
    import torch
    A = I.laplacian_2d(45)
    ctx.set_csr(A)
    lo, hi = 0.0, 8.0
    f = nat.cheb_filter_build(1.0, 1.2, lo, hi)
    assert f.deg > 20
    X = np.random.default_rng(0).standard_normal((3, A.n))
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.empty_like(Xd)
    ctx.filter_apply(f, Xd, Yd, prec=prec)
    Y = Yd.cpu().numpy()
    Yo = oracle_mod.filter_apply(A, lo, hi, f.coef, X.T.copy()).T
    scale = np.abs(f.coef).sum() * np.abs(X).max()
    assert np.max(np.abs(Y - Yo)) <= tol * scale


def test_filter_apply_degree_edge_cases(ctx, nat, oracle_mod):
    import torch
    A = I.anderson_3d(7, 4.0, 0)          # n = 343: 10 full slices + a ragged one
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 60, 0)
    X = np.random.default_rng(1).standard_normal((1, A.n))
    Xd = torch.tensor(X, device="cuda")
    for coef in [np.array([0.7]), np.array([0.1, -0.4]), np.array([0.2, 0.3, -0.5])]:
        f = nat.cheb_filter_build(5.0, 6.0, lo, hi)
        f.coef = coef.copy()
        f.pol.deg = len(coef) - 1
        f.pol.coef = f.coef.ctypes.data_as(nat.C.POINTER(nat.C.c_double))
        Yd = torch.empty_like(Xd)
        ctx.filter_apply(f, Xd, Yd)
        Yo = oracle_mod.filter_apply(A, lo, hi, coef, X.T.copy()).T
        assert np.max(np.abs(Yd.cpu().numpy() - Yo)) <= 1e-13 * np.abs(X).max()


# ------------------------------------------------------------------------------ bounds
@pytest.mark.parametrize("dim,nx", [(2, 30), (3, 11)])
def test_bounds_match_oracle_and_enclose(ctx, oracle_mod, dim, nx):
    A = I.laplacian_2d(nx) if dim == 2 else I.laplacian_3d(nx)
    ctx.set_csr(A)
    lo, hi = ctx.bounds(80, 0)
    olo, ohi = oracle_mod.bounds(A, 80, 0)
    e = lap_eigs(dim, nx)
    assert abs(lo - olo) <= 1e-9 * e[-1] and abs(hi - ohi) <= 1e-9 * e[-1]
    assert lo <= e[0] + 1e-12 * e[-1] and hi >= e[-1] - 1e-12 * e[-1]


# ------------------------------------------------------------------------------ Lanczos
def _solve_both(ctx, nat, oracle_mod, A, a, b, m=None, tol=1e-8, **kw):
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    f = nat.cheb_filter_build(a, b, lo, hi)
    of = oracle_mod.filter_build(a, b, lo, hi)
    r = ctx.chebLanTr(a, b, f, m=m, tol=tol, **kw)
    o = oracle_mod.cheblantr(A, a, b, of, m=m, tol=tol, **kw)
    return r, o


@pytest.mark.parametrize("case", [("2d", 20, 1.0, 1.6), ("3d", 12, 0.8, 1.6),
                                  ("3d", 12, 0.0, 0.9), ("2d", 33, 7.5, 8.0)])
def test_cheblantr_laplacian(ctx, nat, oracle_mod, case):
    kind, nx, a, b = case
    A = I.laplacian_2d(nx) if kind == "2d" else I.laplacian_3d(nx)
    e = lap_eigs(2 if kind == "2d" else 3, nx)
    ex = e[(e >= a) & (e <= b)]
    r, o = _solve_both(ctx, nat, oracle_mod, A, a, b, m=max(2 * len(ex) + 40, 100))
    assert r["status"] == 0
    assert r["nev"] == o["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    Y = r["Y"][:r["nev"]].T
    assert np.max(_dense_residuals(A, r["lam"], Y)) <= 1e-8
    assert np.max(np.abs(r["res"] - _dense_residuals(A, r["lam"], Y))) <= 1e-12
    assert np.max(np.abs(Y.T @ Y - np.eye(r["nev"]))) <= 1e-10
    # same eigenspace as the oracle (vectors of repeated eigenvalues are not unique)
    P, Po = Y @ Y.T, o["Y"] @ o["Y"].T
    assert np.linalg.norm(P - Po, 2) <= 1e-7


def test_cheblantr_stats_count_filter_matvecs(ctx, nat):
    # matvec accounting: every Lanczos step applies the degree-d filter once, i.e. d products
    # with A, so nmv = deg * niter; the timings are non-negative and fit in the total
    A = I.laplacian_2d(40)
    ctx.set_csr(A)
    f = nat.cheb_filter_build(0.5, 0.8, 0.0, 8.0)
    r = ctx.chebLanTr(0.5, 0.8, f, m=120)
    st = r["stats"]
    assert r["status"] == 0 and st["niter"] > 0
    assert st["nmv"] == f.deg * st["niter"]
    assert min(st["t_filter"], st["t_orth"], st["t_restart"]) >= 0.0
    assert st["t_filter"] + st["t_orth"] + st["t_restart"] <= st["t_total"] * 1.05 + 1e-3


@pytest.mark.parametrize("a,b", [(-1.0, 1.0), (3.0, 5.0)])
def test_cheblantr_anderson_bruteforce(ctx, nat, oracle_mod, a, b):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    ex = ev[(ev >= a) & (ev <= b)]
    r, o = _solve_both(ctx, nat, oracle_mod, A, a, b, m=max(2 * len(ex) + 40, 100))
    assert r["nev"] == o["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    assert np.max(_dense_residuals(A, r["lam"], r["Y"][:r["nev"]].T)) <= 1e-8


def test_cheblantr_config_2d_100(ctx, nat, oracle_mod):
    A = I.laplacian_2d(100)
    e = lap_eigs(2, 100)
    ex = e[(e >= 0.40) & (e <= 0.48)]
    r, o = _solve_both(ctx, nat, oracle_mod, A, 0.40, 0.48, m=2 * 69 + 40)
    assert r["status"] == 0 and r["nev"] == o["nev"] == 69
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * ex)
    assert np.all(np.abs(r["lam"] - o["lam"]) <= 1e-9 * ex)
    assert r["res"].max() <= 1e-8
    Y = r["Y"][:69].T
    assert np.max(np.abs(Y.T @ Y - np.eye(69))) <= 1e-10
    res = np.array([np.linalg.norm(oracle_mod.spmv(A, Y[:, j]) - r["lam"][j] * Y[:, j])
                    for j in range(69)]) / 8.0
    assert res.max() <= 1e-8


def test_cheblantr_device_output_matches_host_output(ctx, nat, oracle_mod):
    import torch
    A = I.laplacian_2d(24)
    ctx.set_csr(A)
    lo, hi = ctx.bounds(60, 0)
    f = nat.cheb_filter_build(2.0, 2.5, lo, hi)
    rh = ctx.chebLanTr(2.0, 2.5, f, m=100, cap=80)
    Yd = torch.zeros((80, A.n), dtype=torch.float64, device="cuda")
    rd = ctx.chebLanTr(2.0, 2.5, f, m=100, cap=80, Y=Yd)
    k = rh["nev"]
    assert rd["nev"] == k and np.array_equal(rh["lam"], rd["lam"])
    assert np.array_equal(rh["Y"][:k], Yd[:k].cpu().numpy())


def test_cheblantr_capacity_and_empty_slice(ctx, nat):
    A = I.laplacian_2d(24)
    ctx.set_csr(A)
    lo, hi = ctx.bounds(60, 0)
    f = nat.cheb_filter_build(2.0, 2.5, lo, hi)
    r = ctx.chebLanTr(2.0, 2.5, f, m=100, cap=5, allow_partial=True)
    assert r["status"] == -5 and r["nev"] == 5
    # a slice between two consecutive distinct eigenvalues holds nothing
    e = lap_eigs(2, 24)
    u = np.unique(np.round(e, 12))
    gap = np.argmax(np.diff(u[100:200])) + 100
    a, b = u[gap] + 1e-3, u[gap + 1] - 1e-3
    f = nat.cheb_filter_build(a, b, lo, hi)
    r = ctx.chebLanTr(a, b, f, m=60)
    assert r["status"] == 0 and r["nev"] == 0


def test_set_csr_validation_and_budget(nat):
    A = I.laplacian_2d(10)
    with nat.Context(0) as c:
        bad = I.CSR(A.n, A.row_ptr, A.col_idx.copy(), A.val)
        bad.col_idx[5] = A.n
        with pytest.raises(nat.EvslError) as ei:
            c.set_csr(bad)
        assert ei.value.code == -1
        with pytest.raises(nat.EvslError) as ei:
            c.bounds(10, 0)                    # no matrix set
        assert ei.value.code == -7
    with nat.Context(0, hbm_budget=1024) as c:
        with pytest.raises(nat.EvslError) as ei:
            c.set_csr(A)
        assert ei.value.code == -2


def test_launch_counter_and_profile(ctx, nat):
    A = I.laplacian_2d(64)
    ctx.set_csr(A)
    n0 = ctx.launch_count()
    ctx.profile(True)
    ctx.kpm_dos(30, 4, 0, 0.0, 8.0)
    launches, ms = ctx.profile_get(nat.K_KPM_STEP)
    ctx.profile(False)
    assert launches == 30 and ms > 0
    assert ctx.launch_count() - n0 >= 31


# ------------------------------------------------------------------------------ multi-slice filter
@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 2e-5)])
def test_filter_apply_multi_matches_oracle(ctx, nat, oracle_mod, prec, tol):
    # one column per slice, each with its own degree and coefficients, one launch per degree
    import torch
    A = I.anderson_3d(15, 4.0, 3)              # n = 3375: ragged last slice
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 60, 0)
    cuts = [-1.0, 0.5, 1.4, 2.0, 2.3, 3.5]
    filters = [nat.cheb_filter_build(cuts[i], cuts[i + 1], lo, hi) for i in range(5)]
    degs = [f.deg for f in filters]
    assert len(set(degs)) > 2
    X = np.random.default_rng(2).standard_normal((5, A.n))
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.empty_like(Xd)
    ctx.filter_apply_multi(filters, Xd, Yd, prec=prec)
    Y = Yd.cpu().numpy()
    for t, f in enumerate(filters):
        Yo = oracle_mod.filter_apply(A, lo, hi, f.coef, X[t].copy())[:, 0]
        scale = np.abs(f.coef).sum() * np.abs(X[t]).max()
        assert np.max(np.abs(Y[t] - Yo)) <= tol * scale, (t, degs[t])


def test_filter_apply_multi_single_and_degree_zero(ctx, nat, oracle_mod):
    import torch
    A = I.laplacian_2d(40)
    ctx.set_csr(A)
    f1 = nat.cheb_filter_build(1.0, 1.2, 0.0, 8.0)
    f0 = nat.cheb_filter_build(2.0, 2.5, 0.0, 8.0)
    f0.coef = np.array([0.3])
    f0.pol.deg = 0
    f0.pol.coef = f0.coef.ctypes.data_as(nat.C.POINTER(nat.C.c_double))
    X = np.random.default_rng(4).standard_normal((2, A.n))
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.empty_like(Xd)
    ctx.filter_apply_multi([f0, f1], Xd, Yd)
    Y = Yd.cpu().numpy()
    assert np.max(np.abs(Y[0] - 0.3 * X[0])) <= 1e-15
    Yref = torch.empty_like(Xd[1:2])
    ctx.filter_apply(f1, Xd[1:2].contiguous(), Yref)
    assert np.max(np.abs(Y[1] - Yref.cpu().numpy()[0])) <= 1e-12 * np.abs(f1.coef).sum() * np.abs(X[1]).max()


# ------------------------------------------------------------------------------ multi-slice Lanczos
def test_cheblantr_batch_equals_per_slice_runs(ctx, nat, oracle_mod):
    # the lockstep multi-slice driver performs, per slice, the same operations in the same order
    # as the single-slice one (the block filter kernel does each column's arithmetic exactly like
    # the one-vector kernel), so results agree bitwise
    A = I.laplacian_3d(14)
    e = lap_eigs(3, 14)
    ctx.set_csr(A)
    lo, hi = ctx.bounds(80, 0)
    cuts = [0.0, 0.9, 1.35, 1.7]
    slices = [(cuts[i], cuts[i + 1]) for i in range(3)]
    filters = [nat.cheb_filter_build(a, b, lo, hi) for a, b in slices]
    counts = [int(np.count_nonzero((e >= a) & (e < b))) for a, b in slices]
    ms = [max(2 * c + 40, 100) for c in counts]
    rc = [False, False, True]
    batch = ctx.chebLanTr_batch(slices, filters, ms, right_closed=rc)
    for j, ((a, b), f, m) in enumerate(zip(slices, filters, ms)):
        single = ctx.chebLanTr(a, b, f, m=m, right_closed=rc[j])
        assert batch[j]["status"] == 0
        assert batch[j]["nev"] == single["nev"] == counts[j] + (j == 2) * int(np.count_nonzero(e == cuts[3]))
        assert np.array_equal(batch[j]["lam"], single["lam"])
        k = single["nev"]
        assert np.array_equal(batch[j]["Y"][:k], single["Y"][:k])
        assert batch[j]["stats"]["niter"] == single["stats"]["niter"]


def test_cheblantr_batch_fp32_filter_anderson(ctx, nat, oracle_mod):
    # FP32 filter vectors, FP64 reorthogonalisation and Ritz step: the eigenpairs still meet the
    # FP64 tolerances (exact count vs dense eigensolve, residual <= 1e-8 ||A||)
    A = I.anderson_3d(8, 4.0, 0)                # spectrum [0.167, 12.07]
    ev = np.linalg.eigvalsh(A.to_dense())
    ctx.set_csr(A)
    lo, hi = ctx.bounds(80, 0)
    cuts = [1.5, 2.5, 3.2]
    slices = [(cuts[0], cuts[1]), (cuts[1], cuts[2])]
    filters = [nat.cheb_filter_build(a, b, lo, hi) for a, b in slices]
    counts = [int(np.count_nonzero((ev >= a) & (ev < b))) for a, b in slices]
    ms = [max(2 * c + 40, 100) for c in counts]
    out = ctx.chebLanTr_batch(slices, filters, ms, prec=nat.FP32, right_closed=[False, True])
    for j, (a, b) in enumerate(slices):
        ex = ev[(ev >= a) & ((ev < b) if j == 0 else (ev <= b))]
        assert out[j]["nev"] == len(ex)
        assert np.all(np.abs(out[j]["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
        Y = out[j]["Y"][:len(ex)].T
        assert np.max(_dense_residuals(A, out[j]["lam"], Y)) <= 1e-8


# ------------------------------------------------------------------------------ continuous batching
def test_batch_continuous_admission_same_results_alone_and_in_mix(ctx, nat):
    # jobs join a running batch at different steps and leave when done; each result equals the
    # job solved alone (bitwise: per-column arithmetic does not depend on the batch)
    A = I.laplacian_2d(40)
    ctx.set_csr(A)
    lo, hi = ctx.bounds(80, 0)
    e = lap_eigs(2, 40)
    slices = [(0.5, 0.8), (1.1, 1.3), (2.0, 2.2), (3.0, 3.1)]
    filters = [nat.cheb_filter_build(a, b, lo, hi) for a, b in slices]
    ms = [max(2 * int(np.count_nonzero((e >= a) & (e <= b))) + 40, 100) for a, b in slices]
    alone = [ctx.chebLanTr(a, b, f, m=m) for (a, b), f, m in zip(slices, filters, ms)]
    bt = nat.Batch(ctx)
    jobs, results, step = {}, {}, 0
    arrive = {0: [0, 1], 7: [2], 30: [3]}        # job index -> step at which it is admitted
    while len(results) < len(slices):
        for j in arrive.get(step, []):
            jobs[j] = bt.add(slices[j][0], slices[j][1], filters[j], ms[j], tag=j)
        for job in bt.step():
            results[job.tag] = job.result()
        step += 1
        assert step < 100000
    bt.close()
    for j in range(len(slices)):
        r, s = results[j], alone[j]
        assert r["status"] == 0 and r["nev"] == s["nev"] > 0
        assert np.array_equal(r["lam"], s["lam"])
        assert np.array_equal(r["Y"][:r["nev"]], s["Y"][:s["nev"]])



@pytest.mark.parametrize("prec", [0, 1])
def test_filter_graph_replay_matches_block_kernel_bitwise(ctx, nat, prec):
    # a single-vector filter application replays a cached CUDA graph of its degree launches;
    # its result must equal, bit for bit, the same column filtered by the direct block kernel,
    # on the first call (capture), on the second (replay), and after the matrix is replaced
    # (the cache holds device addresses of the matrix and must be dropped)
    import torch
    for nx in (20, 21):
        A = I.laplacian_3d(nx)
        ctx.set_csr(A)
        f = nat.cheb_filter_build(1.0, 1.3, 0.0, 12.0)
        assert f.deg >= 8
        X = torch.tensor(np.random.default_rng(nx).standard_normal((2, A.n)), device="cuda")
        Y2 = torch.empty_like(X)
        ctx.filter_apply(f, X, Y2, prec=prec)             # two columns: block kernel, direct
        for _ in range(2):
            Y1 = torch.full((1, A.n), np.nan, dtype=torch.float64, device="cuda")
            ctx.filter_apply(f, X[0:1].clone(), Y1, prec=prec)
            assert torch.equal(Y1[0], Y2[0])


# ------------------------------------------------------------------------------ non-restart Lanczos
@pytest.mark.parametrize("case", [("lap2d", 40, 0.5, 0.8), ("lap3d", 12, 0.8, 1.6)])
def test_cheblannr_laplacian_matches_closed_form_and_oracle(ctx, nat, oracle_mod, case):
    # ChebLanNr (one basis, no restarts) finds every copy of the multiple eigenvalues: exact
    # count and values against the closed form, residuals recomputed densely; the oracle's
    # non-restart run finds the same eigenvalues
    kind, nx, a, b = case
    A = I.laplacian_2d(nx) if kind == "lap2d" else I.laplacian_3d(nx)
    e = lap_eigs(2 if kind == "lap2d" else 3, nx)
    ex = e[(e >= a) & (e <= b)]
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    f = nat.cheb_filter_build(a, b, lo, hi)
    m = max(6 * len(ex), 200)
    r = ctx.chebLanNr(a, b, f, m=m)
    assert r["status"] == 0 and r["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    Y = r["Y"][:r["nev"]].T
    assert np.max(_dense_residuals(A, r["lam"], Y)) <= 1e-8
    assert np.max(np.abs(Y.T @ Y - np.eye(r["nev"]))) <= 1e-10
    assert r["stats"]["nmv"] == f.deg * r["stats"]["niter"]
    ro = oracle_mod.cheblannr(A, a, b, oracle_mod.filter_build(a, b, lo, hi), m=m)
    assert ro["nev"] == r["nev"]
    assert np.all(np.abs(ro["lam"] - r["lam"]) <= 1e-9 * np.maximum(1, np.abs(ex)))


@pytest.mark.parametrize("a,b", [(-1.0, 1.0), (3.0, 5.0)])
def test_cheblannr_anderson_bruteforce(ctx, nat, a, b):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    ex = ev[(ev >= a) & (ev <= b)]
    ctx.set_csr(A)
    lo, hi = ctx.bounds(80, 0)
    f = nat.cheb_filter_build(a, b, lo, hi)
    r = ctx.chebLanNr(a, b, f, m=max(6 * len(ex), 200))
    assert r["status"] == 0 and r["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    assert np.max(_dense_residuals(A, r["lam"], r["Y"][:r["nev"]].T)) <= 1e-8


def test_cheblannr_short_basis_reports_noconv_and_fp32_mode(ctx, nat):
    # a basis too short to converge every pair: the converged ones and EVSL_ERR_NOCONV;
    # the FP32 filter with the FP64 polish meets the FP64 tolerances
    A = I.laplacian_2d(40)
    e = lap_eigs(2, 40)
    ex = e[(e >= 0.5) & (e <= 0.8)]
    ctx.set_csr(A)
    f = nat.cheb_filter_build(0.5, 0.8, 0.0, 8.0)
    r = ctx.chebLanNr(0.5, 0.8, f, m=30, allow_partial=True)
    assert r["status"] == -4 and r["stats"]["niter"] == 30 and r["nev"] < len(ex)
    for lam in r["lam"]:
        assert np.min(np.abs(ex - lam)) <= 1e-9 * max(1.0, abs(lam))
    assert np.all(r["res"] <= 1e-8)
    r32 = ctx.chebLanNr(0.5, 0.8, f, m=300, prec=nat.FP32)
    assert r32["status"] == 0 and r32["nev"] == len(ex)
    assert np.all(np.abs(r32["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    assert np.max(_dense_residuals(A, r32["lam"], r32["Y"][:r32["nev"]].T)) <= 1e-8


# ------------------------------------------------------------------------------ subspace iteration
@pytest.mark.parametrize("a,b", [(-1.0, 1.0), (3.0, 5.0), (6.0, 6.5)])
def test_chebsi_anderson_bruteforce(ctx, nat, a, b):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    ex = ev[(ev >= a) & (ev <= b)]
    ctx.set_csr(A)
    lo, hi = ctx.bounds(80, 0)
    f = nat.cheb_filter_build(a, b, lo, hi)
    r = ctx.chebSI(a, b, f, nv=int(1.5 * len(ex)) + 20)
    assert r["status"] == 0 and r["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    Y = r["Y"][:r["nev"]].T
    assert np.max(_dense_residuals(A, r["lam"], Y)) <= 1e-8
    assert np.max(np.abs(Y.T @ Y - np.eye(r["nev"]))) <= 1e-10


def test_chebsi_laplacian_multiplicities_and_oracle(ctx, nat, oracle_mod):
    # the block holds every copy of the 2-D Laplacian's double eigenvalues; same eigenvalues as
    # the oracle's subspace iteration
    A = I.laplacian_2d(40)
    e = lap_eigs(2, 40)
    ex = e[(e >= 0.5) & (e <= 0.8)]
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    f = nat.cheb_filter_build(0.5, 0.8, lo, hi)
    nv = int(1.5 * len(ex)) + 20
    r = ctx.chebSI(0.5, 0.8, f, nv=nv)
    assert r["status"] == 0 and r["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    assert np.max(_dense_residuals(A, r["lam"], r["Y"][:r["nev"]].T)) <= 1e-8
    ro = oracle_mod.chebsi(A, 0.5, 0.8, oracle_mod.filter_build(0.5, 0.8, lo, hi), nv=nv)
    assert ro["nev"] == r["nev"]
    assert np.all(np.abs(ro["lam"] - r["lam"]) <= 1e-9 * np.maximum(1, np.abs(ex)))


def test_chebsi_too_few_passes_reports_noconv(ctx, nat):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    ex = ev[(ev >= 3.0) & (ev <= 5.0)]
    ctx.set_csr(A)
    lo, hi = ctx.bounds(80, 0)
    f = nat.cheb_filter_build(3.0, 5.0, lo, hi)
    r = ctx.chebSI(3.0, 5.0, f, nv=137, maxit=3, allow_partial=True)
    assert r["status"] == -4 and r["stats"]["niter"] <= 3 and r["nev"] < len(ex)
    for lam in r["lam"]:
        assert np.min(np.abs(ex - lam)) <= 1e-9 * max(1.0, abs(lam))
    assert np.all(r["res"] <= 1e-8)


# ------------------------------------------------------------------------------ Lanczos density
def test_landos_matches_oracle(ctx, nat, oracle_mod):
    # same seeded start vectors: the quadrature nodes and weights agree with the oracle's, and the
    # slices cut from them agree too
    A = I.anderson_3d(12, 4.0, 0)
    ctx.set_csr(A)
    m, nvec = 40, 6
    dg = ctx.landos(m, nvec, 4)
    do = oracle_mod.landos(A, m, nvec, 4)
    assert np.array_equal(dg["mused"], do["mused"])
    assert np.max(np.abs(dg["nodes"] - do["nodes"])) <= 1e-9 * 12.0
    assert np.max(np.abs(dg["weights"] - do["weights"])) <= 1e-9
    assert np.allclose(dg["weights"].sum(axis=1), 1.0, atol=1e-12)
    sli, est = nat.slice_by_landos(dg, A.n, 1.0, 5.0, 4)
    sli_o, est_o = oracle_mod.slicer_landos(do, A.n, 1.0, 5.0, 4)
    assert np.allclose(est, est_o, atol=1e-6 * A.n)

def test_batch_admission_respects_hbm_budget(nat):
    # a 64 MiB budget holds the matrix, the workspaces and a few jobs' bases (~6.6 MB each);
    # admission must then refuse with EVSL_ERR_NOMEM and leave the admitted jobs intact
    A = I.laplacian_2d(60)
    with nat.Context(0, hbm_budget=64 * 1024 * 1024) as c:
        c.set_csr(A)
        f = nat.cheb_filter_build(1.0, 1.1, 0.0, 8.0)
        bt = nat.Batch(c)
        admitted, refused = 0, 0
        for _ in range(40):
            try:
                bt.add(1.0, 1.1, f, 100, cap=64)
                admitted += 1
            except nat.EvslError as err:
                assert err.code == -2
                refused += 1
                break
        assert admitted >= 2 and refused == 1
        done = []
        while bt.active:
            done += bt.step()
        assert len(done) == admitted and all(j.result()["status"] == 0 for j in done)
        bt.close()


@pytest.mark.parametrize("case", [("lap2d", 40, 0.5, 0.8), ("lap3d", 14, 0.9, 1.35)])
def test_cheblantr_fp32_filter_meets_fp64_tolerances(ctx, nat, oracle_mod, case):
    # FP32 filter (phase 1, locking at 1e-6 or looser in a widened slice) followed by the FP64
    # polish (filtered subspace iteration on the locked block plus guard vectors, Rayleigh-Ritz
    # with A): same eigenpairs as the FP64 oracle within the FP64 tolerances
    kind, nx, a, b = case
    A = I.laplacian_2d(nx) if kind == "lap2d" else I.laplacian_3d(nx)
    e = lap_eigs(2 if kind == "lap2d" else 3, nx)
    ex = e[(e >= a) & (e <= b)]
    ctx.set_csr(A)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    f = nat.cheb_filter_build(a, b, lo, hi)
    r = ctx.chebLanTr(a, b, f, m=max(2 * len(ex) + 40, 100), prec=nat.FP32)
    assert r["status"] == 0 and r["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1, np.abs(ex)))
    Y = r["Y"][:r["nev"]].T
    assert np.max(_dense_residuals(A, r["lam"], Y)) <= 1e-8
    assert np.max(np.abs(Y.T @ Y - np.eye(r["nev"]))) <= 1e-10
