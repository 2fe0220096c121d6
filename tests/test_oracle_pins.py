"""Pins of the CPU oracle against facts fixed outside it: the paper's printed tables, closed
forms, exact identities, published generator outputs and brute-force dense eigensolves.

Each test names what it pins and where the expected value comes from.  numpy/scipy dense
routines appear here only as independent checks (never inside the oracle).
"""
import numpy as np
import pytest
from numpy.polynomial import chebyshev as npcheb

from closed_form import count_in, lap_eigs, nnz_formula, pencil_eigs
from conftest import golden
from paper_1802_05215_gb300 import inputs as I


# ---------------------------------------------------------------- SplitMix64 (seeded inputs)
def test_splitmix64_published_vectors(oracle_mod):
    for seed, *outs in golden("splitmix64_vectors.txt"):
        want = [int(x) for x in outs]
        assert oracle_mod.splitmix64_sequence(int(seed), 3) == want
        assert [int(x) for x in I.splitmix64_sequence(int(seed), 3)] == want


def test_counter_draw_matches_sequential_definition(oracle_mod):
    # draw(s, t, k) = the (k+1)-th output of SplitMix64 seeded with key(s, t), and
    # key(s, t) = first output of SplitMix64 seeded with s ^ (t * 0xD1B54A32D192ED03).
    for seed, stream in [(0, 1), (7, 2), (2**63 + 5, 3)]:
        s0 = (seed ^ (stream * 0xD1B54A32D192ED03)) & (2**64 - 1)
        key = oracle_mod.splitmix64_sequence(s0, 1)[0]
        seq = oracle_mod.splitmix64_sequence(key, 6)
        assert [oracle_mod.draw(seed, stream, k) for k in range(6)] == seq
        # the numpy implementation of the input module agrees
        assert [int(x) for x in I.draw(seed, stream, np.arange(6))] == seq


# ---------------------------------------------------------------- generators vs Table 1
def test_generator_structure_and_table1_nnz():
    for dim, nx, n, nnz, *_ in golden("table1_laplacians.txt"):
        dim, nx, n, nnz = int(dim), int(nx), int(n), int(nnz)
        assert nx ** dim == n
        assert nnz_formula(dim, nx) == nnz
    for dim, nx in [(2, 1), (2, 5), (2, 17), (3, 2), (3, 6), (3, 9)]:
        A = I.laplacian_2d(nx) if dim == 2 else I.laplacian_3d(nx)
        assert A.nnz == nnz_formula(dim, nx)
        D = A.to_dense()
        assert np.array_equal(D, D.T)
        for r in range(A.n):  # sorted columns
            assert np.all(np.diff(A.col_idx[A.row_ptr[r]:A.row_ptr[r + 1]]) > 0)
    A = I.laplacian_3d(49)
    assert (A.n, A.nnz) == (117649, 809137)


@pytest.mark.parametrize("dim,nx", [(2, 12), (3, 7)])
def test_generator_spectrum_is_closed_form(dim, nx):
    A = I.laplacian_2d(nx) if dim == 2 else I.laplacian_3d(nx)
    ev = np.linalg.eigvalsh(A.to_dense())
    assert np.max(np.abs(ev - lap_eigs(dim, nx))) < 1e-12


def test_closed_form_reproduces_table1_counts():
    for dim, nx, n, nnz, a, b, xi, eta, nu in golden("table1_laplacians.txt"):
        e = lap_eigs(int(dim), int(nx))
        assert count_in(e, float(xi), float(eta)) == int(nu)


def test_anderson_diagonal_is_seeded_uniform():
    A = I.anderson_3d(6, 4.0, 0)
    diag = A.to_dense().diagonal()
    assert np.all(diag >= 4.0) and np.all(diag < 8.0)
    assert np.array_equal(diag, 6.0 + I.anderson_diagonal(216, 4.0, 0))
    assert not np.array_equal(diag, 6.0 + I.anderson_diagonal(216, 4.0, 1))


# ---------------------------------------------------------------- dense symmetric eigensolver
@pytest.mark.parametrize("n", [1, 2, 3, 8, 40, 97])
def test_syev_random(oracle_mod, n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    M = M + M.T
    w, Z = oracle_mod.syev(M)
    scale = max(1.0, np.abs(M).max())
    assert np.max(np.abs(w - np.linalg.eigvalsh(M))) < 1e-13 * n * scale
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(Z.T @ Z - np.eye(n))) < 1e-13 * n
    assert np.max(np.abs(M @ Z - Z * w)) < 1e-13 * n * scale


def test_syev_special_structures(oracle_mod):
    # repeated eigenvalues: Q diag(1,1,1,2,2,5) Q^T
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    lam = np.array([1, 1, 1, 2, 2, 5.0])
    M = (Q * lam) @ Q.T
    w, Z = oracle_mod.syev(M)
    assert np.max(np.abs(w - lam)) < 1e-13
    assert np.max(np.abs(M @ Z - Z * w)) < 1e-13
    # already diagonal, and an arrowhead + tridiagonal matrix as thick restart produces
    w, _ = oracle_mod.syev(np.diag([3.0, -1.0, 2.0]))
    assert np.array_equal(w, [-1.0, 2.0, 3.0])
    T = np.diag([0.9, 0.95, 0.99, 0.3, 0.1, -0.2])
    T[:3, 3] = T[3, :3] = [1e-3, -2e-2, 5e-4]
    T[3, 4] = T[4, 3] = 0.4
    T[4, 5] = T[5, 4] = 0.1
    w, Z = oracle_mod.syev(T)
    assert np.max(np.abs(w - np.linalg.eigvalsh(T))) < 1e-14


# ---------------------------------------------------------------- spectral bounds
@pytest.mark.parametrize("dim,nx", [(2, 20), (3, 10), (2, 100)])
def test_bounds_enclose_closed_form_extremes(oracle_mod, dim, nx):
    A = I.laplacian_2d(nx) if dim == 2 else I.laplacian_3d(nx)
    e = lap_eigs(dim, nx)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    # enclosure up to rounding (a fully converged run gives the extremes to ~1e-15)
    assert lo <= e[0] + 1e-13 * e[-1] and hi >= e[-1] - 1e-13 * e[-1]
    assert (e[0] - lo) < 1e-2 * e[-1] and (hi - e[-1]) < 1e-2 * e[-1]


# ---------------------------------------------------------------- KPM moments and DOS
def _diag_csr(d):
    n = len(d)
    return I.CSR(n, np.arange(n + 1), np.arange(n, dtype=np.int32), np.asarray(d, float))


def test_kpm_exact_on_diagonal_matrix(oracle_mod):
    # For A = diag(lambda_i) and Rademacher v (v_i^2 = 1): v^T T_k(Ahat) v = sum_i T_k(lambda_hat_i)
    rng = np.random.default_rng(0)
    d = np.sort(rng.uniform(-3, 5, 300))
    lmin, lmax = -3.5, 5.25
    mu = oracle_mod.kpm_moments(_diag_csr(d), 60, 3, 11, lmin, lmax)
    lh = (d - 0.5 * (lmax + lmin)) / (0.5 * (lmax - lmin))
    want = np.array([np.cos(k * np.arccos(lh)).sum() for k in range(61)])
    assert mu[0] == len(d)
    assert np.max(np.abs(mu - want)) < 1e-12 * len(d)


def test_kpm_matches_dense_spectral_formula(oracle_mod):
    # mu_k = mean_l v_l^T Z diag(T_k(lambda_hat)) Z^T v_l, with Z from a dense eigensolve
    A = I.anderson_3d(5, 3.0, 2)
    lmin, lmax = -1.0, 14.0
    M, nv, seed = 30, 4, 5
    mu = oracle_mod.kpm_moments(A, M, nv, seed, lmin, lmax)
    w, Z = np.linalg.eigh(A.to_dense())
    lh = (w - 6.5) / 7.5           # c = (lmax + lmin)/2, d = (lmax - lmin)/2
    V = I.rademacher_block(A.n, nv, seed)
    P = Z.T @ V
    want = np.array([np.mean(np.sum(P * P * np.cos(k * np.arccos(lh))[:, None], axis=0))
                     for k in range(M + 1)])
    assert np.max(np.abs(mu - want)) < 1e-11 * A.n


def test_kpm_statistics_against_closed_form_trace(oracle_mod):
    # E[v^T T_k v] = tr T_k(Ahat) = sum_i cos(k arccos lambda_hat_i) (closed-form spectrum);
    # the stochastic error is below 6 sqrt(2 ||T_k||_F^2 / nvec).
    nx, M, nv = 30, 40, 20
    A = I.laplacian_2d(nx)
    e = lap_eigs(2, nx)
    lmin, lmax = 0.0, 8.0
    mu = oracle_mod.kpm_moments(A, M, nv, 0, lmin, lmax)
    lh = (e - 4.0) / 4.0
    for k in range(M + 1):
        tk = np.cos(k * np.arccos(lh))
        sig = np.sqrt(2.0 * np.sum(tk * tk) / nv)
        assert abs(mu[k] - tk.sum()) <= 6 * sig + 1e-9



@pytest.mark.parametrize("M", [0, 1, 7, 40])
def test_kpm_doubling_matches_direct_moments(oracle_mod, M):
    # T_{2k} = 2 T_k^2 - T_0 and T_{2k+1} = 2 T_{k+1} T_k - T_1: the doubled moments equal the
    # directly computed ones (same probes) up to rounding; mu_0 = n exactly
    A = I.anderson_3d(8, 4.0, 0)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    mu_d = oracle_mod.kpm_moments(A, M, 5, 3, lo, hi)
    mu_x = oracle_mod.kpm_moments_doubling(A, M, 5, 3, lo, hi)
    assert mu_x[0] == A.n
    assert np.max(np.abs(mu_x - mu_d)) <= 1e-11 * A.n

def test_jackson_coefficients_identities(oracle_mod):
    for M in [1, 5, 80, 300]:
        g = oracle_mod.jackson(M)
        a = np.pi / (M + 2)
        assert abs(g[0] - 1.0) < 1e-15
        assert abs(g[1] - np.cos(a)) < 1e-14          # first factor is cos(pi/(M+2))
        assert np.all(np.diff(g) <= 1e-15)            # decreasing
        # the damped delta kernel g_0/2 + sum g_k T_k(x) T_k(y) is non-negative
        x = np.cos(np.linspace(0, np.pi, 301))
        for y in [-0.9, 0.0, 0.37]:
            ker = 0.5 * g[0] + sum(g[k] * np.cos(k * np.arccos(x)) * np.cos(k * np.arccos(y))
                                   for k in range(1, M + 1))
            assert ker.min() > -1e-12 * ker.max()


def test_dos_count_endpoints_and_monotone(oracle_mod):
    A = I.laplacian_2d(40)
    lo, hi = oracle_mod.bounds(A, 60, 0)
    mu = oracle_mod.kpm_moments(A, 80, 10, 1, lo, hi)
    assert mu[0] == A.n
    assert abs(oracle_mod.dos_count(mu, lo, hi, hi) - A.n) < 1e-9
    # (t - c)/d at t = lmin is -1 only up to rounding; arccos is sqrt-sensitive there
    assert abs(oracle_mod.dos_count(mu, lo, hi, lo)) < 1e-9 * A.n
    ts = np.linspace(lo, hi, 200)
    N = np.array([oracle_mod.dos_count(mu, lo, hi, t) for t in ts])
    assert np.all(np.diff(N) >= -1e-8 * A.n)
    # smoothed count tracks the exact count to within the kernel width
    e = lap_eigs(2, 40)
    exact = np.array([np.count_nonzero(e <= t) for t in ts])
    assert np.max(np.abs(N - exact)) < 0.05 * A.n


def test_slicer_balances_table4_case(oracle_mod):
    # 49^3 Laplacian on [0, 1]: exact per-slice counts from the closed form must be balanced
    # (Table 4's own spread is 307..345 around 328.5 for six slices)
    A = I.laplacian_3d(49)
    e = lap_eigs(3, 49)
    assert count_in(e, 0.0, 1.0) == 1971
    lo, hi = oracle_mod.bounds(A, 80, 0)
    mu = oracle_mod.kpm_moments(A, 100, 10, 0, lo, hi)
    for ns in [2, 6]:
        sli, est = oracle_mod.slicer(mu, lo, hi, 0.0, 1.0, ns)
        assert sli[0] == 0.0 and sli[-1] == 1.0 and np.all(np.diff(sli) > 0)
        counts = [count_in(e, sli[i], sli[i + 1], right_closed=(i == ns - 1)) for i in range(ns)]
        assert sum(counts) == 1971
        assert max(counts) / min(counts) < 1.3
        assert abs(sum(est) - 1971) < 0.1 * 1971


# ---------------------------------------------------------------- filter construction
def _rho(pol, t):
    c = 0.5 * (pol["lmax"] + pol["lmin"])
    d = 0.5 * (pol["lmax"] - pol["lmin"])
    return npcheb.chebval((np.asarray(t) - c) / d, pol["coef"])


def test_filter_degrees_table2(oracle_mod):
    # sigma damping, tau = 0.8, [a, b] from Table 1.  10 of 12 printed degrees are met
    # exactly; 81^3 [0.40, 0.45] (141) and 100^3 [1.00, 1.018] (588) come out one lower,
    # which the unprinted digits of b = 11.9882 can account for.
    off = []
    for dim, nx, xi, eta, deg in golden("table2_degrees.txt"):
        b = 7.9998 if dim == "2" else 11.9882
        pol = oracle_mod.filter_build(float(xi), float(eta), 0.0, b, damping=oracle_mod.DAMP_SIGMA)
        if pol["deg"] != int(deg):
            off.append((nx, xi, int(deg), pol["deg"]))
    assert off == [("81", "0.40", 141, 140), ("100", "1.00", 588, 587)]


def test_filter_degrees_table4(oracle_mod):
    # all 21 printed degrees, interior slices and the left boundary slices
    for ns, i, left, right, nu, deg in golden("table4_slices.txt"):
        pol = oracle_mod.filter_build(float(left), float(right), 0.0, 11.9882,
                                      damping=oracle_mod.DAMP_SIGMA)
        assert pol["deg"] == int(deg), (ns, i)
        assert pol["boundary"] == (-1 if i == "0" else 0)


@pytest.mark.parametrize("damping", [0, 1, 2])
def test_filter_shape_properties(oracle_mod, damping):
    lmin, lmax = 0.0, 8.0
    a, b = 0.40, 0.48
    pol = oracle_mod.filter_build(a, b, lmin, lmax, damping=damping)
    k = pol["deg"]
    assert abs(_rho(pol, 4.0 + 4.0 * pol["gamma"]) - 1.0) < 1e-12        # rho(gamma) = 1
    ra, rb = _rho(pol, a), _rho(pol, b)
    assert abs(ra - rb) < 1e-10 and abs(ra - pol["bar"]) < 1e-10 and pol["bar"] <= 0.8
    assert a < 4.0 + 4.0 * pol["gamma"] < b
    if damping == 1:
        assert k == 97
    # minimality: the balanced filter of degree k-1 does not reach tau
    prev = oracle_mod.filter_build(a, b, lmin, lmax, damping=damping, maxdeg=k - 1)
    assert prev["reached_max"] and prev["bar"] > 0.8


def test_filter_apply_matches_spectral_evaluation(oracle_mod):
    A = I.laplacian_3d(6)
    lmin, lmax = 0.0, 12.0
    pol = oracle_mod.filter_build(2.0, 2.5, lmin, lmax)
    X = np.random.default_rng(0).standard_normal((A.n, 3))
    Y = oracle_mod.filter_apply(A, lmin, lmax, pol["coef"], X)
    w, Z = np.linalg.eigh(A.to_dense())
    want = Z @ (_rho(pol, w)[:, None] * (Z.T @ X))
    assert np.max(np.abs(Y - want)) < 1e-12 * np.abs(X).max() * len(pol["coef"])


# ---------------------------------------------------------------- filtered TR Lanczos
def _check_eigs(A, r, ex, tol_res=1e-8):
    assert r["nev"] == len(ex)
    lam = r["lam"]
    assert np.all(np.abs(lam - ex) <= 1e-9 * np.maximum(1.0, np.abs(ex)))
    Y = r["Y"]
    normA = np.abs(np.linalg.eigvalsh(A.to_dense())).max() if A.n <= 2000 else None
    R = np.column_stack([A.to_dense() @ Y[:, j] for j in range(Y.shape[1])]) if A.n <= 2000 \
        else None
    if R is not None:
        res = np.linalg.norm(R - Y * lam, axis=0) / normA
        assert res.max() <= tol_res
    assert np.max(np.abs(Y.T @ Y - np.eye(len(lam)))) <= 1e-10


@pytest.mark.parametrize("case", [
    ("2d", 20, 1.0, 1.6), ("3d", 12, 0.8, 1.6), ("3d", 10, 2.0, 2.6), ("3d", 12, 0.0, 0.9),
])
def test_cheblantr_against_closed_form(oracle_mod, case):
    kind, nx, a, b = case
    A = I.laplacian_2d(nx) if kind == "2d" else I.laplacian_3d(nx)
    e = lap_eigs(2 if kind == "2d" else 3, nx)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = e[(e >= a) & (e <= b)]
    r = oracle_mod.cheblantr(A, a, b, pol, m=max(2 * len(ex) + 40, 100))
    assert r["status"] == 0
    _check_eigs(A, r, ex)


def test_cheblantr_multiplicity_eigenspaces(oracle_mod):
    # 3-D Laplacian has eigenvalues of multiplicity 3 and 6: compare eigenspaces, not vectors
    A = I.laplacian_3d(10)
    w, Z = np.linalg.eigh(A.to_dense())
    a, b = 2.0, 2.6
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    r = oracle_mod.cheblantr(A, a, b, pol, m=120)
    sel = (w >= a) & (w <= b)
    P_ref = Z[:, sel] @ Z[:, sel].T
    P = r["Y"] @ r["Y"].T
    assert np.linalg.norm(P - P_ref, 2) < 1e-7


@pytest.mark.parametrize("a,b", [(-1.0, 1.0), (3.0, 5.0), (6.0, 6.5)])
def test_cheblantr_anderson_bruteforce(oracle_mod, a, b):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    lo, hi = oracle_mod.bounds(A, 80, 0)
    assert lo <= ev[0] + 1e-13 * ev[-1] and hi >= ev[-1] - 1e-13 * ev[-1]
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = ev[(ev >= a) & (ev <= b)]
    r = oracle_mod.cheblantr(A, a, b, pol, m=max(2 * len(ex) + 40, 100))
    assert r["status"] == 0
    _check_eigs(A, r, ex)



# ---------------------------------------------------------------- filtered non-restart Lanczos
@pytest.mark.parametrize("case", [("2d", 20, 1.0, 1.6), ("2d", 40, 0.5, 0.8), ("3d", 12, 0.8, 1.6)])
def test_cheblannr_against_closed_form(oracle_mod, case):
    # one Krylov space finds every copy of the Laplacians' multiple eigenvalues (multiplicity 2
    # in 2-D, up to 6 in 3-D): the copies beyond the first grow from rounding in the basis
    kind, nx, a, b = case
    A = I.laplacian_2d(nx) if kind == "2d" else I.laplacian_3d(nx)
    e = lap_eigs(2 if kind == "2d" else 3, nx)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = e[(e >= a) & (e <= b)]
    r = oracle_mod.cheblannr(A, a, b, pol, m=max(6 * len(ex), 200))
    assert r["status"] == 0
    _check_eigs(A, r, ex)
    assert r["nmv"] == r["niter"] * (len(pol["coef"]) - 1)


@pytest.mark.parametrize("a,b", [(-1.0, 1.0), (3.0, 5.0), (6.0, 6.5)])
def test_cheblannr_anderson_bruteforce(oracle_mod, a, b):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = ev[(ev >= a) & (ev <= b)]
    r = oracle_mod.cheblannr(A, a, b, pol, m=max(6 * len(ex), 200))
    assert r["status"] == 0
    _check_eigs(A, r, ex)


def test_cheblannr_short_basis_reports_noconv(oracle_mod):
    # a basis too short to converge every pair returns the converged ones and status -4
    A = I.laplacian_2d(40)
    e = lap_eigs(2, 40)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(0.5, 0.8, lo, hi)
    r = oracle_mod.cheblannr(A, 0.5, 0.8, pol, m=30)
    assert r["status"] == -4 and r["niter"] == 30 and r["nev"] < 40
    ex = e[(e >= 0.5) & (e <= 0.8)]
    for lam in r["lam"]:
        assert np.min(np.abs(ex - lam)) <= 1e-9 * max(1.0, abs(lam))
    assert np.all(r["res"] <= 1e-8)


# ---------------------------------------------------------------- filtered subspace iteration
@pytest.mark.parametrize("a,b", [(-1.0, 1.0), (3.0, 5.0), (6.0, 6.5)])
def test_chebsi_anderson_bruteforce(oracle_mod, a, b):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = ev[(ev >= a) & (ev <= b)]
    r = oracle_mod.chebsi(A, a, b, pol, nv=int(1.5 * len(ex)) + 20)
    assert r["status"] == 0
    _check_eigs(A, r, ex)


@pytest.mark.parametrize("case", [("2d", 40, 0.5, 0.8), ("3d", 12, 0.8, 1.6)])
def test_chebsi_against_closed_form(oracle_mod, case):
    # a block iteration holds every copy of a multiple eigenvalue from the start
    kind, nx, a, b = case
    A = I.laplacian_2d(nx) if kind == "2d" else I.laplacian_3d(nx)
    e = lap_eigs(2 if kind == "2d" else 3, nx)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = e[(e >= a) & (e <= b)]
    r = oracle_mod.chebsi(A, a, b, pol, nv=int(1.5 * len(ex)) + 20)
    assert r["status"] == 0
    _check_eigs(A, r, ex)


def test_chebsi_too_few_passes_reports_noconv(oracle_mod):
    A = I.anderson_3d(7, 4.0, 0)
    ev = np.linalg.eigvalsh(A.to_dense())
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(3.0, 5.0, lo, hi)
    r = oracle_mod.chebsi(A, 3.0, 5.0, pol, nv=137, maxit=3)
    assert r["status"] == -4 and r["niter"] <= 3
    ex = ev[(ev >= 3.0) & (ev <= 5.0)]
    for lam in r["lam"]:
        assert np.min(np.abs(ex - lam)) <= 1e-9 * max(1.0, abs(lam))
    assert np.all(r["res"] <= 1e-8)


# ---------------------------------------------------------------- Lanczos density (quadrature)
def test_landos_full_run_is_the_exact_spectral_measure(oracle_mod):
    # a full-length run on a matrix with distinct eigenvalues: the nodes are the eigenvalues and
    # the weights (v . x_j)^2 for the normalised seeded start vector v (stream 5, vector 0)
    A = I.anderson_3d(7, 4.0, 0)
    w, Z = np.linalg.eigh(A.to_dense())
    v = I.start_vector(A.n, 3, I.STREAM_LANDOS, 0)
    v /= np.linalg.norm(v)
    d = oracle_mod.landos(A, A.n, 1, 3)
    k = int(d["mused"][0])
    assert k == A.n
    assert np.max(np.abs(np.sort(d["nodes"][0, :k]) - w)) <= 1e-10 * np.abs(w).max()
    order = np.argsort(d["nodes"][0, :k])
    assert np.max(np.abs(d["weights"][0, :k][order] - (Z.T @ v) ** 2)) <= 1e-10


def test_landos_quadrature_is_exact_to_degree_2m_minus_1(oracle_mod):
    # m-point Gauss quadrature from m Lanczos steps integrates t^p exactly for p <= 2m - 1:
    # sum_j tau_j theta_j^p = v^T A^p v (v the normalised start vector), and sum_j tau_j = 1
    A = I.laplacian_3d(10)
    D = A.to_dense()
    m, nvec = 6, 3
    d = oracle_mod.landos(A, m, nvec, 7)
    for l in range(nvec):
        v = I.start_vector(A.n, 7, I.STREAM_LANDOS, l)
        v /= np.linalg.norm(v)
        th, tau = d["nodes"][l, :m], d["weights"][l, :m]
        x = v.copy()
        for p in range(2 * m):
            assert abs(np.sum(tau * th ** p) - v @ x) <= 1e-10 * 12.0 ** p
            x = D @ x


def test_landos_count_tracks_closed_form(oracle_mod):
    # the cumulative quadrature count estimates the exact eigenvalue count of a 12^3 Laplacian
    # (statistical: 30 vectors; the count at the top is n exactly)
    A = I.laplacian_3d(12)
    e = lap_eigs(3, 12)
    d = oracle_mod.landos(A, 40, 30, 1)
    assert abs(oracle_mod.landos_count(d, A.n, 13.0) - A.n) <= 1e-9 * A.n
    for t in (2.0, 4.0, 6.0, 8.0, 10.0):
        exact = np.count_nonzero(e <= t)
        assert abs(oracle_mod.landos_count(d, A.n, t) - exact) <= 0.03 * A.n


def test_slicer_ends_hit_the_quantiles_of_the_interpolated_count(oracle_mod):
    # on a coarse grid x_0..x_{N-1} of [xi, eta], the slice ends are where the piecewise-linear
    # interpolant of the cumulative count N(x_j) reaches the equal shares C_0 + (i/ns)(C_{N-1} - C_0)
    # (first crossing, then linear interpolation between the grid points around it); the
    # counts N(x_j) come from the separately pinned dos_count
    A = I.laplacian_2d(40)
    lo, hi = oracle_mod.bounds(A, 60, 0)
    mu = oracle_mod.kpm_moments(A, 80, 10, 1, lo, hi)
    xi, eta = 0.5, 6.5
    for ns, npts in [(4, 9), (3, 7), (5, 16)]:
        sli, est = oracle_mod.slicer(mu, lo, hi, xi, eta, ns, npts)
        x = np.linspace(xi, eta, npts)
        C = np.array([oracle_mod.dos_count(mu, lo, hi, t) for t in x])
        assert np.all(np.diff(C) > 0)
        for i in range(1, ns):
            target = C[0] + (C[-1] - C[0]) * i / ns
            assert abs(np.interp(sli[i], x, C) - target) <= 1e-9 * A.n
        for i in range(ns):
            assert abs(est[i] - (oracle_mod.dos_count(mu, lo, hi, sli[i + 1]) - oracle_mod.dos_count(mu, lo, hi, sli[i]))) <= 1e-9 * A.n


def test_slicer_landos_hand_computed_cuts(oracle_mod):
    # small quadratures whose cuts follow by hand from the reading: a cut goes midway between the
    # first node at which the cumulative count reaches the equal share and the node before it;
    # est counts nodes in [t_i, t_{i+1}) ([t_i, t_{i+1}] for the last slice)
    one = lambda nodes, weights: dict(nodes=np.array([nodes]), weights=np.array([weights]),
                                      mused=np.array([len(nodes)], dtype=np.int32))
    d = one([0.1, 0.3, 0.5, 0.7, 0.9], [0.2] * 5)            # counts 20 per node (n = 100)
    sli, est = oracle_mod.slicer_landos(d, 100, 0.0, 1.0, 2)  # share 50: reached at 0.5
    assert np.allclose(sli, [0.0, 0.4, 1.0], atol=1e-15) and np.allclose(est, [40, 60], atol=1e-12)
    d = one([0.1, 0.3, 0.5, 0.7, 0.9], [0.1, 0.2, 0.3, 0.2, 0.2])   # counts 10, 20, 30, 20, 20
    sli, est = oracle_mod.slicer_landos(d, 100, 0.0, 1.0, 4)  # shares 25, 50, 75
    assert np.allclose(sli, [0.0, 0.2, 0.4, 0.6, 1.0], atol=1e-15)
    assert np.allclose(est, [10, 20, 30, 40], atol=1e-12)
    # two probes merge into one sorted quadrature (each node counts 25); the share 50 is reached
    # exactly at the second node, which is where the cut goes
    d = dict(nodes=np.array([[0.1, 0.5], [0.3, 0.7]]), weights=np.full((2, 2), 0.5),
             mused=np.array([2, 2], dtype=np.int32))
    sli, est = oracle_mod.slicer_landos(d, 100, 0.0, 1.0, 2)
    assert np.allclose(sli, [0.0, 0.2, 1.0], atol=1e-15) and np.allclose(est, [25, 75], atol=1e-12)


def test_slicer_landos_balances_within_one_node(oracle_mod):
    # the slices partition [xi, eta]; their counts add up to the total, and each differs from
    # the equal share by at most the largest single node weight (first-crossing rule); on an
    # Anderson model (no multiple eigenvalues) the exact counts of the slices are balanced
    A = I.anderson_3d(12, 4.0, 0)
    e = np.linalg.eigvalsh(A.to_dense())
    d = oracle_mod.landos(A, 80, 200, 2)
    xi, eta, ns = 1.0, 5.0, 4
    sli, est = oracle_mod.slicer_landos(d, A.n, xi, eta, ns)
    assert sli[0] == xi and sli[-1] == eta and np.all(np.diff(sli) > 0)
    total = oracle_mod.landos_count(d, A.n, eta) - oracle_mod.landos_count(d, A.n, np.nextafter(xi, -1))
    assert abs(est.sum() - total) <= 1e-9 * A.n
    wmax = A.n * d["weights"].max() / d["nodes"].shape[0]
    assert np.all(np.abs(est - total / ns) <= wmax + 1e-9 * A.n)
    exact = np.array([np.count_nonzero((e >= sli[i]) & ((e < sli[i + 1]) if i < ns - 1 else (e <= sli[i + 1])))
                      for i in range(ns)])
    assert exact.max() / exact.min() <= 1.3


# ---------------------------------------------------------------- generalized problems (Sec. 2.4)
def _pencil_eigs(nx):
    return pencil_eigs(nx)


def test_pencil_generator_closed_form():
    A, B = I.laplacian_2d(7), I.mass_matrix_2d(7)
    import scipy.linalg as sl
    w = sl.eigh(A.to_dense(), B.to_dense(), eigvals_only=True)
    assert np.max(np.abs(w - _pencil_eigs(7))) <= 1e-12 * w.max()


def test_lspol_is_a_polynomial_inverse(oracle_mod):
    # |t p(t) - 1| <= eps on an independent fine grid, and p(B) x solves B y = x
    lp = oracle_mod.lspol(0.11, 0.99, 1e-13)
    assert lp["status"] == 0
    tt = np.linspace(0.11, 0.99, 10001)
    p = npcheb.chebval((tt - 0.55) / 0.44, lp["coef"])
    assert np.max(np.abs(tt * p - 1.0)) <= 1.5e-13
    B = I.mass_matrix_2d(12)
    lo, hi = oracle_mod.bounds(B, 80, 0)
    lp = oracle_mod.lspol(lo, hi, 1e-13)
    x = np.random.default_rng(0).standard_normal(B.n)
    y = oracle_mod.poly_solve(B, lp, x)
    assert np.linalg.norm(B.to_dense() @ y - x) <= 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("a,b", [(2.0, 3.0), (10.0, 11.0), (40.0, 42.0)])
def test_cheblannr_gen_against_closed_form(oracle_mod, a, b):
    # A x = lambda B x with B^{-1} by lsPol: exact count (multiplicity 2), eigenvalues, residuals
    # ||A x - lambda B x|| and B-orthonormality against the closed form and dense products
    nx = 20
    A, B = I.laplacian_2d(nx), I.mass_matrix_2d(nx)
    lam = _pencil_eigs(nx)
    blo, bhi = oracle_mod.bounds(B, 80, 0)
    lp = oracle_mod.lspol(blo, bhi, 1e-13)
    lo, hi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    assert lo <= lam[0] and hi >= lam[-1] - 1e-9 * lam[-1]
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = lam[(lam >= a) & (lam <= b)]
    r = oracle_mod.cheblannr_gen(A, B, lp, a, b, pol, m=max(6 * len(ex), 200))
    assert r["status"] == 0 and r["nev"] == len(ex)
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1.0, ex))
    X, Ad, Bd = r["Y"], A.to_dense(), B.to_dense()
    R = Ad @ X - (Bd @ X) * r["lam"]
    assert np.max(np.linalg.norm(R, axis=0)) <= 1e-8 * bhi * hi
    assert np.max(np.abs(X.T @ Bd @ X - np.eye(len(ex)))) <= 1e-10

def test_cheblantr_half_open_slices_partition(oracle_mod):
    # adjacent half-open slices [a, cut) and [cut, b] neither lose nor duplicate eigenvalues
    # (cut midway between two distinct eigenvalues, so rounding cannot decide membership)
    A = I.laplacian_2d(16)
    e = lap_eigs(2, 16)
    cut = 0.5 * (e[100] + e[102]) if e[102] - e[100] > 1e-6 else 0.5 * (e[100] + e[101])
    lo, hi = oracle_mod.bounds(A, 80, 0)
    found = []
    for (a, b, rc) in [(cut - 0.3, cut, False), (cut, cut + 0.3, True)]:
        pol = oracle_mod.filter_build(a, b, lo, hi)
        r = oracle_mod.cheblantr(A, a, b, pol, m=120, right_closed=rc)
        found.append(r["lam"])
    allf = np.sort(np.concatenate(found))
    ex = e[(e >= cut - 0.3) & (e <= cut + 0.3)]
    assert len(allf) == len(ex) and np.max(np.abs(allf - ex)) < 1e-12


def test_cheblantr_config_2d_100(oracle_mod):
    # the 100 x 100 2-D Laplacian on [0.40, 0.48]: exactly 69 eigenvalues (multiplicity 2)
    A = I.laplacian_2d(100)
    e = lap_eigs(2, 100)
    ex = e[(e >= 0.40) & (e <= 0.48)]
    assert len(ex) == 69
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(0.40, 0.48, lo, hi)
    r = oracle_mod.cheblantr(A, 0.40, 0.48, pol, m=2 * 69 + 40)
    assert r["status"] == 0 and r["nev"] == 69
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * ex)
    assert r["res"].max() <= 1e-8
    assert np.max(np.abs(r["Y"].T @ r["Y"] - np.eye(69))) <= 1e-10


def test_lspol_isqrt_is_a_polynomial_inverse_square_root(oracle_mod):
    # |sqrt(t) q(t) - 1| <= eps on an independent fine grid, and q(B)^2 is B^{-1} on a vector
    lq = oracle_mod.lspol_isqrt(0.11, 0.99, 1e-13)
    assert lq["status"] == 0
    tt = np.linspace(0.11, 0.99, 10001)
    q = npcheb.chebval((tt - 0.55) / 0.44, lq["coef"])
    assert np.max(np.abs(np.sqrt(tt) * q - 1.0)) <= 1.5e-13
    B = I.mass_matrix_2d(12)
    lo, hi = oracle_mod.bounds(B, 80, 0)
    lq = oracle_mod.lspol_isqrt(lo, hi, 1e-13)
    x = np.random.default_rng(1).standard_normal(B.n)
    y = oracle_mod.poly_solve(B, lq, oracle_mod.poly_solve(B, lq, x))
    assert np.linalg.norm(B.to_dense() @ y - x) <= 1e-12 * np.linalg.norm(x)


def _pencil_lsp(oracle_mod, A, B):
    blo, bhi = oracle_mod.bounds(B, 80, 0)
    return oracle_mod.lspol(blo, bhi, 1e-13), oracle_mod.lspol_isqrt(blo, bhi, 1e-13)


def test_kpm_gen_matches_dense_pencil_formula(oracle_mod):
    # mu_k = mean_l v_l^T T_k(Shat) v_l with S = B^{-1/2} A B^{-1/2} from dense eigensolves and the
    # same Rademacher probes; mu_0 = n up to the polynomials' 1e-13
    nx = 6
    A, B = I.laplacian_2d(nx), I.mass_matrix_2d(nx)
    lp, lq = _pencil_lsp(oracle_mod, A, B)
    lam = pencil_eigs(nx)
    lo, hi = lam[0] - 0.5, lam[-1] * 1.01
    M, nv, seed = 30, 4, 5
    mu = oracle_mod.kpm_moments_gen(A, B, lp, lq, M, nv, seed, lo, hi)
    wb, Qb = np.linalg.eigh(B.to_dense())
    Bm12 = Qb @ np.diag(wb ** -0.5) @ Qb.T
    w, Z = np.linalg.eigh(Bm12 @ A.to_dense() @ Bm12)
    assert np.max(np.abs(w - lam)) <= 1e-12 * lam[-1]
    lh = (w - 0.5 * (hi + lo)) / (0.5 * (hi - lo))
    P = Z.T @ I.rademacher_block(A.n, nv, seed)
    want = np.array([np.mean(np.sum(P * P * np.cos(k * np.arccos(lh))[:, None], axis=0))
                     for k in range(M + 1)])
    assert abs(mu[0] - A.n) <= 1e-12 * A.n
    assert np.max(np.abs(mu - want)) <= 1e-11 * A.n


def test_kpm_gen_with_scaled_identity_is_standard_kpm(oracle_mod):
    # B = 2I: the pencil's eigenvalues are lambda(A)/2, q(B) v = v / sqrt 2 and B u = sqrt 2 v, so
    # the moments on [lmin/2, lmax/2] are the standard ones on [lmin, lmax]
    A = I.anderson_3d(6, 3.0, 1)
    n = A.n
    B2 = I.CSR(n, np.arange(n + 1), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    lp, lq = oracle_mod.lspol(1.5, 2.5, 1e-13), oracle_mod.lspol_isqrt(1.5, 2.5, 1e-13)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    mg = oracle_mod.kpm_moments_gen(A, B2, lp, lq, 40, 3, 7, lo / 2, hi / 2)
    ms = oracle_mod.kpm_moments(A, 40, 3, 7, lo, hi)
    assert np.max(np.abs(mg - ms)) <= 1e-12 * n


def test_kpm_gen_statistics_against_closed_form_trace(oracle_mod):
    # E[mu_k] = sum_ij T_k(lambda_hat_ij) over the pencil's closed-form eigenvalues; the
    # stochastic error is below 6 sqrt(2 ||T_k||_F^2 / nvec)
    nx, M, nv = 30, 40, 20
    A, B = I.laplacian_2d(nx), I.mass_matrix_2d(nx)
    lp, lq = _pencil_lsp(oracle_mod, A, B)
    lam = pencil_eigs(nx)
    lo, hi = 0.0, lam[-1] * 1.01
    mu = oracle_mod.kpm_moments_gen(A, B, lp, lq, M, nv, 0, lo, hi)
    lh = (lam - 0.5 * (hi + lo)) / (0.5 * (hi - lo))
    for k in range(M + 1):
        tk = np.cos(k * np.arccos(lh))
        sig = np.sqrt(2.0 * np.sum(tk * tk) / nv)
        assert abs(mu[k] - tk.sum()) <= 6 * sig + 1e-9


@pytest.mark.parametrize("a,b,m", [(2.0, 3.0, 40), (40.0, 42.0, 30)])
def test_cheblantr_gen_restarts_against_closed_form(oracle_mod, a, b, m):
    # thick restart with locking on the pencil, with a basis small enough to need several cycles:
    # exact count and eigenvalues, residuals, B-orthonormal eigenvectors
    nx = 20
    A, B = I.laplacian_2d(nx), I.mass_matrix_2d(nx)
    lam = pencil_eigs(nx)
    lp, _ = _pencil_lsp(oracle_mod, A, B)
    lo, hi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    ex = lam[(lam >= a) & (lam <= b)]
    r = oracle_mod.cheblantr_gen(A, B, lp, a, b, pol, m=m)
    assert r["status"] == 0 and r["nev"] == len(ex) and r["nrestart"] >= 3
    assert np.all(np.abs(r["lam"] - ex) <= 1e-9 * np.maximum(1.0, ex))
    X, Ad, Bd = r["Y"], A.to_dense(), B.to_dense()
    assert np.max(np.linalg.norm(Ad @ X - (Bd @ X) * r["lam"], axis=0)) <= 1e-8 * lp["bmax"] * hi
    assert np.max(np.abs(X.T @ Bd @ X - np.eye(len(ex)))) <= 1e-10


def test_cheblantr_gen_matches_dense_generalized_eigensolver(oracle_mod):
    # a pencil whose matrices do not commute: Anderson A and B = 0.4 I + 0.05 L (3-D Laplacian),
    # against scipy's dense generalized eigensolver
    import scipy.linalg as sl
    nx = 6
    A = I.anderson_3d(nx, 3.0, 0)
    L = I.laplacian_3d(nx)
    n = A.n
    Bd = 0.4 * np.eye(n) + 0.05 * L.to_dense()
    rows, cols = np.nonzero(Bd)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    B = I.CSR(n, rp, cols.astype(np.int32), Bd[rows, cols])
    w = sl.eigh(A.to_dense(), Bd, eigvals_only=True)
    lp = oracle_mod.lspol(0.39, 1.01, 1e-13)
    lo, hi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    assert lo <= w[0] + 1e-12 * abs(w[-1]) and hi >= w[-1] - 1e-9 * abs(w[-1])
    for a, b in [(2.0, 4.0), (8.0, 9.0)]:
        ex = w[(w >= a) & (w <= b)]
        pol = oracle_mod.filter_build(a, b, lo, hi)
        r = oracle_mod.cheblantr_gen(A, B, lp, a, b, pol, m=max(2 * len(ex), 40))
        assert r["status"] == 0 and r["nev"] == len(ex)
        assert np.max(np.abs(r["lam"] - ex)) <= 1e-9 * max(1.0, np.abs(ex).max())
        rn = oracle_mod.cheblannr_gen(A, B, lp, a, b, pol, m=max(6 * len(ex), 200))
        assert rn["nev"] == len(ex) and np.max(np.abs(rn["lam"] - ex)) <= 1e-9 * max(1.0, np.abs(ex).max())


def test_cheblantr_unreachable_tolerance_locks_nothing_unconverged(oracle_mod):
    # a tolerance at the residual floor is met by every pair (1e-15 relative), one below it
    # (1e-16) by none: restarts then keep finding candidates that do not lock, which takes the
    # stagnation refinement; a refined pair is kept only if it meets tol, so the run ends with
    # EVSL_ERR_NOCONV and returns nothing it has not converged
    A = I.laplacian_2d(20)
    e = lap_eigs(2, 20)
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(1.0, 1.4, lo, hi)
    r = oracle_mod.cheblantr(A, 1.0, 1.4, pol, m=40, maxit=600, tol=1e-15)
    assert r["status"] == 0 and r["nev"] == count_in(e, 1.0, 1.4) and np.all(r["res"] <= 1e-15)
    r = oracle_mod.cheblantr(A, 1.0, 1.4, pol, m=40, maxit=600, tol=1e-16)
    assert r["status"] == -4 and r["nrestart"] >= 3
    assert np.all(r["res"] <= 1e-16)


def test_empty_slices_run_the_minimum_empty_length(oracle_mod):
    # empty-cycle rule: a test with no Ritz value >= bar counts as stable only after a previous
    # test of the cycle had none either and the cycle ran max(2 ncycle, m/4) steps, so a slice
    # holding no eigenvalue ends only after max(2 ncycle, m/4) = 50 steps
    # (m = 200) in which no Ritz value reached bar: one such run for the non-restart solvers,
    # two candidate-free cycles for thick restart; standard and generalized solvers alike
    A, B = I.laplacian_2d(20), I.mass_matrix_2d(20)
    e, lam = lap_eigs(2, 20), pencil_eigs(20)

    def gap_slice(ev):
        d = np.unique(np.round(ev, 10))
        g = np.diff(d)
        i = int(np.argmax(g[5:-5])) + 5
        return d[i] + 0.25 * g[i], d[i + 1] - 0.25 * g[i]

    a, b = gap_slice(e)
    assert count_in(e, a, b) == 0
    lo, hi = oracle_mod.bounds(A, 80, 0)
    pol = oracle_mod.filter_build(a, b, lo, hi)
    r = oracle_mod.cheblannr(A, a, b, pol, m=200)
    assert r["status"] == 0 and r["nev"] == 0 and r["niter"] == 50
    r = oracle_mod.cheblantr(A, a, b, pol, m=200)
    assert r["status"] == 0 and r["nev"] == 0 and r["niter"] == 100 and r["nrestart"] == 2
    lp, _ = _pencil_lsp(oracle_mod, A, B)
    ga, gb = gap_slice(lam)
    assert np.count_nonzero((lam >= ga) & (lam <= gb)) == 0
    glo, ghi = oracle_mod.bounds_gen(A, B, lp, 80, 0)
    gpol = oracle_mod.filter_build(ga, gb, glo, ghi)
    r = oracle_mod.cheblannr_gen(A, B, lp, ga, gb, gpol, m=200)
    assert r["status"] == 0 and r["nev"] == 0 and r["niter"] == 50
    r = oracle_mod.cheblantr_gen(A, B, lp, ga, gb, gpol, m=200)
    assert r["status"] == 0 and r["nev"] == 0 and r["niter"] == 100 and r["nrestart"] == 2


def _inv_sqrt(M):
    w, Q = np.linalg.eigh(M)
    return Q @ np.diag(w ** -0.5) @ Q.T


def _anderson_pencil(nx):
    # Anderson A (W = 3) with B = 0.4 I + 0.05 L (3-D Laplacian): matrices that do not commute
    A = I.anderson_3d(nx, 3.0, 0)
    n = A.n
    Bd = 0.4 * np.eye(n) + 0.05 * I.laplacian_3d(nx).to_dense()
    rows, cols = np.nonzero(Bd)
    rp = np.zeros(n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(np.bincount(rows, minlength=n))
    return A, I.CSR(n, rp, cols.astype(np.int32), Bd[rows, cols]), Bd


def test_landos_gen_quadrature_is_exact_to_degree_2m_minus_1(oracle_mod):
    # m B-Lanczos steps give the m-point Gauss quadrature of v^T f(S) v, S = B^{-1/2} A B^{-1/2}:
    # sum_j tau_j theta_j^p = v^T S^p v for p <= 2m - 1 (v the normalised seeded start vector)
    A, B = I.laplacian_2d(6), I.mass_matrix_2d(6)
    lp, lq = _pencil_lsp(oracle_mod, A, B)
    Bm = _inv_sqrt(B.to_dense())
    S = Bm @ A.to_dense() @ Bm
    smax = np.linalg.eigvalsh(S).max()
    m, nvec = 6, 3
    d = oracle_mod.landos_gen(A, B, lp, lq, m, nvec, 7)
    assert list(d["mused"]) == [m] * nvec
    for l in range(nvec):
        v = I.start_vector(A.n, 7, I.STREAM_LANDOS, l)
        v /= np.linalg.norm(v)
        th, tau = d["nodes"][l, :m], d["weights"][l, :m]
        x = v.copy()
        for p in range(2 * m):
            assert abs(np.sum(tau * th ** p) - v @ x) <= 1e-10 * smax ** p
            x = S @ x


def test_landos_gen_full_run_is_the_exact_spectral_measure(oracle_mod):
    # a full-length run on a pencil with distinct eigenvalues: the nodes are the pencil's
    # eigenvalues and the weights (v . y_j)^2, y_j the eigenvectors of S
    A, B, Bd = _anderson_pencil(6)
    lp, lq = oracle_mod.lspol(0.39, 1.01, 1e-13), oracle_mod.lspol_isqrt(0.39, 1.01, 1e-13)
    Bm = _inv_sqrt(Bd)
    w, Y = np.linalg.eigh(Bm @ A.to_dense() @ Bm)
    d = oracle_mod.landos_gen(A, B, lp, lq, A.n, 1, 3)
    k = int(d["mused"][0])
    assert k == A.n
    assert np.max(np.abs(np.sort(d["nodes"][0, :k]) - w)) <= 1e-10 * np.abs(w).max()
    v = I.start_vector(A.n, 3, I.STREAM_LANDOS, 0)
    v /= np.linalg.norm(v)
    order = np.argsort(d["nodes"][0, :k])
    assert np.max(np.abs(d["weights"][0, :k][order] - (Y.T @ v) ** 2)) <= 1e-10


def test_landos_gen_with_scaled_identity_is_the_standard_density(oracle_mod):
    # B = 2I: the pencil's eigenvalues are lambda(A)/2 and the start vectors are the same, so the
    # nodes are the standard run's halved and the weights are equal
    A = I.anderson_3d(6, 3.0, 1)
    n = A.n
    B2 = I.CSR(n, np.arange(n + 1), np.arange(n, dtype=np.int32), np.full(n, 2.0))
    lp, lq = oracle_mod.lspol(1.5, 2.5, 1e-13), oracle_mod.lspol_isqrt(1.5, 2.5, 1e-13)
    dg = oracle_mod.landos_gen(A, B2, lp, lq, 30, 3, 5)
    ds = oracle_mod.landos(A, 30, 3, 5)
    assert np.array_equal(dg["mused"], ds["mused"])
    assert np.max(np.abs(2.0 * dg["nodes"] - ds["nodes"])) <= 1e-12 * np.abs(ds["nodes"]).max()
    assert np.max(np.abs(dg["weights"] - ds["weights"])) <= 1e-12


def test_landos_gen_count_tracks_the_pencil_closed_form(oracle_mod):
    # the cumulative quadrature count of the 20^2 pencil estimates its closed-form counts
    # (statistical: 30 vectors of 40 steps); the count above the spectrum is n
    A, B = I.laplacian_2d(20), I.mass_matrix_2d(20)
    lp, lq = _pencil_lsp(oracle_mod, A, B)
    lam = pencil_eigs(20)
    d = oracle_mod.landos_gen(A, B, lp, lq, 40, 30, 1)
    assert abs(oracle_mod.landos_count(d, A.n, 1.1 * lam[-1]) - A.n) <= 1e-9 * A.n
    for t in (5.0, 15.0, 30.0, 50.0, 65.0):
        assert abs(oracle_mod.landos_count(d, A.n, t) - np.count_nonzero(lam <= t)) <= 0.03 * A.n
