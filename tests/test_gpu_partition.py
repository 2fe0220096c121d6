"""The partition layer's GPU steps on one GPU: per-probe KPM sums against the oracle's, their
independence of how the probes are split (bitwise), and the whole layer with one rank."""
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


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-5)])
def test_probe_moments_match_oracle_and_any_split(nat, oracle_mod, prec, tol):
    A = I.anderson_3d(13, 4.0, 2)                   # n = 2197: a ragged last slice
    M, nv = 40, 9
    with nat.Context(0) as ctx:
        ctx.set_csr(A)
        lo, hi = oracle_mod.bounds(A, 60, 0)
        full = ctx.kpm_probe_moments(M, 0, nv, 5, lo, hi, prec=prec)
        parts = [ctx.kpm_probe_moments(M, f, c, 5, lo, hi, prec=prec) for f, c in [(0, 4), (4, 1), (5, 4)]]
        mu = ctx.kpm_dos(M, nv, 5, lo, hi, prec=prec)
    # bitwise: a probe's sums do not depend on the probes it shares a block with
    assert np.array_equal(np.concatenate(parts), full)
    ref = oracle_mod.kpm_probe_moments(A, M, 0, nv, 5, lo, hi)
    assert np.all(full[:, 0] == A.n)
    assert np.max(np.abs(full - ref)) <= tol * A.n
    assert np.max(np.abs(full.mean(axis=0) - mu)) <= tol * A.n


def test_partition_layer_one_rank_on_the_gpu(nat):
    # the whole layer with one process: bounds, per-probe KPM, slicing, LPT, solves, gather
    from paper_1802_05215_gb300 import partition
    A = I.laplacian_2d(30)
    with nat.Context(0) as ctx:
        ctx.set_csr(A)
        be = partition.NativeBackend(ctx, A.n)
        plan, res = partition.solve_interval(be, 0.6, 1.4, 3, 60, 8, want_vectors=True)
        mu = ctx.kpm_dos(60, 8, 0, plan.lmin, plan.lmax)
    assert plan.owned == [[0, 1, 2]]
    assert np.max(np.abs(plan.mu - mu)) <= 1e-12 * A.n
    e = lap_eigs(2, 30)
    lam = np.sort(np.concatenate([r["lam"] for r in res]))
    ex = e[(e >= 0.6) & (e <= 1.4)]
    assert len(lam) == len(ex) and np.max(np.abs(lam - ex)) <= 1e-9 * ex.max()
    for r in res:
        assert r["status"] == 0 and r["Y"].shape == (r["nev"], A.n)
