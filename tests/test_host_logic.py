"""Host-side logic of the serving layer (no GPU): request generation, Krylov dimensions and the
latency/throughput summary."""
import numpy as np
import pytest

from closed_form import lap_eigs
from paper_1802_05215_gb300 import serve


def test_krylov_dim_grows_with_the_estimate_and_has_a_floor():
    dims = [serve.krylov_dim(e) for e in (0, 10, 30, 31, 100, 1000)]
    assert dims[0] == 100 and dims == sorted(dims) and serve.krylov_dim(1000) == 2040


def test_make_requests_cut_between_distinct_eigenvalues():
    # Laplacian spectra have multiple eigenvalues: every request's ends must sit strictly
    # between two distinct eigenvalues, and its stored estimate is the exact count
    spectra = {"lap2d_30": lap_eigs(2, 30), "lap3d_12": lap_eigs(3, 12)}
    reqs = serve.make_requests(spectra, spectra, nreq=60, rate=4.0, seed=3)
    assert [r.rid for r in reqs] == list(range(60))
    assert all(b.arrival > a.arrival for a, b in zip(reqs, reqs[1:]))
    for r in reqs:
        ev = spectra[r.matrix]
        gap = 1e-11 * np.abs(ev).max()
        assert np.min(np.abs(ev - r.a)) > gap and np.min(np.abs(ev - r.b)) > gap
        assert r.est == np.count_nonzero((ev >= r.a) & (ev <= r.b)) >= 20
    again = serve.make_requests(spectra, spectra, nreq=60, rate=4.0, seed=3)
    assert [(r.matrix, r.a, r.b, r.arrival) for r in again] == [(r.matrix, r.a, r.b, r.arrival) for r in reqs]


def test_make_requests_refuses_a_spectrum_without_gaps():
    with pytest.raises(ValueError):
        serve.make_requests({"flat": None}, {"flat": np.ones(400)}, nreq=1, rate=1.0)


def test_summarize_latency_percentiles_and_throughput():
    outs = [serve.Outcome(rid=i, arrival=0.1 * i, start=0.1 * i, finish=0.1 * i + 1.0 + i, nev=10 + i,
                          res_max=1e-10 * (i + 1), lam=np.zeros(0)) for i in range(20)]
    s = serve.summarize(outs, wall=25.0)
    lat = np.array([1.0 + i for i in range(20)])
    assert s["eigenpairs"] == sum(10 + i for i in range(20)) and s["requests"] == 20
    assert abs(s["eigenpairs_per_s"] - s["eigenpairs"] / 25.0) < 1e-12
    assert abs(s["p50_latency_s"] - np.percentile(lat, 50)) < 1e-12
    assert abs(s["p99_latency_s"] - np.percentile(lat, 99)) < 1e-12
    assert s["max_residual"] == pytest.approx(2e-9)
    empty = serve.summarize([], wall=1.0)
    assert empty["eigenpairs"] == 0 and np.isnan(empty["p50_latency_s"])
