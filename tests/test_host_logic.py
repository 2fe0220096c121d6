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


class _FakeNative:
    """Stand-in for the binding, to run the server's admission and worker logic on the CPU: a
    job's device bytes are n * (cap + m + 1) * 8 (its Lanczos bases), charged against one
    device-wide budget shared by all contexts; a job finishes after `est` steps of its batch."""

    FP32, FP64 = 1, 0
    EvslError = None

    def __init__(self):
        from paper_1802_05215_gb300 import native
        self.EvslError = native.EvslError
        self.budget, self.used = 0, 0
        self.slow_n = 0                     # contexts of this order take 0.1 s in batch.add
        self.steps = {}
        self.overlap = 0                    # most batches stepping at once
        self._stepping = 0
        import threading
        self._mu = threading.Lock()
        fake = self

        class Ctx:
            def __init__(self, device=0, budget=0):
                self.n = 0

            def set_csr(self, A):
                self.n = A.n

            def bounds(self, steps, seed):
                return 0.0, 8.0

            def close(self):
                pass

        class Job:
            def __init__(self, tag, need, left):
                self.tag, self.need, self.left = tag, need, left

            def result(self):
                return dict(status=0, nev=3, lam=np.arange(3.0), res=np.full(3, 1e-10),
                            Y=np.zeros((3, 4)))

        class Batch:
            def __init__(self, ctx, tol=1e-8, prec=0):
                self.ctx, self.active = ctx, []

            def add(self, a, b, filt, m, cap=None, right_closed=True, tag=None):
                need = self.ctx.n * ((cap or m + 64) + m + 1) * 8
                with fake._mu:
                    if fake.budget and fake.used + need > fake.budget:
                        raise fake.EvslError(-2, "no room")
                    fake.used += need
                if fake.slow_n and self.ctx.n == fake.slow_n:
                    import time
                    time.sleep(0.1)           # the memory is taken, the call has not returned
                job = Job(tag, need, max(1, int(b - a)))
                self.active.append(job)
                return job

            def step(self):
                import time
                with fake._mu:
                    fake._stepping += 1
                    fake.overlap = max(fake.overlap, fake._stepping)
                time.sleep(0.002)
                done = []
                for j in self.active:
                    j.left -= 1
                    if j.left == 0:
                        done.append(j)
                self.active = [j for j in self.active if j.left > 0]
                with fake._mu:
                    for j in done:
                        fake.used -= j.need
                    fake._stepping -= 1
                return done

            def close(self):
                pass

        self.Context, self.Batch = Ctx, Batch

    def set_device_budget(self, device, nbytes):
        self.budget = nbytes

    def cheb_filter_build(self, a, b, lo, hi):
        return None


def test_server_admission_refuses_what_never_fits_and_overlaps_matrices(monkeypatch):
    from paper_1802_05215_gb300 import inputs
    fake = _FakeNative()
    monkeypatch.setattr(serve, "native", fake)
    mats = {"p": inputs.laplacian_2d(10), "q": inputs.laplacian_2d(12)}
    srv = serve.Server(mats, hbm_budget=600_000)       # one "p" job (212 kB) and one "q" job (305 kB)
    # request b - a sets the fake job's step count; est sets its Krylov dimension (>= 100)
    big = serve.krylov_dim(5000)                     # bases far beyond the budget
    reqs = [serve.Request(0, 0.00, "p", 0.0, 20.0, 10.0),
            serve.Request(1, 0.00, "q", 0.0, 20.0, 10.0),
            serve.Request(2, 0.01, "p", 0.0, 5.0, 5000.0),   # can never be admitted
            serve.Request(3, 0.02, "q", 0.0, 3.0, 10.0),
            serve.Request(4, 0.02, "p", 0.0, 4.0, 10.0)]
    assert big > 100
    out = srv.run(reqs, batched=True)
    assert [o.rid for o in out] == [0, 1, 2, 3, 4]
    assert out[2].status == -2 and out[2].nev == 0
    assert all(o.status == 0 and o.nev == 3 for i, o in enumerate(out) if i != 2)
    assert fake.overlap == 2                         # the two matrices' batches stepped together
    assert fake.used == 0 and fake.budget == 0       # everything released, budget reset
    # request 4 waited behind the refused request 2 of the same matrix, never ahead of it
    assert out[4].start >= out[2].finish


def test_server_admission_waits_for_a_job_still_being_admitted(monkeypatch):
    # matrix q's job holds its memory while its add call is still running; a request of matrix
    # p that does not fit beside it arrives meanwhile.  Nothing counts as active yet, but the
    # request must wait (and run once q's job has finished), not be refused as never fitting.
    from paper_1802_05215_gb300 import inputs
    fake = _FakeNative()
    fake.slow_n = 144
    monkeypatch.setattr(serve, "native", fake)
    mats = {"p": inputs.laplacian_2d(10), "q": inputs.laplacian_2d(12)}
    srv = serve.Server(mats, hbm_budget=400_000)       # p job 212 kB, q job 305 kB: one at a time
    reqs = [serve.Request(0, 0.00, "q", 0.0, 5.0, 10.0),
            serve.Request(1, 0.02, "p", 0.0, 5.0, 10.0)]
    out = srv.run(reqs, batched=True)
    assert [o.status for o in out] == [0, 0] and [o.nev for o in out] == [3, 3]
    assert out[1].start >= out[0].finish - 0.01          # p admitted after q released its memory
    assert fake.used == 0
