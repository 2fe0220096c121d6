"""Serving of slice solves with continuous batching (requests = (matrix, interval) pairs).

A Server keeps every matrix it has seen resident on the GPU (one context per matrix, CSR
uploaded once, each context on its own CUDA stream) and runs one continuous batch per matrix in
a worker thread of its own.  Admission is decided against ONE GPU-wide HBM budget shared by all
the matrices' contexts (evsl_set_device_budget): a request joins its matrix's batch as soon as
the device has room for its Lanczos bases and step workspaces.  All admitted jobs of a matrix
advance together (one multi-slice filter pass per degree per step), a job leaves the batch the
step it finishes, and the batches of different matrices run concurrently on their own streams
(the library's calls release the interpreter lock, so the workers' kernels overlap on the
device).  A request that cannot fit even when no job is running anywhere is refused with
EVSL_ERR_NOMEM in its outcome instead of waiting forever.  The plain mode runs the same
requests one at a time in arrival order with the FP64 filter, for comparison.

Every request is one slice: its filter is built for [a, b] on the matrix's spectral bounds, and
its Krylov dimension comes from the estimated count in [a, b].
"""
from __future__ import annotations

import dataclasses
import threading
import time

import numpy as np

from . import inputs, native


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float          # seconds after the start of the run
    matrix: str             # key into the server's matrix table
    a: float
    b: float
    est: float              # estimated eigenvalue count (DOS)
    right_closed: bool = True


@dataclasses.dataclass
class Outcome:
    rid: int
    arrival: float
    start: float
    finish: float
    nev: int
    res_max: float
    lam: np.ndarray
    status: int = 0
    Y: np.ndarray | None = None   # eigenvectors (rows), kept when the run asks for them

    @property
    def latency(self):
        return self.finish - self.arrival


def krylov_dim(est: float) -> int:
    return int(max(2 * est + 40, 100))


class ResidentMatrix:
    def __init__(self, key: str, A: inputs.CSR, device: int, bounds_steps=80):
        self.key = key
        self.A = A
        self.ctx = native.Context(device)
        self.ctx.set_csr(A)
        self.lmin, self.lmax = self.ctx.bounds(bounds_steps, 0)
        self.batch = None

    def filter(self, a, b):
        return native.cheb_filter_build(a, b, self.lmin, self.lmax)

    def close(self):
        if self.batch:
            self.batch.close()
        self.ctx.close()


class Server:
    """Continuous-batching server over resident matrices (one GPU, one HBM budget)."""

    def __init__(self, matrices: dict, device: int = 0, hbm_budget: int = 0,
                 prec=native.FP32, tol=1e-8):
        self.device = device
        self.mats = {k: ResidentMatrix(k, A, device) for k, A in matrices.items()}
        self.hbm_budget = hbm_budget
        self.prec = prec
        self.tol = tol

    def close(self):
        for m in self.mats.values():
            m.close()

    def run(self, requests: list[Request], batched: bool = True, prec=None,
            keep_vectors: bool = False) -> list[Outcome]:
        """Serve the requests against the wall clock; returns one outcome per request, in the
        order given.  prec: filter precision of the batched mode (default: the server's).
        keep_vectors: store each result's eigenvectors (host rows) in its outcome."""
        prec = self.prec if prec is None else prec
        pending = sorted(requests, key=lambda r: r.arrival)
        out: dict[int, Outcome] = {}
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731

        def outcome(r, start, res):
            nev = res["nev"]
            return Outcome(r.rid, r.arrival, start, now(), nev,
                           float(res["res"].max()) if nev else 0.0, res["lam"], res["status"],
                           np.array(res["Y"][:nev]) if keep_vectors else None)

        if not batched:
            for r in pending:
                while now() < r.arrival:
                    time.sleep(min(0.001, r.arrival - now()))
                M = self.mats[r.matrix]
                f = M.filter(r.a, r.b)
                st = now()
                res = M.ctx.chebLanTr(r.a, r.b, f, m=krylov_dim(r.est), tol=self.tol,
                                      prec=native.FP64, right_closed=r.right_closed,
                                      allow_partial=True)
                out[r.rid] = outcome(r, st, res)
            return [out[r.rid] for r in requests]

        native.set_device_budget(self.device, self.hbm_budget)
        lock = threading.Condition()
        queues: dict[str, list[Request]] = {k: [] for k in self.mats}
        active = {k: 0 for k in self.mats}        # admitted, unfinished jobs per matrix
        adding = [0]                               # batch.add calls in progress (all workers)
        remaining = [len(requests)]
        errors: list[BaseException] = []
        for M in self.mats.values():
            M.batch = native.Batch(M.ctx, tol=self.tol, prec=prec)

        def worker(key: str):
            M = self.mats[key]
            started: dict[int, float] = {}
            try:
                while True:
                    with lock:
                        while not queues[key] and active[key] == 0 and remaining[0] > 0 and not errors:
                            lock.wait(0.05)
                        if remaining[0] == 0 or errors:
                            return
                        admit = list(queues[key])
                    # admission in arrival order, as the device budget allows; a job counts as
                    # active from the moment its add starts, so that no other worker takes the
                    # device for idle while this one is allocating
                    for r in admit:
                        f = M.filter(r.a, r.b)
                        with lock:
                            adding[0] += 1
                        try:
                            M.batch.add(r.a, r.b, f, krylov_dim(r.est), right_closed=r.right_closed, tag=r.rid)
                        except native.EvslError as e:
                            with lock:
                                adding[0] -= 1
                            if e.code != -2:
                                raise
                            with lock:
                                idle = sum(active.values()) == 0 and adding[0] == 0 and not M.batch.active
                                if idle:
                                    # nothing runs or is being admitted anywhere and it still does
                                    # not fit: it never will
                                    out[r.rid] = Outcome(r.rid, r.arrival, now(), now(), 0, 0.0,
                                                         np.zeros(0), -2, None)
                                    queues[key].remove(r)
                                    remaining[0] -= 1
                                    lock.notify_all()
                            break             # keep arrival order: later requests wait too
                        started[r.rid] = now()
                        with lock:
                            adding[0] -= 1
                            active[key] += 1
                            queues[key].remove(r)
                    if not M.batch.active:
                        with lock:                # queued work that does not fit yet: wait for
                            lock.wait(0.005)      # another matrix's jobs to free memory
                        continue
                    for job in M.batch.step():
                        rq = next(q for q in requests if q.rid == job.tag)
                        oc = outcome(rq, started[job.tag], job.result())
                        with lock:
                            out[job.tag] = oc
                            active[key] -= 1
                            remaining[0] -= 1
                            lock.notify_all()
            except BaseException as e:        # surface the failure in the dispatcher
                with lock:
                    errors.append(e)
                    lock.notify_all()

        threads = [threading.Thread(target=worker, args=(k,), daemon=True) for k in self.mats]
        for t in threads:
            t.start()
        try:
            i = 0
            while i < len(pending):
                wait = pending[i].arrival - now()
                if wait > 0:
                    time.sleep(min(wait, 0.002))
                    continue
                with lock:
                    while i < len(pending) and pending[i].arrival <= now():
                        queues[pending[i].matrix].append(pending[i])
                        i += 1
                    lock.notify_all()
                    if errors:
                        break
        finally:
            for t in threads:
                t.join()
            for M in self.mats.values():
                M.batch.close()
                M.batch = None
            native.set_device_budget(self.device, 0)
        if errors:
            raise errors[0]
        return [out[r.rid] for r in requests]


def make_requests(server_mats: dict, spectra: dict, nreq: int, rate: float, seed: int = 0,
                  count_range=(20, 120)) -> list[Request]:
    """Poisson arrivals (rate per second); each request picks a matrix and an interval holding
    about a uniformly drawn number of eigenvalues of the known spectrum (closed form for the
    Laplacians, or a reference list).  The ends are placed midway between two distinct
    eigenvalues (a drawn end inside a cluster of equal eigenvalues -- equal to 1e-10 of the
    spectral radius, as closed-form multiple eigenvalues differ in their last bits -- moves
    outwards to the cluster's edge), so the exact count, stored as the request's estimate, does
    not depend on rounding."""
    rng = np.random.default_rng(seed)
    keys = sorted(server_mats)
    t = 0.0
    reqs = []
    for rid in range(nreq):
        t += rng.exponential(1.0 / rate)
        key = keys[rng.integers(len(keys))]
        ev = np.sort(np.asarray(spectra[key], dtype=float))
        tie = 1e-10 * np.abs(ev).max()
        c = int(rng.integers(count_range[0], count_range[1] + 1))
        i0 = int(rng.integers(1, len(ev) - c - 1))
        e = i0 + c
        while i0 > 1 and ev[i0] - ev[i0 - 1] <= tie:
            i0 -= 1
        while e < len(ev) - 1 and ev[e] - ev[e - 1] <= tie:
            e += 1
        if ev[i0] - ev[i0 - 1] <= tie or ev[e] - ev[e - 1] <= tie:
            raise ValueError(f"no distinct eigenvalues to cut between for matrix {key}")
        a = 0.5 * (ev[i0 - 1] + ev[i0])
        b = 0.5 * (ev[e - 1] + ev[e])
        exact = int(np.count_nonzero((ev >= a) & (ev <= b)))
        reqs.append(Request(rid, t, key, float(a), float(b), float(exact)))
    return reqs


def percentile(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else float("nan")


def summarize(outcomes: list[Outcome], wall: float) -> dict:
    lat = [o.latency for o in outcomes]
    neig = sum(o.nev for o in outcomes)
    return {"eigenpairs": neig, "eigenpairs_per_s": neig / wall if wall > 0 else float("nan"),
            "p50_latency_s": percentile(lat, 50), "p99_latency_s": percentile(lat, 99),
            "requests": len(outcomes), "wall_s": wall,
            "max_residual": max((o.res_max for o in outcomes), default=0.0)}


__all__ = ["Request", "Outcome", "Server", "make_requests", "summarize", "krylov_dim"]
