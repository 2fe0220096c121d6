"""Serving of slice solves with continuous batching (requests = (matrix, interval) pairs).

A Server keeps every matrix it has seen resident on the GPU (one context per matrix, CSR
uploaded once) and runs one continuous batch per matrix: a request is admitted into its
matrix's batch as soon as the HBM budget has room for its Lanczos bases, all admitted jobs of a
matrix advance together (one multi-slice filter pass per degree per step), and a job leaves the
batch the step it finishes.  The plain mode runs the same requests one at a time in arrival
order with the FP64 filter, for comparison.

Every request is one slice: its filter is built for [a, b] on the matrix's spectral bounds, and
its Krylov dimension comes from the KPM estimate of the count in [a, b].
"""
from __future__ import annotations

import dataclasses
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


@dataclasses.dataclass
class Outcome:
    rid: int
    arrival: float
    start: float
    finish: float
    nev: int
    res_max: float
    lam: np.ndarray

    @property
    def latency(self):
        return self.finish - self.arrival


def krylov_dim(est: float) -> int:
    return int(max(2 * est + 40, 100))


class ResidentMatrix:
    def __init__(self, key: str, A: inputs.CSR, device: int, budget: int, bounds_steps=80):
        self.key = key
        self.A = A
        self.ctx = native.Context(device, budget)
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
    """Continuous-batching server over resident matrices (one GPU)."""

    def __init__(self, matrices: dict, device: int = 0, hbm_budget_per_matrix: int = 0,
                 prec=native.FP32, tol=1e-8):
        self.mats = {k: ResidentMatrix(k, A, device, hbm_budget_per_matrix)
                     for k, A in matrices.items()}
        self.prec = prec
        self.tol = tol

    def close(self):
        for m in self.mats.values():
            m.close()

    def run(self, requests: list[Request], batched: bool = True, prec=None) -> list[Outcome]:
        """Serve the requests against the wall clock; returns one outcome per request.
        prec: filter precision of the batched mode (default: the server's)."""
        prec = self.prec if prec is None else prec
        pending = sorted(requests, key=lambda r: r.arrival)
        queue: list[Request] = []
        out: dict[int, Outcome] = {}
        started: dict[int, float] = {}
        t0 = time.perf_counter()
        now = lambda: time.perf_counter() - t0  # noqa: E731
        i = 0
        if not batched:
            for r in pending:
                while now() < r.arrival:
                    time.sleep(min(0.001, r.arrival - now()))
                M = self.mats[r.matrix]
                f = M.filter(r.a, r.b)
                st = now()
                res = M.ctx.chebLanTr(r.a, r.b, f, m=krylov_dim(r.est), tol=self.tol,
                                      prec=native.FP64, allow_partial=True)
                out[r.rid] = Outcome(r.rid, r.arrival, st, now(), res["nev"],
                                     float(res["res"].max()) if res["nev"] else 0.0, res["lam"])
            return [out[r.rid] for r in requests]
        for M in self.mats.values():
            M.batch = native.Batch(M.ctx, tol=self.tol, prec=prec)
        while len(out) < len(requests):
            t = now()
            while i < len(pending) and pending[i].arrival <= t:
                queue.append(pending[i])
                i += 1
            # admission in arrival order, as HBM allows (a refused job waits in the queue)
            still = []
            for r in queue:
                M = self.mats[r.matrix]
                try:
                    M.batch.add(r.a, r.b, M.filter(r.a, r.b), krylov_dim(r.est), tag=r.rid)
                    started[r.rid] = now()
                except native.EvslError as e:
                    if e.code != -2:
                        raise
                    still.append(r)
            queue = still
            busy = False
            for M in self.mats.values():
                if M.batch.active:
                    busy = True
                    for job in M.batch.step():
                        res = job.result()
                        rq = next(q for q in requests if q.rid == job.tag)
                        out[job.tag] = Outcome(job.tag, rq.arrival, started[job.tag], now(),
                                               res["nev"], float(res["res"].max()) if res["nev"] else 0.0,
                                               res["lam"])
            if not busy and i < len(pending):
                time.sleep(max(0.0, min(0.002, pending[i].arrival - now())))
        for M in self.mats.values():
            M.batch.close()
            M.batch = None
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
