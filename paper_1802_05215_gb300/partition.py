"""Spectrum slicing spread over processes (one GPU each).

Sec. 2.6 names the first level of parallelism: the slices of [xi, eta] are independent, so
groups of slices go to separate processes.  Sec. 2.1's density estimate that places the slices is
an average over probe vectors, so its probes can be spread over the processes too.  For P
processes (ranks 0 .. P-1), each holding a replica of the matrix:

 1. spectral bounds on rank 0, broadcast;
 2. KPM: rank r computes the per-probe sums of its contiguous share of the probes
    (evsl_kpm_probe_moments); the rows of all ranks are gathered and added in probe order, so
    every rank holds the same moments, bitwise equal to those of one process (any split);
 3. DOS slicing on rank 0; slice ends and count estimates broadcast;
 4. slices assigned to ranks by longest processing time on estimated count x filter degree
    (schedule.assign_slices), computed identically on every rank;
 5. each rank solves its own slices;
 6. results (eigenvalues, residuals, status; eigenvectors on request) gathered to rank 0,
    ordered by slice.

The collectives are torch.distributed object collectives on the default process group (gloo
on CPU, NCCL between GPUs): a few kilobytes per call and no exchange on the data path.  Without
an initialised process group (or with one rank) they are the identity.

A backend supplies the numerical steps; `NativeBackend` runs them on this process's GPU through
the C ABI.  Anything with the same methods can stand in (the CPU tests use the FP64 oracle).
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .schedule import assign_slices, slice_costs


# ------------------------------------------------------------------------------ collectives
def world_info() -> tuple[int, int]:
    """(rank, world size) of the default process group, (0, 1) without one."""
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            return dist.get_rank(), dist.get_world_size()
    except ImportError:
        pass
    return 0, 1


def broadcast(obj, src: int = 0):
    rank, world = world_info()
    if world == 1:
        return obj
    import torch.distributed as dist
    box = [obj if rank == src else None]
    dist.broadcast_object_list(box, src=src)
    return box[0]


def all_gather(obj) -> list:
    rank, world = world_info()
    if world == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, obj)
    return out


def gather(obj, dst: int = 0):
    """List of every rank's obj on rank dst (rank order), None elsewhere."""
    rank, world = world_info()
    if world == 1:
        return [obj]
    import torch.distributed as dist
    out = [None] * world if rank == dst else None
    dist.gather_object(obj, out, dst=dst)
    return out


# ------------------------------------------------------------------------------ the steps
def probe_share(nvec: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous share (first probe, count) of rank among nvec probes: the first nvec % world
    ranks take one probe more."""
    base, extra = divmod(nvec, world)
    count = base + (1 if rank < extra else 0)
    first = rank * base + min(rank, extra)
    return first, count


def sharded_moments(backend, degree: int, nvec: int, seed: int, lmin: float, lmax: float) -> np.ndarray:
    """KPM moments mu_0..degree of nvec probes split over the ranks: every rank computes its
    share's per-probe sums, the rows are gathered, and all ranks add them in probe order
    (mu_k = (1/nvec) sum_l v_l^T T_k(Ahat) v_l)."""
    rank, world = world_info()
    first, count = probe_share(nvec, rank, world)
    rows = (backend.kpm_probe_moments(degree, first, count, seed, lmin, lmax) if count
            else np.zeros((0, degree + 1)))
    parts = all_gather((first, np.asarray(rows, dtype=np.float64)))
    table = np.concatenate([p[1] for p in sorted(parts, key=lambda p: p[0])], axis=0)
    if table.shape != (nvec, degree + 1):
        raise RuntimeError(f"gathered probe table has shape {table.shape}, expected {(nvec, degree + 1)}")
    mu = np.zeros(degree + 1)
    for row in table:
        mu += row
    return mu / nvec


@dataclasses.dataclass
class Plan:
    lmin: float
    lmax: float
    mu: np.ndarray
    sli: np.ndarray          # slice ends t_0 .. t_ns
    est: np.ndarray          # estimated eigenvalue count per slice
    degrees: list            # filter degree per slice
    owned: list              # owned[r] = slices of rank r (increasing)

    def slice(self, s: int) -> tuple[float, float]:
        return float(self.sli[s]), float(self.sli[s + 1])


def plan(backend, xi: float, eta: float, nslices: int, kpm_degree: int, kpm_nvec: int, seed: int = 0,
         bounds_steps: int = 80) -> Plan:
    """Steps 1-4: bounds (rank 0), sharded KPM, slicing (rank 0), filters' degrees and the LPT
    assignment; every rank returns the same plan."""
    rank, world = world_info()
    lo, hi = broadcast(backend.bounds(bounds_steps, seed) if rank == 0 else None)
    mu = sharded_moments(backend, kpm_degree, kpm_nvec, seed, lo, hi)
    sl = broadcast(backend.slice_by_dos(mu, lo, hi, xi, eta, nslices) if rank == 0 else None)
    sli, est = np.asarray(sl[0]), np.asarray(sl[1])
    degs = [int(backend.filter(sli[i], sli[i + 1], lo, hi).deg) for i in range(nslices)]
    owned = assign_slices(slice_costs(est, degs), world)
    return Plan(lo, hi, mu, sli, est, degs, owned)


def krylov_dim(est: float) -> int:
    """Krylov dimension from the slice's estimated count (memory grows with it)."""
    return int(max(2 * est + 40, 100))


def solve_own(backend, p: Plan, tol: float = 1e-8, seed: int = 0, want_vectors: bool = False) -> list[dict]:
    """Step 5: this rank's slices, one result dict per slice (slice index, ends, eigenvalues,
    residuals, status, statistics; eigenvectors as host rows when want_vectors)."""
    rank, _ = world_info()
    nslices = len(p.sli) - 1
    out = []
    for s in p.owned[rank]:
        a, b = p.slice(s)
        f = backend.filter(a, b, p.lmin, p.lmax)
        r = backend.solve(a, b, f, krylov_dim(p.est[s]), s == nslices - 1, tol, seed)
        rec = {"slice": s, "a": a, "b": b, "nev": int(r["nev"]), "lam": np.asarray(r["lam"]),
               "res": np.asarray(r["res"]), "status": int(r["status"])}
        if want_vectors:
            rec["Y"] = np.asarray(r["Y"])[: r["nev"]]
        out.append(rec)
    return out


def gather_results(local: list[dict], nslices: int):
    """Step 6: every rank's slice results on rank 0, in slice order (None on other ranks)."""
    allr = gather(local, dst=0)
    if allr is None:
        return None
    merged = sorted((r for part in allr for r in part), key=lambda r: r["slice"])
    if [r["slice"] for r in merged] != list(range(nslices)):
        raise RuntimeError("gathered slices do not cover the interval exactly once")
    return merged


def solve_interval(backend, xi: float, eta: float, nslices: int, kpm_degree: int, kpm_nvec: int, seed: int = 0,
                   tol: float = 1e-8, want_vectors: bool = False):
    """The whole sharded path.  Rank 0 returns (plan, results of all slices in slice order);
    the other ranks return (plan, None)."""
    p = plan(backend, xi, eta, nslices, kpm_degree, kpm_nvec, seed)
    mine = solve_own(backend, p, tol, seed, want_vectors)
    return p, gather_results(mine, nslices)


# ------------------------------------------------------------------------------ GPU backend
class NativeBackend:
    """The steps on this process's GPU through the C ABI (one context, matrix resident)."""

    def __init__(self, ctx, n: int):
        from . import native
        self.native = native
        self.ctx = ctx
        self.n = n

    def bounds(self, steps, seed):
        return self.ctx.bounds(steps, seed)

    def kpm_probe_moments(self, degree, first, count, seed, lmin, lmax):
        return self.ctx.kpm_probe_moments(degree, first, count, seed, lmin, lmax)

    def slice_by_dos(self, mu, lmin, lmax, xi, eta, nslices):
        return self.native.slice_by_dos(mu, self.n, lmin, lmax, xi, eta, nslices)

    def filter(self, a, b, lmin, lmax):
        return self.native.cheb_filter_build(a, b, lmin, lmax)

    def solve(self, a, b, filt, m, right_closed, tol, seed, Y=None, cap=None):
        return self.ctx.chebLanTr(a, b, filt, m=m, tol=tol, seed=seed, right_closed=right_closed,
                                  cap=cap or m, Y=Y)


__all__ = ["world_info", "broadcast", "all_gather", "gather", "probe_share", "sharded_moments", "Plan", "plan",
           "krylov_dim", "solve_own", "gather_results", "solve_interval", "NativeBackend"]
