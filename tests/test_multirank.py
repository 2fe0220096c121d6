"""Multi-rank slicing on CPU: world_size-2 gloo process groups running the partition layer
(probes split over ranks with a gather of per-probe rows, slice ends broadcast, LPT assignment,
results gathered on rank 0) with the oracle standing in for each rank's device."""
import os
import socket

import numpy as np

from closed_form import lap_eigs


def test_assign_slices_lpt():
    from paper_1802_05215_gb300.schedule import assign_slices, slice_costs
    costs = slice_costs([100, 100, 100, 100, 10], [50, 40, 30, 20, 5])
    own = assign_slices(costs, 2)
    assert sorted(sum(own, [])) == list(range(5))
    loads = [sum(costs[s] for s in o) for o in own]
    assert max(loads) - min(loads) <= max(costs)
    assert assign_slices(costs, 1) == [list(range(5))]
    assert assign_slices([1.0, 1.0], 4)[2:] == [[], []]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


class OracleBackend:
    """The partition layer's numerical steps by the CPU oracle (standing in for a GPU per rank)."""

    def __init__(self, A):
        import oracle
        self.o, self.A, self.n = oracle, A, A.n

    def bounds(self, steps, seed):
        return self.o.bounds(self.A, steps, seed)

    def kpm_probe_moments(self, degree, first, count, seed, lmin, lmax):
        return self.o.kpm_probe_moments(self.A, degree, first, count, seed, lmin, lmax)

    def slice_by_dos(self, mu, lmin, lmax, xi, eta, nslices):
        return self.o.slicer(mu, lmin, lmax, xi, eta, nslices)

    def filter(self, a, b, lmin, lmax):
        from types import SimpleNamespace
        pol = self.o.filter_build(a, b, lmin, lmax)
        return SimpleNamespace(deg=pol["deg"], pol=pol)

    def solve(self, a, b, filt, m, right_closed, tol, seed):
        r = self.o.cheblantr(self.A, a, b, filt.pol, m=m, tol=tol, seed=seed, right_closed=right_closed)
        return dict(r, Y=r["Y"].T)


CASE = dict(nx=24, xi=0.5, eta=1.5, ns=4, M=60, nvec=7, seed=0)


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    sys.path.insert(0, os.path.join(root, "tests"))
    import torch.distributed as dist

    from paper_1802_05215_gb300 import inputs, partition
    from test_multirank import CASE, OracleBackend
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = inputs.laplacian_2d(CASE["nx"])
    plan, results = partition.solve_interval(OracleBackend(A), CASE["xi"], CASE["eta"], CASE["ns"], CASE["M"],
                                             CASE["nvec"], CASE["seed"], want_vectors=True)
    out.put((rank, plan.mu, plan.owned, results))
    dist.barrier()
    dist.destroy_process_group()


def test_probe_share_covers_the_probes_once():
    from paper_1802_05215_gb300.partition import probe_share
    for nvec, world in [(7, 2), (40, 3), (3, 5), (64, 8)]:
        got = [probe_share(nvec, r, world) for r in range(world)]
        idx = [l for f, c in got for l in range(f, f + c)]
        assert idx == list(range(nvec))
        assert max(c for _, c in got) - min(c for _, c in got) <= 1


def test_two_rank_partition_moments_bitwise_and_eigenvalues_closed_form():
    # two gloo ranks: KPM probes split 4 + 3, one all-gather of per-probe rows, slice ends from
    # rank 0, LPT assignment, eigenpairs gathered on rank 0.  The moments equal, bit for bit,
    # the single-process oracle's and the partition layer's own one-rank run; the gathered
    # eigenvalues are the closed-form spectrum of [xi, eta], each slice's count exact.
    import torch.multiprocessing as mp

    import oracle
    from paper_1802_05215_gb300 import inputs, partition
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict((r, (mu, owned, res)) for r, mu, owned, res in (q.get(timeout=600) for _ in range(2)))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    A = inputs.laplacian_2d(CASE["nx"])
    lo, hi = oracle.bounds(A, 80, CASE["seed"])
    mu_ref = oracle.kpm_moments(A, CASE["M"], CASE["nvec"], CASE["seed"], lo, hi)
    single, single_res = partition.solve_interval(OracleBackend(A), CASE["xi"], CASE["eta"], CASE["ns"], CASE["M"],
                                                  CASE["nvec"], CASE["seed"])
    for r in (0, 1):
        assert np.array_equal(got[r][0], mu_ref)
        assert np.array_equal(got[r][0], single.mu)
    assert got[0][1] == got[1][1] and sorted(sum(got[0][1], [])) == list(range(CASE["ns"]))
    assert got[1][2] is None
    res = got[0][2]
    assert [r["slice"] for r in res] == list(range(CASE["ns"]))
    e = lap_eigs(2, CASE["nx"])
    for r in res:
        ex = e[(e >= r["a"]) & ((e <= r["b"]) if r["slice"] == CASE["ns"] - 1 else (e < r["b"]))]
        assert r["status"] == 0 and r["nev"] == len(ex)
        assert np.max(np.abs(np.sort(r["lam"]) - ex)) < 1e-9
        assert r["Y"].shape == (r["nev"], A.n)
    lam = np.sort(np.concatenate([r["lam"] for r in res]))
    ex = e[(e >= CASE["xi"]) & (e <= CASE["eta"])]
    assert len(lam) == len(ex) and np.max(np.abs(lam - ex)) < 1e-9
    # the same eigenvalues as the one-process run of the same layer
    assert np.array_equal(lam, np.sort(np.concatenate([r["lam"] for r in single_res])))


def _rate_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r found 10 (r + 1) eigenpairs in 1 + r seconds
    out.put((rank, bench.whole_job_rate(10.0 * (rank + 1), 1.0 + rank, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_bench_whole_job_rate_over_two_gloo_ranks():
    # the bench's N-rank value: all ranks' eigenpairs over the slowest rank's time, the same on
    # every rank; without a process group the rank's own numbers
    import torch.multiprocessing as mp

    import bench
    assert bench.whole_job_rate(5.0, 2.0, "cpu") == (5.0, 2.0, 2.5)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rate_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] == got[1] == (30.0, 2.0, 15.0)
