"""Multi-rank slice sharding on CPU: world_size-2 gloo process group, each rank solving its own
slices (the oracle stands in for the device), results gathered on the host."""
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


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist

    import oracle
    from paper_1802_05215_gb300 import inputs
    from paper_1802_05215_gb300.schedule import assign_slices, slice_costs
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    A = inputs.laplacian_2d(24)
    xi, eta, ns = 0.5, 1.5, 4
    lo, hi = oracle.bounds(A, 60, 0)
    mu = oracle.kpm_moments(A, 60, 8, 0, lo, hi)
    sli, est = oracle.slicer(mu, lo, hi, xi, eta, ns)
    pols = [oracle.filter_build(sli[i], sli[i + 1], lo, hi) for i in range(ns)]
    own = assign_slices(slice_costs(est, [p["deg"] for p in pols]), world)[rank]
    lams = []
    for s in own:
        m = int(max(2 * est[s] + 40, 100))
        r = oracle.cheblantr(A, sli[s], sli[s + 1], pols[s], m=m, right_closed=(s == ns - 1))
        assert r["status"] == 0
        lams.append(r["lam"])
    mine = np.concatenate(lams) if lams else np.zeros(0)
    gathered = [None] * world
    dist.all_gather_object(gathered, (own, mine.tolist()))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_slice_sharding_matches_closed_form():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    owned = sorted(sum([g[0] for g in gathered], []))
    assert owned == [0, 1, 2, 3]
    lam = np.sort(np.concatenate([np.array(g[1]) for g in gathered]))
    e = lap_eigs(2, 24)
    ex = e[(e >= 0.5) & (e <= 1.5)]
    assert len(lam) == len(ex)
    assert np.max(np.abs(lam - ex)) < 1e-9


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
