"""The multi-rank path of the benchmark, on CPU with two gloo ranks: the
path is partitioned by replica (each rank advances its own seeded system,
no data-path collective), the job's time is the slowest rank's, and the
whole-job rate counts every rank's particles."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    c = bench.workload("lj4096", seed=rank)
    ms_local = 10.0 * (rank + 1)                   # rank 1 is the slower one
    ms_max = bench.max_over_ranks(ms_local, dist, "cpu")
    rate = bench.whole_job_rate(c.N, 100, 3, world, ms_max)
    out.put((rank, c.N, float(c.r[:, :3].sum()), ms_max, rate))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_time_by_the_slowest_and_count_every_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, n0, s0, m0, v0), (r1, n1, s1, m1, v1) = res
    assert (r0, r1) == (0, 1)
    assert n0 == n1 == 4096                        # weak scaling: the same size on every rank
    assert s0 != s1                                # ... but each rank's own seeded system
    assert m0 == m1 == 20.0                        # both ranks see the slowest rank's time
    assert v0 == v1 == pytest.approx(4096 * 100 * 3 * 2 / 20e-3)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(7.5) == 7.5
    assert bench.whole_job_rate(1000, 10, 2, 1, 5.0) == pytest.approx(1000 * 10 * 2 / 5e-3)


def _replica_rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import workloads as W
    from paper_1912_04232_b300.replicas import split_replicas
    specs = W.replica_plan(R=512, n_max=8192, seed=0)
    mine = split_replicas([sp.N for sp in specs], world)[rank]
    # this rank's replicas, generated here from their own seeds
    sums = {i: float(W.replica_initial(specs[i])[0][:, :3].astype(np.float64).sum()) for i in mine}
    everyone = [None] * world
    dist.all_gather_object(everyone, (rank, sorted(sums.items()), sum(specs[i].N for i in mine)))
    if rank == 0:
        out.put(everyone)
    dist.barrier()
    dist.destroy_process_group()


def test_configuration_4_replicas_split_over_two_gloo_ranks():
    # each rank takes a share of the 512 replicas; the shares are disjoint,
    # cover the set, balance the particles, and every replica is generated on
    # its rank exactly as one process generates it (its state depends on its
    # own seed only)
    import workloads as W
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    everyone = q.get(timeout=180)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    specs = W.replica_plan(R=512, n_max=8192, seed=0)
    seen = {}
    loads = []
    for rank, items, load in everyone:
        loads.append(load)
        for i, s in items:
            assert i not in seen
            seen[i] = s
    assert sorted(seen) == list(range(512))
    assert sum(loads) == sum(sp.N for sp in specs)
    assert max(loads) <= 1.01 * min(loads)
    for i in (0, 1, 255, 511):
        assert seen[i] == float(W.replica_initial(specs[i])[0][:, :3].astype(np.float64).sum())


def test_replica_split_is_deterministic_and_balanced():
    from paper_1912_04232_b300.replicas import split_replicas
    rng = np.random.default_rng(3)
    sizes = np.exp(rng.uniform(np.log(64), np.log(8192), 300)).astype(int)
    for world in (1, 2, 3, 8):
        a = split_replicas(sizes, world)
        assert a == split_replicas(list(sizes), world)
        assert sorted(i for s in a for i in s) == list(range(300))
        loads = [int(sizes[s].sum()) for s in a]
        # largest-first greedy: no rank exceeds another by more than one replica
        assert max(loads) - min(loads) <= int(sizes.max())
    assert split_replicas(sizes, 1) == [list(range(300))]
    with pytest.raises(ValueError):
        split_replicas(sizes, 0)
