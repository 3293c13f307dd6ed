"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas) agree on the job time, the slowest
rank's, and the whole-job rate counts the units of both; the reference arm runs on rank 0 only."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, step_ms, units, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.job_throughput(step_ms[rank], units, world)
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, units = 2, 1_000_000
    step_ms = [10.0, 30.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_rank, args=(world, _free_port(), step_ms, units, out), nprocs=world, start_method="spawn")
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 30.0
        assert abs(value - world * units / 0.030) < 1e-6 * value


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.job_throughput(20.0, 500, 1) == (20.0, 500 / 0.020)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("RANK", "1")

    class Args:
        steps, warmup, gpus = 1, 0, 2
    bench.run_reference(Args())
    assert capsys.readouterr().out == ""


def _shard_rank(rank, world, port, out):
    """One rank of the sharded batch: the library's assignment, then the job figures by all_reduce."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import torch
    import paper_2608_16208_b300 as bie
    import workloads as wl
    import numpy as np
    specs = wl.batch_surfaces(seed=0, count=64)
    costs = [16 * sp["Np"] * 48 * sp["Mt"] * np.log2(sp["Mt"]) for sp in specs]
    owner, load = bie.shard_surfaces(costs, world)
    mine = [i for i in range(64) if owner[i] == rank]
    # every rank computes the same assignment, so the shares partition the batch
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    t = torch.tensor([float(sum(costs[i] for i in mine))], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    out[rank] = (gathered, float(t.item()), [float(v) for v in load])
    dist.destroy_process_group()


def test_sharded_batch_partitions_the_surfaces():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_shard_rank, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    gathered, worst, load = res[0]
    assert res[1][0] == gathered
    every = sorted(i for share in gathered for i in share)
    assert every == list(range(64))
    assert abs(worst - max(load)) <= 1e-9 * worst
    # longest-processing-time keeps the largest load within 4/3 of the balanced share
    assert max(load) <= (4.0 / 3.0) * sum(load) / world


def test_shard_assignment_is_greedy_lpt():
    import paper_2608_16208_b300 as bie
    owner, load = bie.shard_surfaces([5.0, 1.0, 4.0, 3.0, 3.0], 2)
    # in decreasing cost 5, 4, 3, 3, 1 (equal costs keep their order), each to the least-loaded rank:
    # 5 -> 0, 4 -> 1, 3 -> 1 (4 < 5), 3 -> 0 (5 < 7), 1 -> 1 (7 < 8)
    assert list(owner) == [0, 1, 1, 1, 0]
    assert list(load) == [8.0, 8.0]
