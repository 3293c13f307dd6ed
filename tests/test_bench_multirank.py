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
