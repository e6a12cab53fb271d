"""The multi-rank side of bench.py on the CPU: world-size-2 gloo process groups stand in
for the per-GPU ranks (the path does not shard: each rank runs an independent replica,
the job's time is the slowest rank's and its throughput sums the replicas)."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(times[rank], world)
        out[rank] = (ms, bench.whole_job_value(1000, 10, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("times", [(2.0, 5.0), (7.5, 1.25)])
def test_two_gloo_ranks_agree_on_the_slowest_time_and_the_job_value(times):
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    slowest = max(times)
    for rank in range(world):
        ms, value = res[rank]
        assert ms == slowest
        assert value == pytest.approx(1000 * 10 * world / (slowest * 1e-3))


def test_single_process_keeps_its_own_time():
    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_value(4096 * 4096, 1000, 1, 544.0) == pytest.approx(
        4096 * 4096 * 1000 / 0.544)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    """Under torchrun the other ranks of the reference arm exit 0 without work."""
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = bench.argparse.Namespace(steps=3, warmup=3, gpus=2)
    assert bench.run_reference(args, "large-4096") == 0
    assert capsys.readouterr().out == ""
