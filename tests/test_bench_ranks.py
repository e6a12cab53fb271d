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


def test_traffic_summaries_are_keyed_as_the_bench_looks_them_up(tmp_path, monkeypatch):
    """The committed ncu traffic summaries are found under the names bench.py passes (the
    workload's grid name and precision, the batch mix's size), and only there."""
    from paper_1909_02894_gb300 import workloads as W

    name = W.large_4096(n=64, steps=1).name.replace("64", "4096")
    assert name == "large-4096^2"
    h = bench.kernel_hash()
    f = tmp_path / "profiles"
    f.mkdir()
    (f / "line_pass_traffic.txt").write_text(
        f"# c\nworkload = {name}\nprecision = c64\nkernel_hash = {h}\n"
        "dram_bytes_per_launch = 123\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "kernel_hash", lambda: h)
    assert bench.ncu_traffic(name, "c64") == 123.0
    assert bench.ncu_traffic(name, "c128") is None
    assert bench.ncu_traffic("large-4096", "c64") is None


def test_kernel_hash_ignores_comments_but_not_code(tmp_path, monkeypatch):
    """The committed ncu counters are keyed by a hash of the kernel code: a comment edit
    keeps it, any code edit changes it."""
    import shutil

    src = os.path.join(bench.ROOT, "paper_1909_02894_gb300", "csrc")
    dst = tmp_path / "paper_1909_02894_gb300" / "csrc"
    dst.mkdir(parents=True)
    for f in bench.KERNEL_SOURCES:
        shutil.copy(os.path.join(src, f), dst / f)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_hash()
    p = dst / "common.cuh"
    text = p.read_text()
    p.write_text(text + "\n// a comment\n/* another\n   comment */\n")
    assert bench.kernel_hash() == h0
    p.write_text(text + "\nstatic const int dgb_unused_for_hash_test = 1;\n")
    assert bench.kernel_hash() != h0


def test_clock_summary_reports_the_median_and_every_active_reason():
    """The clock record of a bench line: median SM clock under load, the highest max clock,
    and each throttle reason seen Active in any sample (nvidia-smi csv, noheader, nounits)."""
    c = bench.Clocks(0)
    c.out = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1500, 2070, 1400.0, 0x0000000000000040, Not Active, Active, Not Active, Active",
        "garbage line",
    ])
    s = c.summary()
    assert s["samples"] == 4
    assert s["sm_mhz"] == 2025.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]
    c.out = ""
    assert c.summary()["reasons"] == ["unsampled"]
