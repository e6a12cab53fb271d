"""The FP64 oracle timed on the host cores, on the CPU: the reference arm of bench.py (one
JSON line with the keys the benchmark contract names, and the same metric and unit as the
GPU arm) and the cpu_baseline record's sample calibration."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args],
                         capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1, out.stdout
    return json.loads(lines[0])


def test_reference_arm_prints_one_contract_line():
    d = run_bench("--impl", "reference", "--workload", "plain-128-c128", "--steps", "2",
                  "--warmup", "1")
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["metric"] == d["unit"] == "grid-point*steps/s"
    assert d["higher_is_better"] is True and d["steps"] == 2 and d["warmup"] == 1
    assert d["value"] > 0 and d["ms_per_step"] > 0
    assert d["config"]["workload"] == "plain-128^2"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"]
    assert "sample" in cb
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}


def test_reference_arm_on_a_rank_other_than_zero_prints_nothing():
    env = dict(os.environ, WORLD_SIZE="2", RANK="1", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl",
                          "reference", "--steps", "1", "--warmup", "0"],
                         capture_output=True, text=True, timeout=300, cwd=ROOT, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_cpu_baseline_lengthens_the_sample_on_a_tiny_grid():
    """On a grid so small that a 2-step run takes microseconds, the oracle baseline keeps
    lengthening its runs until the timed difference is long enough: the rate stays finite
    and plausible instead of a division by timer noise, and the sample says how many steps
    it took."""
    import bench
    from paper_1909_02894_gb300 import workloads as W

    w = W.plain_128(n=16, steps=1)
    rec, state = bench.cpu_baseline(w, check_steps=2)
    assert state.shape == (2, 16, 16)
    assert 0 < rec["value"] < 1e11
    steps = int(rec["sample"].split("difference of ")[1].split("-step")[0])
    assert steps > 2
    assert 0 < rec["single_thread"]["value"] < 1e11
