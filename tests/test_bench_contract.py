"""The benchmark's reference arm on the host (no GPU): `bench.py --impl
reference` times the FP64 oracle and prints one JSON line with the keys of the
benchmark contract (the same line shape as the GPU arm)."""

import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["unit"] == "trajectories/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 1 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    assert "workload" in d["config"]


@pytest.mark.gpu
def test_gpu_arm_profiling_line():
    """A short single-arithmetic run of the GPU arm: one JSON line with the
    roofline object, the clock record and the launch count."""
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--only", "df64", "--ntraj", "2000",
                        "--steps", "1", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [x for x in r.stdout.splitlines() if x.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "gpu_launches", "clocks"):
        assert key in d, key
    rl = d["roofline"]
    assert rl["bound"] == "alu" and rl["unit"] == "TFLOP/s" and 0 < rl["frac"] < 1.5
    assert abs(rl["frac"] - rl["achieved"] / rl["peak"]) < 1e-12
    assert rl["traffic"] is None  # traffic is reported for the full-size launch only
    assert d["gpu_launches"] > 0 and d["value"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]


def test_lockstep_launch_count_follows_the_library_schedule():
    """The bench's `gpu_launches` for the lock-step exponential path counts the
    library's schedule: its default catch-up cadence is the one the library's
    run enqueues, and at a catch-up every eight intervals the count per run is
    217 (the ncu launch list of two runs of that build held 434 launches)."""
    import importlib.util
    import inspect
    import re
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    with open(os.path.join(ROOT, "paper_1810_03047_gb300", "csrc", "qtm_api.cpp")) as f:
        every = int(re.search(r"kCatchUpEvery\s*=\s*(\d+)", f.read()).group(1))
    assert inspect.signature(bench.lockstep_launches).parameters["every"].default == every
    assert bench.lockstep_launches(101, every=8) == 217
    # 100 products, 101 per-interval launches, 7 catch-ups, the finish, the reduction
    assert bench.lockstep_launches(101, every=16) == 100 + 101 + 7 + 1 + 2
