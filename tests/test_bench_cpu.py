"""bench.py's host-side logic without a GPU: the clock record that decides
whether a run is kept, and the JSON line of the reference arm (the CPU
oracle), whose keys the benchmark contract fixes."""
import json
import os
import subprocess
import sys

import pytest

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_clock_summary_takes_the_median_and_the_active_reasons():
    cs = bench.ClockSampler(0)
    t = "2026/12/04 10:00:0{}.000"
    cs.lines = [
        t.format(1) + ", 0, 2070, 2070, 910.2, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        t.format(2) + ", 0, 1980, 2070, 1399.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        t.format(3) + ", 0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "[N/A], garbage",
        t.format(4) + ", 0, [N/A], 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
    ]
    s = cs.summary()
    assert s == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3,
                 "window": "headline leg (tuning, warm-up, timed region)"}
    cs.lines = [t.format(1) + ", 0, 1500, 2070, 700, 0x8, Active, Not Active, Active, Not Active"]
    assert cs.summary()["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    cs.lines = []
    assert cs.summary()["samples"] == 0 and cs.summary()["sm_mhz"] is None


def test_clock_summary_keeps_the_timed_window_when_it_has_three_samples():
    cs = bench.ClockSampler(0)
    rows = [(0, 1200), (1, 2070), (2, 2060), (3, 2050), (4, 1300)]
    cs.lines = [f"2026/12/04 10:00:0{s}.000, 0, {mhz}, 2070, 900, 0x0, Not Active, Not Active, Not Active, "
                "Not Active" for s, mhz in rows]
    cs.mark(bench._dt.datetime(2026, 12, 4, 10, 0, 1), bench._dt.datetime(2026, 12, 4, 10, 0, 3))
    s = cs.summary()
    assert s["window"] == "timed region" and s["samples"] == 3 and s["sm_mhz"] == 2060.0
    cs.mark(bench._dt.datetime(2026, 12, 4, 10, 0, 1), bench._dt.datetime(2026, 12, 4, 10, 0, 1, 500))
    assert cs.summary()["samples"] == 5           # fewer than three inside: the whole leg


def test_batch_sample_instances_match_the_full_batch():
    full = bench.wl.gaussian_batch_2d(count=64, seed=4, steps=0, sides=range(16, 65, 16))
    some = bench.wl.gaussian_batch_2d(count=64, seed=4, steps=0, sides=range(16, 65, 16), only={0, 32})
    assert [q.name for q in some] == ["gauss_0", "gauss_32"]
    for q, r in zip(some, bench.batch_sample(full)):
        assert q.name == r.name and q.a == r.a and q.s == r.s
        assert (q.psi0 == r.psi0).all() and (q.V == r.V).all()


def test_fewer_than_three_warmup_steps_are_refused():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "2"], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert r.returncode == 2 and "--warmup must be >= 3" in r.stderr


def test_reference_arm_prints_one_contract_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["value"] > 0 and d["higher_is_better"] is True and d["dtype"] == "f64"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
