"""The CPU legs of bench.py: the reference arm (the oracle timed on the host) prints
one JSON line with the contract's keys, and the all-cores oracle timing runs one
spawned process per core on its own copy of the mesh."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
           "--warmup", "3", "--ref-seconds", "0.2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "cell-updates/s" and d["steps"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_all_cores_oracle_rate():
    sys.path.insert(0, ROOT)
    import bench
    rate, procs, steps, slowest = bench.cpu_oracle_rate_all_cores(1)
    expected = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    assert procs == expected and steps == 1
    assert rate > 0 and slowest > 0
    assert abs(rate - procs * bench.CELLS / slowest) <= 1e-9 * rate


def _fake_headline(bench):
    roof = {"bound": "alu", "achieved": 0.94, "peak": bench.FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": 0.94 / bench.FP64_PEAK_TFLOPS, "traffic": 14479885,
            "kernel": "predict_kernel<5, fp64>", "mean_picard_iters": 3.07,
            "predict_ms_per_launch": 0.535, "face_update_ms_per_launch": 0.162,
            "peak_note": "FP64 from unit counts and max clock"}
    head = bench.headline_line(
        world=1, steps=20, warmup=5, value=1.42e8, ms_per_step=70.4,
        tuning={"predict_cells_per_block": 32, "face_cells_per_block": 64, "graph_steps": 16,
                "predict_ms": 0.5},
        roofline=roof, e2e={"value": 1.41e8, "unit": "cell-updates/s",
                            "h2d_bytes_per_step": 14400000, "d2h_bytes_per_step": 14400000},
        launches=4000, clocks={"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 9},
        errors={"l1_density_vs_exact": 9.5e-16})
    head["cpu_baseline"] = {"value": 4.5e5, "unit": "cell-updates/s", "cores": 1, "kind": "oracle",
                            "sample": "55 time steps of the same 10^5-cell N=5 mesh (12.0 s, 1 thread)",
                            "all_cores": {"value": 7.1e6, "unit": "cell-updates/s", "cores": 16,
                                          "kind": "oracle", "sample": "16 processes, each 55 steps"}}
    return head


def test_headline_is_the_last_compact_line():
    """Studies print on earlier lines (a failing one prints its error), the
    headline prints last, holds only the contract's keys and stays small."""
    import io
    sys.path.insert(0, ROOT)
    import bench
    out = io.StringIO()
    big = {"rows": [{"i": i, "x": 1.0 / (i + 1)} for i in range(3000)]}  # ~60 KB study
    bench.print_study("big", lambda: big, out=out)

    def broken():
        raise RuntimeError("no GPU here")
    bench.print_study("broken", broken, out=out)
    head = _fake_headline(bench)
    bench.print_headline(head, out=out)
    lines = out.getvalue().splitlines()
    assert len(lines) == 3
    s0, s1, last = (json.loads(x) for x in lines)
    assert s0["study"] == "big" and s0["result"] == big
    assert s1["study"] == "broken" and "no GPU here" in s1["error"]
    assert len(lines[-1]) <= bench.MAX_HEADLINE_BYTES
    assert last["value"] > 0 and last["unit"] == "cell-updates/s"
    assert set(last) <= set(bench.HEADLINE_KEYS)
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "dtype", "config", "roofline", "cpu_baseline", "e2e",
              "clocks", "gpu_launches"):
        assert k in last, k
    assert last["roofline"]["frac"] == head["roofline"]["frac"]


def test_headline_rejects_extra_keys_and_oversize():
    import io
    import pytest
    sys.path.insert(0, ROOT)
    import bench
    head = _fake_headline(bench)
    head["variants"] = [1, 2, 3]
    with pytest.raises(ValueError):
        bench.print_headline(head, out=io.StringIO())
    head = _fake_headline(bench)
    head["config"]["workload"] = "x" * 5000
    with pytest.raises(ValueError):
        bench.print_headline(head, out=io.StringIO())
