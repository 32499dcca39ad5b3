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


def test_headline_carries_fp32_forms_and_latency():
    """The metric names FP64 vs the FP32 predictor and p50/p99 latency: the
    headline summarises both studies and still fits the size limit."""
    import io
    sys.path.insert(0, ROOT)
    import bench
    long = "x" * 300  # study lines carry long workload strings; the summary drops them
    variants = [{"name": n, "workload": long, "value": v, "rel_linf_vs_fp64_path": e,
                 "l1_density_vs_exact": 1e-14}
                for n, v, e in (("dg5-1e5-incr", 5.3e8, 1.4e-13), ("dg5-1e5-fp32ff1", 3.8e8, 3e-8),
                                ("dg5-1e5-fp32pred", 1.2e8, 8e-9), ("dg7-1e6-incr", 3.8e8, 1e-13))]
    variants.append({"name": "dg5-1e5-ffpred", "workload": long, "error": "RuntimeError: x"})
    pt = {"server": {"p50_s": 0.058, "p99_s": 0.35, "solves_per_s": 161.0},
          "baseline_per_solve_fp64": {"p50_s": 3.7, "p99_s": 7.6, "solves_per_s": 15.3}}
    serving = {"workload": long, "saturation": {"solves_per_s": 238.0},
               "open_loop": [dict(pt, arrival_rate_frac_of_saturation=f) for f in (0.5, 0.8, 1.0)]}
    serving["open_loop"][1]["server"] = dict(pt["server"], p50_s=0.0579)
    head = _fake_headline(bench)
    head["fp32_predictor"] = bench.fp32_predictor_summary(variants, head["value"])
    head["latency"] = bench.latency_summary(serving)
    out = io.StringIO()
    line = bench.print_headline(head, out=out)
    assert len(line) <= bench.MAX_HEADLINE_BYTES
    d = json.loads(line)
    forms = d["fp32_predictor"]["forms"]
    assert set(forms) == {"increment", "fp32_ff_sweep", "fp32_fp64_sweeps"}
    assert forms["increment"]["value"] == 5.3e8
    assert abs(forms["increment"]["vs_fp64"] - 5.3e8 / head["value"]) <= 1e-12
    assert forms["fp32_fp64_sweeps"]["rel_linf_vs_fp64_path"] == 8e-9
    lat = d["latency"]
    assert lat["p50_s"] == 0.0579 and lat["p99_s"] == 0.35 and lat["load"] == "0.8 x saturation"
    assert lat["saturation_solves_per_s"] == 238.0 and lat["plain_fp64"]["p50_s"] == 3.7
    # missing or failed studies leave the keys out rather than breaking the line
    assert bench.fp32_predictor_summary(None, 1.0) is None
    assert bench.fp32_predictor_summary([{"name": "dg5-1e5-incr", "error": "x"}], 1.0) is None
    assert bench.latency_summary(None) is None
    assert bench.latency_summary({"open_loop": []}) is None


def test_reference_arm_under_two_rank_launch():
    """Launched as the multi-GPU bench is (torch.distributed.run, two ranks), the
    reference arm prints one line from rank 0; the other rank exits 0 without work."""
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-seconds", "0.2"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_reference_step_budget():
    """The reference arm's per-step oracle sample shrinks with the step count so
    the whole run stays within minutes; an explicit --ref-seconds wins."""
    sys.path.insert(0, ROOT)
    import bench
    assert bench.ref_step_seconds(3, 5) == 12.0
    assert bench.ref_step_seconds(5, 20) == 6.0
    assert bench.ref_step_seconds(10, 1000) == 1.0
    assert bench.ref_step_seconds(3, 5, 0.2) == 0.2
    for w, k in ((3, 5), (5, 20), (3, 50), (10, 200)):
        total = (w + k) * bench.ref_step_seconds(w, k)
        assert total <= max(bench.REF_TOTAL_SECONDS, (w + k) * 1.0)
