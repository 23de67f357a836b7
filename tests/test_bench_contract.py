"""The benchmark's output contract, on the CPU: the reference arm (the FP64
oracle timed on the host cores) prints one JSON line with every key the
throughput line carries; non-zero ranks of a multi-process launch print
nothing and exit 0; a recorded DRAM-traffic figure is used only for the
kernel source and tuned schedule it was captured on."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench(args, env=None, timeout=300):
    e = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        e.pop(k, None)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=timeout)


def test_reference_arm_prints_one_complete_line():
    import bench
    r = _bench(["--impl", "reference", "--steps", "2", "--warmup", "3", "--scale", "0.05"])
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["ms_per_step"] > 0
    assert (line["n_gpus"], line["steps"], line["warmup"]) == (1, 2, 3)
    assert line["higher_is_better"] is True and line["scaling"] == "weak" and line["vs_baseline"] is None
    assert line["dtype"] == "f64" and line["data"] == "synthetic"
    assert line["config"]["workload"] == "large-2.2m" and line["config"]["sample"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["sample"] and cb["value"] == line["value"]
    assert cb["unit"] == line["unit"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_exit_quietly():
    r = _bench(["--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"],
               env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip() == ""


def test_recorded_traffic_is_tied_to_source_and_schedule(monkeypatch):
    import bench
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["filter.sweep"]
    key = next(iter(rec))
    workload, weights = key.split("/")
    entries = rec[key]
    scheds = [e["sweep_schedule"] for e in entries]
    assert len({tuple(s) for s in scheds}) == len(scheds)  # one record per schedule
    for entry in entries:
        sched = entry["sweep_schedule"]
        want = entry["dram_bytes_per_launch"]
        # the per-launch mean is the mean of the recorded launches
        per = entry["per_launch"]
        assert want == pytest.approx(sum(p["dram_read"] + p["dram_write"] for p in per) / len(per))
        monkeypatch.setattr(bench, "sweep_source_hash", lambda: entry["source_hash"])
        assert bench.recorded_traffic("filter.sweep", workload, weights, sched) == want
        if list(reversed(sched)) not in scheds:
            assert bench.recorded_traffic("filter.sweep", workload, weights, list(reversed(sched))) is None
        assert bench.recorded_traffic("filter.sweep", workload, "bf16" if weights != "bf16" else "f32",
                                      sched) is None
        monkeypatch.setattr(bench, "sweep_source_hash", lambda: "0" * 16)
        assert bench.recorded_traffic("filter.sweep", workload, weights, sched) is None
