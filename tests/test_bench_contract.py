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


def _traffic_csv(path, reads):
    """An ncu launch-list CSV with one k_sweep launch per entry of reads."""
    head = ["ID", "Kernel Name", "Metric Name", "Metric Unit", "Metric Value", "Extra"]
    rows = [head]
    for i, rd in enumerate(reads):
        name = f"void k_sweep_dr<float, 4, 4, 2, 2, {i % 2}, 0, 0>(gift::SweepArgs)"
        rows += [[str(i), name, "dram__bytes_read.sum", "byte", f"{rd:,}", ""],
                 [str(i), name, "dram__bytes_write.sum", "byte", "1,000", ""],
                 [str(i), name, "gpu__time_duration.sum", "ns", "100", ""]]
    with open(path, "w", newline="") as f:
        import csv
        csv.writer(f).writerows(rows)


def test_record_traffic_keeps_one_record_per_schedule(tmp_path, monkeypatch):
    """A capture replaces the record of its own schedule, keeps the records of
    other schedules taken on the same kernel source, and drops records of an
    older source."""
    import argparse
    import shutil
    import bench
    root = tmp_path / "repo"
    (root / "profiles").mkdir(parents=True)
    shutil.copytree(os.path.join(ROOT, "paper_2502_17632_gb300", "csrc"), root / "paper_2502_17632_gb300" / "csrc")
    monkeypatch.setattr(bench, "ROOT", str(root))
    cur = bench.sweep_source_hash()
    stale = {"dram_bytes_per_launch": 1.0, "per_launch": [], "source_hash": "0" * 16, "sweep_schedule": [1, 2, 3, 4]}
    with open(root / "profiles" / "traffic.json", "w") as f:
        json.dump({"filter.sweep": {"large-2.2m/f32": [stale]}}, f)

    def record(reads, sched):
        csv_path = tmp_path / "t.csv"
        _traffic_csv(csv_path, reads)
        args = argparse.Namespace(record_traffic=str(csv_path), schedule=sched, workload="large-2.2m",
                                  weights="f32")
        bench.record_traffic(args)
        with open(root / "profiles" / "traffic.json") as f:
            return json.load(f)["filter.sweep"]["large-2.2m/f32"]

    recs = record([100, 200, 300, 400], "4842,4842,0,4844")
    assert [r["sweep_schedule"] for r in recs] == [[4842, 4842, 0, 4844]]  # the stale record is gone
    assert recs[0]["source_hash"] == cur and recs[0]["dram_bytes_per_launch"] == pytest.approx(1250.0)
    recs = record([500, 600, 700, 800], "4844,4842,0,4844")
    assert sorted(tuple(r["sweep_schedule"]) for r in recs) == [(4842, 4842, 0, 4844), (4844, 4842, 0, 4844)]
    recs = record([1000, 1000, 1000, 1000], "4842,4842,0,4844")  # replaces its own schedule's record
    by = {tuple(r["sweep_schedule"]): r["dram_bytes_per_launch"] for r in recs}
    assert by == {(4842, 4842, 0, 4844): pytest.approx(2000.0), (4844, 4842, 0, 4844): pytest.approx(1650.0)}
    assert bench.recorded_traffic("filter.sweep", "large-2.2m", "f32", [4844, 4842, 0, 4844]) == pytest.approx(1650.0)
    assert bench.recorded_traffic("filter.sweep", "large-2.2m", "f32", [4842, 4842, 0, 4842]) is None
