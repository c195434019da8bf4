"""CPU test of bench.py's reference arm (the FP64 oracle timed on host cores):
one JSON line with the contract's keys, the same metric, unit and workload
as the GPU arm, and no output from ranks other than 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra):
    env = dict(os.environ, **env_extra)
    return subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2", "--warmup", "1"],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_prints_one_contract_line():
    r = _run({"RANK": "0"})
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    sys.path.insert(0, ROOT)
    import bench
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["higher_is_better"] is True and d["vs_baseline"] is None and d["data"] == "synthetic"
    assert d["config"]["workload"].startswith("MLP 784-100-10")
    assert "model" not in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_is_silent_on_other_ranks():
    r = _run({"RANK": "1", "WORLD_SIZE": "2"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_host_threads_follows_the_thread_variables(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("OPENBLAS_NUM_THREADS", "3")
    assert bench.host_threads() == 3
    monkeypatch.setenv("OPENBLAS_NUM_THREADS", "bad")
    monkeypatch.setenv("OMP_NUM_THREADS", "5")
    assert bench.host_threads() == 5
    monkeypatch.delenv("OPENBLAS_NUM_THREADS")
    monkeypatch.delenv("OMP_NUM_THREADS")
    monkeypatch.delenv("MKL_NUM_THREADS", raising=False)
    assert bench.host_threads() >= 1


def test_cpu_baseline_reports_single_thread_and_all_cores():
    """The GPU line's cpu_baseline: the oracle timed single-threaded and with
    one single-threaded process per host core, each rate with its thread count."""
    sys.path.insert(0, ROOT)
    import bench
    d = bench.cpu_baseline(seconds=0.5, J_s=1, M_s=200)
    assert d["kind"] == "oracle" and d["unit"] == bench.UNIT and d["cores"] == bench.host_threads()
    assert d["single_thread"]["cores"] == 1 and d["single_thread"]["value"] > 0
    assert d["all_cores"]["cores"] == d["cores"] and d["value"] == d["all_cores"]["value"] > 0
