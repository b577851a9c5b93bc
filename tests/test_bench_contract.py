"""The benchmark's JSON line contract, checked on the CPU through the reference arm
(the oracle timed on the host cores) on the small R-MAT, and the rank handling
of a multi-process launch (only rank 0 prints)."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(*args, env=None):
    e = dict(os.environ)
    e.update(env or {})
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, env=e,
                          capture_output=True, text=True, timeout=300)


def test_reference_arm_prints_one_contract_line():
    r = _run("--impl", "reference", "--workload", "rmat16", "--steps", "2", "--warmup", "1")
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["unit"] == "GTEPS" and d["higher_is_better"] is True and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["config"]["workload"] == "rmat16"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    r = _run("--impl", "reference", "--workload", "rmat16", "--steps", "1", "--warmup", "0",
             env={"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"})
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""


def test_clock_sampler_summary_and_kept_copy(tmp_path, monkeypatch):
    """The clock record during the timed region: a stand-in nvidia-smi prints two samples, one
    with power capping active; the summary takes the median clock and lists the reason."""
    fake = tmp_path / "bin"
    fake.mkdir()
    exe = fake / "nvidia-smi"
    exe.write_text("#!/bin/sh\n"
                   "echo '0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active'\n"
                   "echo '0, 1950, 2070, 1400.0, 0x4, Not Active, Not Active, Not Active, Active'\n"
                   "sleep 30\n")
    exe.chmod(0o755)
    monkeypatch.setenv("PATH", str(fake) + os.pathsep + os.environ["PATH"])
    sys.path.insert(0, ROOT)
    import time
    import bench
    keep = tmp_path / "keep"
    c = bench.ClockSampler(0, str(keep))
    c.start()
    time.sleep(1.0)
    r = c.stop()
    assert r == {"sm_mhz": 2010.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 2}
    assert (keep / "clocks_rank0.csv").read_text().count("\n") == 2
    assert not os.path.exists(c.path)


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    sys.path.insert(0, ROOT)
    import bench
    c = bench.ClockSampler(0)
    c.start()
    assert c.stop() is None
    assert not os.path.exists(c.path)
