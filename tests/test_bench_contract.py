"""Host-side pieces of bench.py: the reference arm's JSON line (the oracle on a bounded
sample), the rule that the stored stencil traffic is dropped once the stencil changes, and
where the raw clock samples are written."""
import json
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_contract_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "2",
                          "--warmup", "1", "--ref-seconds", "1", "--oracle-slice"], cwd=ROOT,
                         capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    # the line names what was timed: the slice's cells, the oracle steps of one bench step,
    # and a per-step time that is the measured one (cells x steps / rate)
    assert d["config"]["cells"] == 256 * 128 * 256 and "256x128x256" in d["config"]["workload"]
    per = d["config"]["cells"] * d["config"]["steps_per_bench_step"] / (d["value"] * 1e9)
    assert abs(d["ms_per_step"] / 1e3 - per) <= 1e-6 * per
    assert "set-up outside the timer" in d["cpu_baseline"]["sample"]


def test_stored_traffic_is_dropped_when_the_stencil_changes(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    assert bench.stencil_traffic("k_yee_tma_batch") is not None   # committed captures match the sources
    assert bench.stencil_traffic("k_yee_tb2") is not None
    # a copy of the tree whose stencil source differs by one byte
    fake = tmp_path / "root"
    (fake / "profiles").mkdir(parents=True)
    (fake / "paper_2208_04371_b300" / "csrc").mkdir(parents=True)
    name = "k_yee_tma_batch_traffic_lossy_line_768x384x256.json"
    shutil.copy(os.path.join(ROOT, "profiles", name), fake / "profiles" / name)
    src = open(os.path.join(ROOT, "paper_2208_04371_b300", "csrc", "yf_tma.cu"), "rb").read()
    (fake / "paper_2208_04371_b300" / "csrc" / "yf_tma.cu").write_bytes(src + b"\n")
    monkeypatch.setattr(bench, "ROOT", str(fake))
    assert bench.stencil_traffic("k_yee_tma_batch") is None


def test_clock_samples_go_to_the_temp_directory_unless_given_one(tmp_path):
    sys.path.insert(0, ROOT)
    import tempfile

    import bench
    s = bench.ClockSampler(3)
    assert os.path.dirname(s.path) == tempfile.gettempdir()
    assert os.path.basename(s.path) == "yf_bench_clocks_rank3.csv"
    s = bench.ClockSampler(0, str(tmp_path))
    assert s.path == os.path.join(str(tmp_path), "yf_bench_clocks_rank0.csv")
    # without nvidia-smi (or a GPU) the sampler reports that nothing was sampled
    if shutil.which("nvidia-smi") is None:
        s.start()
        assert s.stop()["reasons"] == ["unsampled"]
