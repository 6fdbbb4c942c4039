"""The reference arm of bench.py on CPU: the oracle, timed on the host cores,
prints one JSON line with the same metric and config keys as the GPU arm, and
only rank 0 of a multi-rank launch runs it."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(extra_env=None, config="batched"):
    env = dict(os.environ)
    env.update(extra_env or {})
    args = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1", "--warmup", "0"]
    if config is not None:
        args += ["--config", config]
    r = subprocess.run(args, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


@pytest.mark.parametrize("config", ["batched", "mid", None])
def test_reference_arm_prints_the_contract_line(config):
    """None runs the default workload (1M x 1M, d = 384, bf16) on row slices."""
    lines = _run(config=config)
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference"
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in rec, key
    assert rec["value"] > 0 and rec["ms_per_step"] > 0
    assert rec["steps"] == 1 and rec["warmup"] == 0 and rec["n_gpus"] == 1
    assert rec["higher_is_better"] is True and rec["vs_baseline"] is None
    assert rec["data"] == "synthetic" and "workload" in rec["config"]
    if config is None:
        assert rec["config"]["workload"].startswith("precision") and rec["dtype"] == "bf16"
    cpu = rec["cpu_baseline"]
    assert cpu["kind"] == "oracle" and cpu["cores"] >= 1 and cpu["value"] == rec["value"] and cpu["sample"]
    e2e = rec["e2e"]
    assert e2e["value"] == rec["value"] and e2e["unit"] == rec["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_runs_on_rank_zero_only():
    assert _run({"RANK": "1", "WORLD_SIZE": "2", "LOCAL_RANK": "1"}) == []


def test_screen_traffic_is_dropped_once_the_kernel_source_changes(tmp_path, monkeypatch):
    """bench.py reports the committed DRAM bytes of the screen only while
    k_screen.cu is the source those counters were taken from."""
    import hashlib
    sys.path.insert(0, ROOT)
    import bench
    src = b"// a kernel source\n"
    (tmp_path / "paper_2307_03043_gb300" / "csrc").mkdir(parents=True)
    (tmp_path / "paper_2307_03043_gb300" / "csrc" / "k_screen.cu").write_bytes(src)
    (tmp_path / "profiles").mkdir()
    rec = {"mid/TF32": {"k_screen_sha256": hashlib.sha256(src).hexdigest(), "dram_bytes_per_launch": 123}}
    (tmp_path / "profiles" / "screen_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "CONFIG", "mid")
    assert bench.screen_traffic("TF32") == 123
    assert bench.screen_traffic("BF16") is None
    (tmp_path / "paper_2307_03043_gb300" / "csrc" / "k_screen.cu").write_bytes(src + b"// changed\n")
    assert bench.screen_traffic("TF32") is None
