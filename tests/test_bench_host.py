"""Host logic of bench.py that needs no GPU: the DRAM traffic figure is taken
from the committed ncu record only while every source file it names is
unchanged."""

import hashlib
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _tree(tmp_path, files, record):
    csrc = tmp_path / "paper_2209_01158_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name, text in files.items():
        (csrc / name).write_text(text)
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "traffic.json").write_text(json.dumps(record))
    return csrc


def _sha(text):
    return hashlib.sha256(text.encode()).hexdigest()


def test_traffic_needs_every_named_source_unchanged(tmp_path, monkeypatch):
    import bench
    files = {"k.cu": "kernel", "s.cuh": "sync"}
    rec = {"step_kernel_fp64": {"sources": {n: _sha(t) for n, t in files.items()},
                                "dram_bytes_per_cell_iteration": 61.0}}
    csrc = _tree(tmp_path, files, rec)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_unit("step_kernel_fp64") == 61.0
    (csrc / "s.cuh").write_text("sync, changed")
    assert bench.traffic_per_unit("step_kernel_fp64") is None
    assert bench.traffic_per_unit("no_such_kernel") is None


def test_traffic_single_source_record(tmp_path, monkeypatch):
    import bench
    rec = {"k": {"source": "k.cu", "source_sha256": _sha("kernel"), "dram_bytes_per_cell_iteration": 18.0}}
    _tree(tmp_path, {"k.cu": "kernel"}, rec)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.traffic_per_unit("k") == 18.0


def test_reference_arm_prints_the_contract_line():
    """`bench.py --impl reference` runs the CPU oracle on a crop and prints one
    JSON line with the reference arm's keys (no GPU needed)."""
    import subprocess
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                          "--steps", "1", "--warmup", "0", "--crop", "32"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    for k in ("metric", "unit", "higher_is_better", "config", "cpu_baseline", "e2e"):
        assert k in line
    assert line["cpu_baseline"]["kind"] == "oracle"
    assert line["e2e"]["h2d_bytes_per_step"] == 0
