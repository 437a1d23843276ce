"""The reference arm of bench.py (the FP64 oracle timed on the host) prints one
JSON line with the keys of the bench contract; run here on the 32^3 workload."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "c1", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["steps"] == 1
    assert d["unit"] == "NCG iters/s" and d["higher_is_better"] is True
    assert "workload" in d["config"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"] and cb["cores"] >= 1 and cb["sample"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_traffic_record_follows_the_source_digest(tmp_path, monkeypatch):
    """bench.py reports a kernel's ncu DRAM bytes only while the committed
    summary carries the digest of the current CUDA sources and the workload."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2510_24543_gb300 import build as B

    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    rec = {"kernels": {"k": {"workload": "c3p", "dram_bytes_per_launch": 1.5e8}}}
    path = tmp_path / "profiles" / "traffic.json"
    path.write_text(json.dumps({**rec, "sources": B._digest()}))
    assert bench.traffic_record("k", "c3p") == 1.5e8
    assert bench.traffic_record("k", "c1") is None
    assert bench.traffic_record("other", "c3p") is None
    path.write_text(json.dumps({**rec, "sources": "not the current sources"}))
    assert bench.traffic_record("k", "c3p") is None
