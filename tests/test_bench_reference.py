"""The bench's reference arm (the oracle on the host cores) prints one JSON
line with the keys the bench contract asks of it: run on a small torus, no
GPU needed."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--cells", "24x8",
           "--targets", "400", "--steps", "2", "--warmup", "1"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, out.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    assert d["metric"] == "phi_grad_evals_per_s" and d["unit"] == "evals/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["cpu_baseline"]["cores"] >= 1 and d["cpu_baseline"]["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert d["config"]["workload"].startswith("graded_torus")


def test_product_arm_fails_without_a_gpu():
    """With no CUDA device the product arm exits non-zero and prints no
    result line: there is no CPU path behind it."""
    try:
        import torch
        if torch.cuda.is_available():
            import pytest
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--steps", "1", "--warmup", "1", "--no-cpu-baseline",
           "--no-e2e"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.returncode != 0
    assert not any(l.startswith("{") for l in out.stdout.splitlines())


def test_dram_traffic_follows_the_kernel_source(tmp_path, monkeypatch):
    """The roofline's DRAM traffic comes from a recorded ncu capture only while
    the sources it was taken on are unchanged (their SHA-256 matches)."""
    import hashlib
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    h = hashlib.sha256()
    for name in ("eval.cu", "tree.cu", "ff.cuh"):
        with open(os.path.join(ROOT, "paper_1909_13356_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    sha = h.hexdigest()
    assert bench.kernel_sources_sha256() == sha
    rec = {"k_eval_ff": {"dram_bytes_per_launch": 1234.0, "sources_sha256": sha, "summary": "profiles/x.md"}}
    path = tmp_path / "dram.json"
    path.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "DRAM_FILE", str(path))
    assert bench._dram_traffic("k_eval_ff") == (1234.0, "profiles/x.md")
    assert bench._dram_traffic("k_eval_mixed") == (None, None)
    rec["k_eval_ff"]["sources_sha256"] = "0" * 64
    path.write_text(json.dumps(rec))
    assert bench._dram_traffic("k_eval_ff") == (None, None)
    monkeypatch.setattr(bench, "DRAM_FILE", str(tmp_path / "missing.json"))
    assert bench._dram_traffic("k_eval_ff") == (None, None)
