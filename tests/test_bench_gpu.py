"""bench.py's JSON line on a reduced corpus: every key of the contract, with
values of the right kind (the default run measures the full workload; this
only guards the line's shape and its arithmetic)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(*args):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=900)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_sweep_line_has_the_contract():
    d = run("--docs", "20000", "--burnin", "2", "--steps", "3", "--warmup", "3", "--cpu-docs", "300",
            "--serve-low-requests", "20", "--serve-high-rate", "400", "--serve-high-seconds", "0.5",
            "--batch-scale", "0.02", "--batch-steps", "2")
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "roofline", "cpu_baseline", "e2e", "gpu_launches", "clocks"):
        assert k in d, k
    assert d["n_gpus"] == 1 and d["steps"] == 3 and d["warmup"] == 3 and d["scaling"] == "weak"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["higher_is_better"] is True
    assert d["config"]["workload"] and d["gpu_launches"] >= 5 * 3
    r = d["roofline"]
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] > 0
    assert r["frac"] == pytest.approx(r["achieved"] / r["peak"])
    ph = d["phi_step"]
    assert 0 < ph["nnz_n"] <= d["config"]["N"] and ph["nnz_phi"] > 0
    assert ph["bytes_per_sweep"] == pytest.approx(6 * d["config"]["N"] + 14 * ph["nnz_phi"] + 8 * ph["nnz_n"])
    assert ph["frac"] == pytest.approx(ph["achieved"] / ph["peak"])
    sw = d["sweep_roofline"]
    assert sw["bytes_per_sweep"] == pytest.approx(r["algorithmic_bytes_per_launch"] + ph["bytes_per_sweep"])
    assert sw["frac"] == pytest.approx(sw["achieved"] / sw["peak"])
    c = d["cpu_baseline"]
    assert c["kind"] == "oracle" and c["cores"] >= 1 and c["value"] > 0 and c["sample"]
    e = d["e2e"]
    assert e["value"] > 0 and e["unit"] == d["unit"] and e["h2d_bytes_per_step"] > 0 and e["d2h_bytes_per_step"] > 0
    assert "sm_mhz" in d["clocks"] and "reasons" in d["clocks"]
    sv = d["serving"]
    assert sv["identical_to_alone"] is True and sv["rate_docs_per_s"] <= sv["one_at_a_time_capacity_docs_per_s"]
    for arm in ("continuous", "one_at_a_time", "high_rate"):
        assert sv[arm]["p99_ms"] >= sv[arm]["p50_ms"] > 0 and sv[arm]["docs_per_s"] > 0, arm
    assert sv["one_at_a_time"]["service_p99_ms"] >= sv["one_at_a_time"]["service_p50_ms"] > 0
    bt = d["batched"]
    assert bt["identical_topics"] is True and bt["N"] > 0 and bt["speedup_vs_sequential"] > 0


def test_reference_line_has_the_contract():
    d = run("--impl", "reference", "--steps", "1", "--warmup", "0", "--ref-docs", "200")
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
