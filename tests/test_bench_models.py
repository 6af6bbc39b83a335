"""bench.py's byte models and roofline arithmetic, on CPU: the
algorithmic bytes of a z-step and of a Phi-step, and the fractions built on
them (the GPU line's values come from these functions)."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_z_step_bytes_follow_the_algorithmic_model():
    # per token 4 (word) + 2 + 2 (topic in, out) + 4 (sigma_a); 6 per min(K_d, K_v)
    # element; 8 per alias draw; 8 per document
    assert bench.z_bytes(1, 0, 0, 0) == 12
    assert bench.z_bytes(0, 1, 0, 0) == 6
    assert bench.z_bytes(0, 0, 1, 0) == 8
    assert bench.z_bytes(0, 0, 0, 1) == 8
    assert bench.z_bytes(1000, 133_000, 208, 3) == 12_000 + 798_000 + 1_664 + 24
    # the implementation's widths: 64-bit sigma_a and column offset, 6-byte alias slot
    assert bench.z_bytes_impl(1, 0, 0, 0) == 24 and bench.z_bytes_impl(0, 0, 1, 0) == 6


def test_phi_step_bytes_and_fraction():
    assert bench.phi_bytes(1, 0, 0) == 6.0 and bench.phi_bytes(0, 1, 0) == 14.0 and bench.phi_bytes(0, 0, 1) == 8.0
    r = bench.phi_roofline(2.0, 99_061_588, 3_929_551, 3_284_896, 6778.3)
    b = 6 * 99_061_588 + 14 * 3_929_551 + 8 * 3_284_896
    assert r["bytes_per_sweep"] == b
    assert r["achieved"] == pytest.approx(b / 2e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6778.3)
    assert r["nnz_n"] == 3_284_896 and r["unit"] == "GB/s"


def test_whole_job_throughput():
    assert bench.aggregate_tokens_per_s(99_061_588, 20, 1, 757.0) == pytest.approx(99_061_588 * 20 / 0.757)
    assert bench.aggregate_tokens_per_s(10, 2, 4, 1000.0) == pytest.approx(80.0)
