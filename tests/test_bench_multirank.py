"""The benchmark's multi-rank logic, on CPU with gloo and two ranks: the
timed region is the slowest rank's, the value counts every rank's tokens,
and only rank 0 reports."""
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    ms = [120.0, 80.0][rank]
    m = bench.reduce_max(ms, world)
    out[rank] = (m, bench.aggregate_tokens_per_s(1000, 5, world, m))
    dist.barrier()
    dist.destroy_process_group()


def test_slowest_rank_sets_the_time_and_value_counts_all_ranks():
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert out[0] == out[1]
    ms, value = out[0]
    assert ms == 120.0
    assert value == pytest.approx(2 * 1000 * 5 / 0.120)


def test_single_rank_is_the_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5


def test_reference_arm_non_zero_rank_exits_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_launch_count_and_profile_record_follow_the_source(tmp_path, monkeypatch):
    """Library kernels per sweep depend on the Phi mode and on a word above 2^17 tokens; the ncu
    record is used only while the kernel source hashes to the value it was taken on."""
    import numpy as np
    import bench
    assert bench.kernels_per_sweep(np.zeros(10, np.int32), 0) == 5
    assert bench.kernels_per_sweep(np.zeros(1 << 18, np.int32), 0) == 6
    assert bench.kernels_per_sweep(np.arange(10, dtype=np.int32), 1) == 8
    # the z-step as the handle laid it out: the cooperative kernel beside the main one when
    # some document is on CTAs; beside four per warp, the one-warp kernel for over-long documents
    w = np.zeros(310, np.int32)
    one = {"docs_per_warp": 1, "coop_docs": 0, "one_warp_docs": 2}
    assert bench.kernels_per_sweep(w, 0, one) == 5
    assert bench.kernels_per_sweep(w, 0, dict(one, coop_docs=1)) == 6
    four = {"docs_per_warp": 4, "coop_docs": 0, "one_warp_docs": 0}
    assert bench.kernels_per_sweep(w, 0, four) == 5
    assert bench.kernels_per_sweep(w, 0, dict(four, coop_docs=2, one_warp_docs=1)) == 7
    assert bench.kernels_per_sweep(w, 0, one, slice_docs=1) == 6
    rec = bench.recorded_profile()
    if rec:
        assert rec["source_sha"] == bench.kernel_source_hash()
    monkeypatch.setattr(bench, "kernel_source_hash", lambda: "0000000000000000")
    assert bench.recorded_profile() == {} and bench.recorded_traffic() is None
