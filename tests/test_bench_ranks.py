"""The bench's multi-rank host logic, on CPU with gloo (world size 2).

Under torchrun every rank fuses its own frames into its own volume (replicas:
no data exchanged on the fusion path). The only collective is the job total
taken after the timed region: points summed over ranks, elapsed time the
maximum over ranks. These tests run that reduction as two gloo processes, and
check that the ranks get disjoint inputs and that the reference arm prints
from rank 0 only.
"""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}",
                            rank=rank, world_size=world)
    try:
        # rank r fused 1000*(r+1) points in 1.5 + r seconds
        pts, ms = bench.reduce_job(1000 * (rank + 1), 1.5 + rank, world, "cpu")
        # the same call again with the slowest rank first
        pts2, ms2 = bench.reduce_job(7, 9.0 - rank, world, "cpu")
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
        json.dump({"pts": pts, "ms": ms, "pts2": pts2, "ms2": ms2}, fh)


def test_reduce_job_gloo_world2(tmp_path):
    import torch.multiprocessing as mp

    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        d = json.load(open(tmp_path / f"rank{r}.json"))
        assert d["pts"] == 1000 + 2000          # points summed
        assert d["ms"] == pytest.approx(2.5)    # the slowest rank's time
        assert d["pts2"] == 14
        assert d["ms2"] == pytest.approx(9.0)


def test_reduce_job_single_rank_is_identity():
    import bench

    assert bench.reduce_job(123, 4.5, 1, "cpu") == (123, 4.5)


def test_ranks_fuse_disjoint_frames():
    import bench

    seen = set()
    for r in range(8):
        idx = bench.frame_indices(r)
        assert len(idx) == bench.N_FRAMES == len(set(idx))
        assert not seen & set(idx)
        seen |= set(idx)


def test_reference_arm_prints_on_rank0_only():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "3"], env=env, capture_output=True,
                       text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
