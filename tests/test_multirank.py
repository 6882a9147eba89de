"""The bench's multi-rank logic on CPU: two gloo ranks (world size 2).

Transforms shard across ranks as independent work (one seed per rank, no
collective on the data path); the job's time is the slowest rank's, and the
reported value is the units all ranks processed over that time.  The
reference arm (the CPU oracle) runs on rank 0 only.
"""
import contextlib
import io
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as tdist

    import bench

    tdist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        prm = bench.rank_transforms(rank)
        digest = torch.tensor([float(np.float64(prm.astype(np.float64).sum())), float(prm[0, 0])], dtype=torch.float64)
        got = [torch.zeros(2, dtype=torch.float64) for _ in range(world)]
        tdist.all_gather(got, digest)
        seconds = 1.0 + rank  # rank 1 is the slow one
        t = bench.max_over_ranks(seconds, world)
        value = bench.whole_job_rate(world, 4, 1000, t)
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            args = type("A", (), {"gpus": world, "steps": 1, "warmup": 0})()
            if rank != 0:
                bench.run_reference(args, rank, world)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([t, value, len(prm), got[0][0].item(), got[1][0].item(), len(buf.getvalue())]))
    finally:
        tdist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp

    world = 2
    tmp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    r0 = np.load(tmp_path / "rank0.npy")
    r1 = np.load(tmp_path / "rank1.npy")
    for r in (r0, r1):
        assert r[0] == 2.0  # the max over ranks, seen identically by both
        assert r[1] == pytest.approx(2 * 4 * 1000 / 2.0)  # whole job: both ranks' units over the slowest time
        assert r[2] == 4096
    assert r0[3] == r1[3] and r0[4] == r1[4]
    assert r0[3] != r0[4]  # the two ranks evaluate different transforms
    assert r1[5] == 0  # rank 1 runs no reference work and prints nothing


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(1, 5, 10, 2.0) == 25.0
    a, b = bench.rank_transforms(0), bench.rank_transforms(0)
    np.testing.assert_array_equal(a, b)
    assert a.shape == (bench.N_T, 9) and a.dtype == np.float32
