"""The multi-rank host logic of bench.py on CPU: two gloo ranks.

Each rank solves its own graded torus (its own seed); the whole-job time is
the slowest rank's and the units are summed over ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t_ms = [1250.0, 1730.5][rank]
        units = [1_000_000 + 17, 2_105_920][rank]
        t, u = bench.reduce_over_ranks(dist, t_ms, units, "cpu")
        dist.barrier()
        np.save(os.path.join(out_dir, f"r{rank}.npy"), np.array([t, u], dtype=np.float64))
    finally:
        dist.destroy_process_group()


def test_reduce_over_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        t, u = np.load(tmp_path / f"r{r}.npy")
        assert t == 1730.5
        assert u == 1_000_017 + 2_105_920


def test_reduce_single_process_is_identity():
    import bench
    assert bench.reduce_over_ranks(None, 12.5, 7, "cpu") == (12.5, 7)


def test_rank_shards_are_independent_problems():
    import argparse
    import bench
    args = argparse.Namespace(small=True, targets=2000)
    w0, w1 = bench.workload(args, 0), bench.workload(args, 1)
    import synth
    ref = synth.torus_c2(n_targets=2000, nu=60, nv=16)
    # rank 0 is the single-GPU workload
    assert np.array_equal(w0["mesh"].verts, ref["mesh"].verts)
    assert np.array_equal(w0["targets"], ref["targets"])
    # rank 1 has the same size and connectivity but its own jitter and targets
    assert w1["mesh"].verts.shape == w0["mesh"].verts.shape
    assert np.array_equal(w1["mesh"].tris, w0["mesh"].tris)
    assert not np.allclose(w1["mesh"].verts, w0["mesh"].verts)
    assert not np.allclose(w1["targets"], w0["targets"])
