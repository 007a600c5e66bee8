"""The multi-rank host logic on CPU: two gloo ranks.

One problem is split into contiguous Morton ranges of its targets and chart
nodes, one per rank, with the mesh replicated; each rank evaluates its own
range and the gathered results, in the caller's order, equal the
single-process result.  The whole-job time is the slowest rank's and the
units are summed over ranks.
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


def _init(rank, world, port):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    return dist


def _rank_main(rank, world, port, out_dir):
    dist = _init(rank, world, port)
    import bench
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


def _small_problem():
    import synth
    w = synth.torus_c2(n_targets=1500, nu=24, nv=8)
    return w


def _shard_main(rank, world, port, out_dir):
    """Each rank evaluates (with the oracle, on the host) only its Morton range
    of the targets; rank 0 gathers the shards in the caller's order."""
    dist = _init(rank, world, port)
    import oracle
    from paper_1909_13356_gb300 import shard
    try:
        w = _small_problem()
        m, x = w["mesh"], w["targets"]
        idx = shard.morton_ranges(x, world)[rank]
        y, nw, sg = oracle.sources(m.verts, m.tris, m.sigma, 3, 0)
        phi, grad = oracle.phi_grad(y, nw, sg, x[idx], nthreads=1)
        vals = np.concatenate([phi[:, None], grad], axis=1)
        full = shard.gather(dist, idx, vals, len(x))
        if rank == 0:
            np.save(os.path.join(out_dir, "gathered.npy"), full)
        np.save(os.path.join(out_dir, f"idx{rank}.npy"), idx)
    finally:
        dist.destroy_process_group()


def test_sharded_evaluation_gathers_to_the_single_result(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    mp.spawn(_shard_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    w = _small_problem()
    m, x = w["mesh"], w["targets"]
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 3, 0)
    phi, grad = oracle_mod.phi_grad(y, nw, sg, x, nthreads=1)
    full = np.load(tmp_path / "gathered.npy")
    assert np.array_equal(full[:, 0], phi)
    assert np.array_equal(full[:, 1:], grad)
    i0, i1 = np.load(tmp_path / "idx0.npy"), np.load(tmp_path / "idx1.npy")
    assert len(np.intersect1d(i0, i1)) == 0 and len(i0) + len(i1) == len(x)


def test_morton_ranges_partition_the_points():
    from paper_1909_13356_gb300 import shard
    g = np.random.default_rng(3)
    pts = g.normal(size=(10_007, 3))
    keys = shard.morton_keys(pts)
    for nparts in (1, 2, 3, 8):
        parts = shard.morton_ranges(pts, nparts)
        assert len(parts) == nparts
        allidx = np.concatenate(parts)
        assert np.array_equal(np.sort(allidx), np.arange(len(pts)))      # disjoint, complete
        sizes = [len(p) for p in parts]
        assert all(s % 256 == 0 for s in sizes[:-1])                      # whole target blocks
        assert max(sizes) - min(sizes) <= 256 + len(pts) % 256
        for a, b in zip(parts[:-1], parts[1:]):                          # contiguous in Morton order
            if len(a) and len(b):
                assert keys[a].max() <= keys[b].min()
        for p in parts:                                                   # each range in Morton order
            assert np.all(np.diff(keys[p].astype(np.int64)) >= 0)


def test_gather_without_a_process_group_scatters_in_place():
    from paper_1909_13356_gb300 import shard
    idx = np.array([4, 0, 2])
    out = shard.gather(None, idx, np.array([40.0, 0.0, 20.0]), 5)
    assert out[4] == 40.0 and out[0] == 0.0 and out[2] == 20.0


def test_chart_node_positions_lie_on_their_triangles():
    from paper_1909_13356_gb300 import shard
    verts = np.array([[0.0, 0, 0], [2.0, 0, 0], [0.0, 3, 0], [0, 0, 1.0]])
    tris = np.array([[0, 1, 2], [0, 2, 3]])
    tri = np.array([0, 1, 1])
    uvw = np.array([[0.5, 0.25, 0.1], [0.0, 0.0, 0.1], [0.5, 0.5, 0.1]])
    p = shard.chart_node_positions(verts, tris, tri, uvw)
    assert np.allclose(p, [[1.0, 0.75, 0.0], [0.0, 0.0, 0.0], [0.0, 1.5, 0.5]])


def test_replica_problems_are_independent():
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
