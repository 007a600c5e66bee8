"""Batched chart solves: many meshes in one set of launches per Newton sweep
(optionally replayed from a captured CUDA graph) give each mesh the result of
its own solve, within the chart-position tolerance."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as lsm
    ctx = lsm.Context(0)
    g = synth.rng(44)
    ms = [synth.ellipsoid(int(T), g) for T in (200, 340, 520, 260, 800, 230, 410, 300)]
    meshes = [ctx.upload(m.verts, m.tris, m.sigma, n_gl=4) for m in ms]
    return lsm, ctx, ms, meshes


@pytest.mark.parametrize("prec,tol,pos_tol", [(1, 1e-10, 1e-9), (0, 1e-12, 1e-10)])
@pytest.mark.parametrize("use_graph", [True, False])
def test_batch_matches_each_mesh_alone(setup, prec, tol, pos_tol, use_graph):
    lsm, ctx, ms, meshes = setup
    b = lsm.Batch(ctx, meshes)
    x, h, st, stats = b.solve_charts(order=6, tol=tol, precision=prec, use_graph=use_graph)
    assert stats.n_nodes == sum(m.m for m in ms) * 25
    assert np.all(st & 255 == 0), np.unique(st)
    o = 0
    for mesh in meshes:
        xa, ha, sa, _ = mesh.solve_charts(order=6, tol=tol, precision=prec)
        n = len(ha)
        assert np.all(sa & 255 == 0)
        assert np.abs(x[o:o + n] - xa).max() < pos_tol
        o += n
    b.free()


@pytest.mark.parametrize("ff_block,mixed_block", [(128, 256), (128, 128), (64, 64)])
def test_batch_layouts_match_each_mesh_alone(ff_block, mixed_block):
    """Work items of the other target-tile sizes (float-float 128 and 64,
    mixed 256, 128 and 64 targets): the batched solve still equals each
    mesh's own solve under the same options, and the nodes meet the bar."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as lsm
    ctx = lsm.Context(0, ff_block=ff_block, mixed_block=mixed_block)
    g = synth.rng(45)
    ms = [synth.ellipsoid(int(T), g) for T in (240, 610, 330)]
    meshes = [ctx.upload(m.verts, m.tris, m.sigma, n_gl=4) for m in ms]
    b = lsm.Batch(ctx, meshes)
    x, h, st, stats = b.solve_charts(order=6, tol=1e-10, precision=lsm.MIXED, use_graph=True)
    assert np.all(st & 255 == 0), np.unique(st)
    o = 0
    for mesh in meshes:
        xa, ha, sa, _ = mesh.solve_charts(order=6, tol=1e-10, precision=lsm.MIXED)
        n = len(ha)
        assert np.abs(x[o:o + n] - xa).max() < 1e-9
        o += n
    b.free()
    for mesh in meshes:
        mesh.free()
    ctx.close()


def test_batch_residual_against_oracle(setup, oracle_mod):
    lsm, ctx, ms, meshes = setup
    b = lsm.Batch(ctx, meshes[:3])
    x, h, st, stats = b.solve_charts(order=6, tol=1e-11, precision=lsm.MIXED)
    o = 0
    for m in ms[:3]:
        n = m.m * 25
        y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 4, 0)
        phi, _ = oracle_mod.phi_grad(y, nw, sg, x[o:o + n:11])
        assert np.abs(phi - 0.5).max() < 1e-11
        o += n
    b.free()


def test_batch_autotune_then_solve(setup):
    """lsm_batch_autotune picks the mixed kernel's near-field radius (within
    the mixed bound) and target tile on a sample of the batch's meshes; the
    batched solve with that choice still gives each mesh its own result."""
    lsm, ctx, ms, meshes = setup
    b = lsm.Batch(ctx, meshes)
    r = b.autotune(order=6, err_budget=5e-8)
    assert r["use_tree"] == 0 and r["candidates"] == 9   # 3 radii x 3 target tiles
    assert min(abs(r["cutoff"] - c) for c in (6.4, 6.5, 7.0)) < 1e-12
    assert r["targets_per_block"] in (64, 128, 256)
    assert r["err_phi"] <= 5e-8 and r["sample_targets"] == sum(m.m for m in ms) * 25
    x, h, st, stats = b.solve_charts(order=6, tol=1e-10, precision=lsm.MIXED, use_graph=True)
    assert np.all(st & 255 == 0)
    o = 0
    for mesh in meshes:
        xa, ha, sa, _ = mesh.solve_charts(order=6, tol=1e-10, precision=lsm.MIXED)
        n = len(ha)
        assert np.abs(x[o:o + n] - xa).max() < 1e-9
        o += n
    b.free()
