"""One problem split across ranks (Morton ranges of targets and chart nodes,
mesh replicated), run here as shards in sequence on one GPU: the shards'
results, put back in the caller's order, equal the single call's.

Not bitwise: each call Morton-sorts its own targets over their own bounding
box and forms its own target blocks, so the near/far split of a tile, and
the summation order, can differ at block edges.  Both sides are within the
path's tolerance of the oracle, so they agree within that tolerance (the
measured differences are far smaller)."""
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
    from paper_1909_13356_gb300 import shard
    w = synth.torus_c2(n_targets=200_000, nu=120, nv=32)
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)   # 276,480 nodes: treecodes on
    return lsm, shard, w, m, mesh


@pytest.mark.parametrize("prec,tol", [(1, 1e-7), (2, 1e-12)])
def test_target_shards_equal_the_single_call(setup, prec, tol):
    lsm, shard, w, m, mesh = setup
    x = w["targets"]
    xd = torch.from_numpy(x).cuda()
    phi, grad = mesh.eval_phi_grad(xd, prec)
    for nparts in (2, 3):
        parts = shard.morton_ranges(x, nparts)
        vals = []
        for idx in parts:
            p, g = mesh.eval_phi_grad(xd[torch.from_numpy(idx).cuda()], prec)
            vals.append(torch.cat([p[:, None], g], 1).cpu().numpy())
        full = np.empty((len(x), 4))
        for idx, v in zip(parts, vals):
            full[idx] = v
        assert np.abs(full[:, 0] - phi.cpu().numpy()).max() <= tol
        assert np.abs(full[:, 1:] - grad.cpu().numpy()).max() <= 1e-7 / m.sigma.min()


def test_chart_node_shards_equal_the_single_solve(setup):
    lsm, shard, w, m, mesh = setup
    order = 4
    x1, h1, st1, s1 = mesh.solve_charts(order=order, tol=1e-12, precision=lsm.MIXED)
    tri, uvw = lsm.refined_nodes(order, np.zeros(m.m, dtype=np.int32))
    x0 = shard.chart_node_positions(m.verts, m.tris, tri, uvw)
    parts = shard.morton_ranges(x0, 2)
    xs = np.empty_like(x1)
    sts = np.empty_like(st1)
    for idx in parts:
        xp, hp, stp, sp = mesh.solve_charts_nodes(tri[idx], uvw[idx], tol=1e-12, precision=lsm.MIXED)
        xs[idx], sts[idx] = xp, stp
        assert sp.n_failed == 0
    assert np.all(sts & 255 == 0) and np.all(st1 & 255 == 0)
    assert np.abs(xs - x1).max() <= 1e-9
