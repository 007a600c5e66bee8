"""GPU parity of the Hessian of Phi and of the charts' second derivatives and
curvatures (Sec. 3.3, eq. uu_vector and its analogues) against the oracle.

The Hessian sums near tiles in FP64 and far tiles in FP32 (compensated): the
bar is 1e-7 of the largest Hessian entry.  The curvature kernel is FP64
elementwise work on the same inputs as the oracle: 1e-10 relative.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lsm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as m
    m.load()
    return m


def test_hessian_matches_oracle(lsm, oracle_mod):
    """Graded torus 48 x 16 cells (55,296 nodes), 2,000 targets within 3
    sigma, including targets on source nodes."""
    m = synth.torus(1.0, 0.3, 48, 16, 8.0, 0.05, 71)
    x = synth.targets_near_surface(m, 2000, synth.rng(72), 3.0)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, None, 6, 0)
    x[:5] = y[:5]
    _, _, Ho = oracle_mod.phi_grad_hess(y, nw, sg, x)
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, None, n_gl=6)
    H = mesh.eval_hessian(x)
    assert np.abs(H - Ho).max() <= 1e-7 * np.abs(Ho).max()
    # device pointers give the same values
    Hd = mesh.eval_hessian(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.array_equal(Hd, H)


@pytest.fixture(scope="module")
def sphere(lsm):
    """Icosphere level 2, sigma by the workloads' rule, 4x4 sources, order-8
    charts solved on the FP64 path; grad Phi and the Hessian at the nodes."""
    m = synth.icosphere(2)
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, None, n_gl=4)
    x, h, st, stats = mesh.solve_charts(order=8, tol=1e-13, precision=lsm.FP64)
    assert stats.n_failed == 0
    _, g = mesh.eval_phi_grad(x, lsm.FP64)
    H = mesh.eval_hessian(x)
    return m, ctx, mesh, x, h, g, H


def test_chart_curvature_matches_oracle(lsm, oracle_mod, sphere):
    m, ctx, mesh, x, h, g, H = sphere
    uu, uv, vv, km, kg = mesh.chart_curvature(8, h, g, H)
    ouu, ouv, ovv, okm, okg = oracle_mod.chart_second(m.verts, m.tris, h, g, H, n=6)
    for a, b in ((uu, ouu), (uv, ouv), (vv, ovv), (km, okm), (kg, okg)):
        assert np.abs(a - b).max() <= 1e-10 * np.abs(b).max()
    # the chart curvature is the level set's, div(-grad Phi/|grad Phi|)
    S = np.stack([np.stack([H[:, 0], H[:, 1], H[:, 2]], 1), np.stack([H[:, 1], H[:, 3], H[:, 4]], 1),
                  np.stack([H[:, 2], H[:, 4], H[:, 5]], 1)], 1)
    gn = np.linalg.norm(g, axis=1)
    kdiv = -(np.trace(S, axis1=1, axis2=2) * gn ** 2 - np.einsum("ni,nij,nj->n", g, S, g)) / gn ** 3
    assert np.abs(km - kdiv).max() <= 1e-8 * np.abs(kdiv).max()
    # a slightly smoothed unit sphere: mean curvature near 2, Gaussian near 1
    assert 1.8 < km.min() and km.max() < 2.3 and 0.8 < kg.min() and kg.max() < 1.3


def test_gauss_bonnet_on_the_gpu(lsm, oracle_mod, sphere):
    """Gaussian curvature integrated over the charts: 4 pi on the sphere, 0 on
    a torus (Gauss-Bonnet, 2 pi chi)."""
    m, ctx, mesh, x, h, g, H = sphere
    _, _, jac = mesh.chart_frames(8, h, g)
    _, _, _, _, kg = mesh.chart_curvature(8, h, g, H)
    _, _, cw = oracle_mod.simplex_rule(6, 0)
    assert abs(np.sum(np.tile(cw, m.m) * jac * kg) - 4 * np.pi) < 1e-7
    t = synth.torus(1.0, 0.4, 24, 10, 1.0, 0.0, 63)
    mt = ctx.upload(t.verts, t.tris, None, n_gl=6)
    xt, ht, st, stats = mt.solve_charts(order=10, tol=1e-13, precision=lsm.FP64)
    assert stats.n_failed == 0
    _, gt = mt.eval_phi_grad(xt, lsm.FP64)
    Ht = mt.eval_hessian(xt)
    _, _, jt = mt.chart_frames(10, ht, gt)
    _, _, _, _, kt = mt.chart_curvature(10, ht, gt, Ht)
    _, _, cw7 = oracle_mod.simplex_rule(7, 0)
    assert abs(np.sum(np.tile(cw7, t.m) * jt * kt)) < 5e-6


def test_hessian_rejects_sigma_x_mesh(lsm):
    m = synth.cube(1.0, 2)
    ctx = lsm.Context(0)
    mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=3)
    with pytest.raises(lsm.LsmError):
        mesh.eval_hessian(np.zeros((3, 3)))


def test_hessian_with_treecode(lsm, oracle_mod):
    """A mesh above the treecode threshold (graded torus 120 x 32, 276,480
    nodes): the Hessian over the treecode's lists (far pairs through the
    proxies) against the direct sum on the GPU and the oracle on a sample of
    50,000 dense targets; fewer far pairs."""
    m = synth.torus(1.0, 0.3, 120, 32, 20.0, 0.05, 73)
    x = synth.targets_near_surface(m, 50_000, synth.rng(74), 3.0)
    out = {}
    for name, kw in (("tree", {}), ("direct", {"tree_min_sources": -1})):
        ctx = lsm.Context(0, **kw)
        mesh = ctx.upload(m.verts, m.tris, None, n_gl=6)
        ctx.read_stats(reset=True)
        out[name] = (mesh.eval_hessian(x), ctx.read_stats(reset=True))
    (Ht, st_t), (Hd, st_d) = out["tree"], out["direct"]
    scale = np.abs(Hd).max()
    assert np.abs(Ht - Hd).max() <= 1e-7 * scale
    assert st_t["kind_pairs_near"][3] == st_d["kind_pairs_near"][3]
    assert st_t["kind_pairs_far"][3] < 0.5 * st_d["kind_pairs_far"][3]
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, None, 6, 0)
    sel = np.random.default_rng(75).choice(len(x), 100, replace=False)
    _, _, Ho = oracle_mod.phi_grad_hess(y, nw, sg, x[sel])
    assert np.abs(Ht[sel] - Ho).max() <= 1e-7 * scale
