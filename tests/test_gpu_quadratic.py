"""Quadratic (6-node curvilinear) skeleton patches (Sec. 5, quadratic
skeletons) on the GPU against the oracle's quadratic patches.

The oracle evaluates the patch map through the Lagrange basis functions; the
CUDA kernels use the monomial form of the same interpolant, so agreement is
not a shared-code artefact.  Bars as for flat meshes: Phi 1e-12 (FP64 and
float-float) and 1e-7 (mixed); grad Phi 1e-12 / sigma_min and 1e-7 /
sigma_min; chart positions 1e-10 (FP64) and 1e-9 (mixed finished in
float-float); frames 1e-12 relative; Gauss flux 1e-13.
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
    return m


@pytest.fixture(scope="module")
def ctx(lsm):
    return lsm.Context(0)


@pytest.fixture(scope="module")
def sphere(lsm, ctx, oracle_mod):
    q = synth.quadratic_icosphere(2)          # 320 patches, every node on the unit sphere
    mesh = ctx.upload_quadratic(q.verts, q.tris6, n_gl=4)
    src = oracle_mod.sources_quad(q.verts, q.tris6, None, 4, 0)
    return q, mesh, src


def test_straight_edged_patches_equal_the_flat_mesh(lsm, ctx, oracle_mod):
    m = synth.cube(1.0, 3)
    q = synth.quadratic_from_flat(m, 0.5)
    sig = np.full(m.m, 0.15)
    flat = ctx.upload(m.verts, m.tris, sig, n_gl=4, subdiv=1)
    quad = ctx.upload_quadratic(q.verts, q.tris6, sig, n_gl=4, subdiv=1)
    x = synth.targets_uniform(3000, -1.4, 1.4, synth.rng(61))
    pf, gf = flat.eval_phi_grad(x, lsm.FP64)
    pq, gq = quad.eval_phi_grad(x, lsm.FP64)
    assert np.abs(pq - pf).max() < 1e-13 and np.abs(gq - gf).max() < 1e-12
    xf, hf, sf, _ = flat.solve_charts(order=4, tol=1e-12, precision=lsm.FP64)
    xq, hq, sq, _ = quad.solve_charts(order=4, tol=1e-12, precision=lsm.FP64)
    assert np.all(sq & 255 == 0) and np.abs(xq - xf).max() < 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-7), (2, 1e-12)])
def test_curved_sphere_phi_matches_oracle(lsm, oracle_mod, sphere, prec, tol):
    q, mesh, (y, nw, sg) = sphere
    x = synth.targets_uniform(2000, -1.2, 1.2, synth.rng(62))
    po, go = oracle_mod.phi_grad(y, nw, sg, x)
    p, g = mesh.eval_phi_grad(x, prec)
    smin = mesh.info()["sigma_min"]
    assert np.abs(p - po).max() <= tol
    gtol = 1e-12 if prec == 0 else 1e-7
    assert np.abs(g - go).max() <= gtol / smin
    # the resident sigma follows the curved area rule
    geo = oracle_mod.geometry_quad(q.verts, q.tris6, None, 4, 0)
    assert abs(mesh.info()["sigma_min"] - geo["sigma"].min()) < 1e-14
    assert abs(mesh.info()["sigma_max"] - geo["sigma"].max()) < 1e-14


@pytest.mark.parametrize("prec,pos_tol", [(0, 1e-10), (1, 1e-9)])
def test_curved_sphere_charts_frames_flux(lsm, oracle_mod, sphere, prec, pos_tol):
    q, mesh, src = sphere
    order = 4
    n = order // 2 + 2
    x, h, st, stats = mesh.solve_charts(order=order, tol=1e-12, precision=prec)
    assert stats.n_failed == 0 and np.all(st & 255 == 0)
    tri, uv, w = oracle_mod.refined_nodes(q.m, n, np.zeros(q.m))
    x0, hd, sl = oracle_mod.chart_nodes_quad_at(q.verts, q.tris6, tri, uv)
    r = oracle_mod.solve_charts(*src, x0, hd, sl, tol=1e-13, max_iter=40)
    assert np.abs(x - r["x"]).max() < pos_tol
    # frames and flux on the same solved charts and gradient
    _, g = oracle_mod.phi_grad(*src, x)
    xu, xv, jac = mesh.chart_frames(order, h, g)
    ou, ov, oj = oracle_mod.chart_frames_quad_at(q.verts, q.tris6, tri, uv, h, g)
    assert np.abs(xu - ou).max() < 1e-12 * np.abs(ou).max()
    assert np.abs(xv - ov).max() < 1e-12 * np.abs(ov).max()
    assert np.abs(jac - oj).max() < 1e-12 * np.abs(oj).max()
    e_gpu = mesh.gauss_flux(order, x, g, jac, (0.1, -0.05, 0.02))
    e_or = oracle_mod.gauss_flux_w(x, g, oj, w, (0.1, -0.05, 0.02))
    assert abs(e_gpu - e_or) < 1e-13
    assert abs(e_gpu) < 1e-5


def test_curved_refined_charts_match_oracle(lsm, oracle_mod, sphere):
    """Refined charts on quadratic patches keep the parent's curved map."""
    q, mesh, src = sphere
    levels = np.random.default_rng(63).integers(0, 2, q.m)
    tri, uvw = lsm.refined_nodes(4, levels)
    x, h, st, stats = mesh.solve_charts_nodes(tri, uvw, tol=1e-12, precision=lsm.FP64)
    assert np.all(st & 255 == 0)
    x0, hd, sl = oracle_mod.chart_nodes_quad_at(q.verts, q.tris6, tri, uvw[:, :2])
    r = oracle_mod.solve_charts(*src, x0, hd, sl, tol=1e-13, max_iter=40)
    assert np.abs(x - r["x"]).max() < 1e-10


def test_quadratic_torus_with_treecodes(lsm, ctx, oracle_mod):
    """A curved torus above the treecode threshold (7,680 patches, 6x6 rule:
    276,480 sources): mixed and float-float paths with their treecodes
    against the oracle on sampled targets, and a chart solve to 1e-12
    re-evaluated by the oracle."""
    q = synth.quadratic_torus(1.0, 0.3, 120, 32)
    mesh = ctx.upload_quadratic(q.verts, q.tris6, n_gl=6)
    assert mesh.info()["n_sources"] == 276_480
    y, nw, sg = oracle_mod.sources_quad(q.verts, q.tris6, None, 6, 0)
    # targets within 3 sigma of the curved surface: a point of a random patch
    # moved along its pseudonormal
    g = synth.rng(64)
    sel_t = g.integers(0, q.m, 40_000)
    uvs = g.uniform(size=(40_000, 2))
    flip = uvs.sum(1) > 1
    uvs[flip] = 1 - uvs[flip]
    x0, hd, sl = oracle_mod.chart_nodes_quad_at(q.verts, q.tris6, sel_t.astype(np.int32), uvs)
    x = x0 + hd * (g.uniform(-3, 3, 40_000) * sl)[:, None]
    smp = g.choice(40_000, 300, replace=False)
    po, go = oracle_mod.phi_grad(y, nw, sg, x[smp])
    for prec, tol in ((lsm.MIXED, 1e-7), (lsm.FF, 1e-12)):
        p, gr = mesh.eval_phi_grad(torch.from_numpy(x).cuda(), prec)
        assert np.abs(p.cpu().numpy()[smp] - po).max() <= tol
        assert np.abs(gr.cpu().numpy()[smp] - go).max() <= 1e-7 / mesh.info()["sigma_min"]
    xc, h, st, stats = mesh.solve_charts(order=4, tol=1e-12, precision=lsm.MIXED)
    assert stats.n_failed == 0
    sel = g.choice(len(h), 300, replace=False)
    pc, _ = oracle_mod.phi_grad(y, nw, sg, xc[sel])
    assert np.abs(pc - 0.5).max() < 1e-12


def test_inconsistent_edge_nodes_are_rejected(lsm, ctx):
    q = synth.quadratic_icosphere(1)
    t6 = q.tris6.copy()
    # give one patch its own node on an edge its neighbour shares with it
    extra = np.concatenate([q.verts, q.verts[t6[0, 3]][None] * 1.01])
    t6[0, 3] = len(q.verts)
    with pytest.raises(lsm.LsmError) as e:
        ctx.upload_quadratic(extra, t6)
    assert e.value.code == -4
    with pytest.raises(lsm.LsmError):
        lsm.Batch(ctx, [ctx.upload_quadratic(q.verts, q.tris6)])
