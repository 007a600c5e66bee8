"""GPU parity of refined charts (Sec. 3.4): charts solved at the nodes of
triangles split 1 -> 4 (per-triangle levels, non-conforming), their frames
and the Gauss flux at explicit nodes, against the oracle on the same nodes.
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


@pytest.fixture(scope="module")
def refined(lsm, oracle_mod):
    """Icosphere level 1 (80 triangles), 4x4 sources, order 4 (4x4 chart rule),
    random per-triangle levels 0..2."""
    m = synth.icosphere(1)
    levels = np.random.default_rng(81).integers(0, 3, m.m).astype(np.int32)
    tri, uvw = lsm.refined_nodes(4, levels)
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, None, n_gl=4)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, None, 4, 0)
    return m, levels, tri, uvw, ctx, mesh, (y, nw, sg)


def test_refined_solve_matches_oracle(lsm, oracle_mod, refined):
    m, levels, tri, uvw, ctx, mesh, (y, nw, sg) = refined
    x, h, st, stats = mesh.solve_charts_nodes(tri, uvw, tol=1e-13, precision=lsm.FP64)
    assert stats.n_failed == 0 and stats.n_nodes == len(tri)
    x0, hd, sl = oracle_mod.chart_nodes_at(m.verts, m.tris, tri, uvw[:, :2])
    r = oracle_mod.solve_charts(y, nw, sg, x0, hd, sl, tol=1e-13, max_iter=40)
    assert (r["status"] == 0).all()
    assert np.abs(x - r["x"]).max() < 1e-10
    assert np.abs(h - r["h"]).max() < 1e-10


def test_refined_frames_and_flux_match_oracle(lsm, oracle_mod, refined):
    m, levels, tri, uvw, ctx, mesh, (y, nw, sg) = refined
    x, h, st, stats = mesh.solve_charts_nodes(tri, uvw, tol=1e-13, precision=lsm.FP64)
    _, g = mesh.eval_phi_grad(x, lsm.FP64)
    xu, xv, jac = mesh.chart_frames_nodes(tri, uvw, h, g)
    ou, ov, oj = oracle_mod.chart_frames_at(m.verts, m.tris, tri, uvw[:, :2], h, g)
    assert np.abs(xu - ou).max() <= 1e-12 * np.abs(ou).max()
    assert np.abs(jac - oj).max() <= 1e-12 * np.abs(oj).max()
    x0 = (0.05, -0.1, 0.02)
    e = mesh.gauss_flux_nodes(tri, uvw, x, g, jac, x0)
    eo = oracle_mod.gauss_flux_w(x, g, jac, uvw[:, 2], x0)
    assert abs(e - eo) <= 1e-13
    # non-conforming refinement keeps the charts closed: the error is the
    # quadrature's, between the all-coarse and all-fine ones (order 4 on this
    # sphere: 2.2e-7 unrefined, 2.4e-12 at level 2)
    assert abs(e) < 2.2e-7


def test_refined_mixed_solve_with_treecodes(lsm, oracle_mod):
    """Refinement on a mesh above the treecode threshold, mixed sweeps then
    float-float, to 1e-12 (oracle re-evaluates a sample)."""
    m = synth.torus(1.0, 0.3, 120, 32, 20.0, 0.05, 82)
    levels = (np.random.default_rng(83).random(m.m) < 0.2).astype(np.int32)
    tri, uvw = lsm.refined_nodes(4, levels)
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, None, n_gl=6)
    x, h, st, stats = mesh.solve_charts_nodes(tri, uvw, tol=1e-12, precision=lsm.MIXED)
    assert stats.n_failed == 0
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, None, 6, 0)
    sel = np.random.default_rng(84).choice(len(tri), 40, replace=False)
    po, _ = oracle_mod.phi_grad(y, nw, sg, x[sel])
    assert np.abs(po - 0.5).max() < 1e-12


def test_refined_nodes_reject_bad_triangles(lsm, refined):
    m, levels, tri, uvw, ctx, mesh, _ = refined
    bad = tri.copy()
    bad[3] = m.m
    with pytest.raises(lsm.LsmError):
        mesh.solve_charts_nodes(bad, uvw)


def test_flux_per_triangle_matches_oracle(lsm, oracle_mod, refined):
    """The Gauss flux split by skeleton triangle (on refined, non-conforming
    node sets) against the oracle's flux over each triangle's nodes, and the
    total against lsm_gauss_flux_nodes."""
    m, levels, tri, uvw, ctx, mesh, (y, nw, sg) = refined
    x, h, st, stats = mesh.solve_charts_nodes(tri, uvw, tol=1e-13, precision=lsm.FP64)
    _, g = mesh.eval_phi_grad(x, lsm.FP64)
    _, _, jac = mesh.chart_frames_nodes(tri, uvw, h, g)
    x0 = (0.05, -0.1, 0.02)
    per = mesh.flux_per_triangle(tri, uvw, x, g, jac, x0)
    for j in range(m.m):
        sel = tri == j
        ref = oracle_mod.gauss_flux_w(x[sel], g[sel], jac[sel], uvw[sel, 2], x0) - 1.0
        assert abs(per[j] - ref) < 1e-14
    tot = mesh.gauss_flux_nodes(tri, uvw, x, g, jac, x0)
    assert abs((1.0 + per.sum()) - tot) < 1e-13


def test_adaptive_refinement_driver(lsm):
    """lsm_refine_adaptive on a sphere with sharp Gaussian bumps.  Its first
    decision is recomputed here from lsm_flux_per_triangle at levels 0 and 1
    (a triangle is refined exactly when its flux moves by more than the
    tolerance); the charts at the levels it returns close the Gauss flux
    better than the unrefined charts, with fewer nodes than refining every
    triangle to the same maximum level."""
    m = synth.bumped_icosphere(2, 12, 7)
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4)
    x0 = (0.03, -0.02, 0.05)
    order = 2

    def solve(lv):
        tri, uvw = lsm.refined_nodes(order, lv)
        x, h, st, stats = mesh.solve_charts_nodes(tri, uvw, tol=1e-12, precision=lsm.MIXED)
        assert stats.n_failed == 0
        _, g = mesh.eval_phi_grad(x, lsm.FF)
        _, _, jac = mesh.chart_frames_nodes(tri, uvw, h, g)
        return tri, uvw, x, g, jac

    def per_tri(lv):
        return mesh.flux_per_triangle(*solve(lv), x0)

    def eps(lv):
        tri, uvw, x, g, jac = solve(lv)
        return abs(mesh.gauss_flux_nodes(tri, uvw, x, g, jac, x0)), len(tri)

    z = np.zeros(m.m, dtype=np.int32)
    est = np.abs(per_tri(z + 1) - per_tri(z))
    srt = np.sort(est)
    k = len(srt) // 2
    tol = float(0.5 * (srt[k - 1] + srt[k]))   # between two estimates: no tie at the tolerance
    levels, rounds = mesh.refine_adaptive(order=order, flux_tol=tol, max_level=2, x0=x0)
    assert rounds >= 1 and levels.min() >= 0 and levels.max() <= 2
    # first round: refined exactly where the estimate exceeds the tolerance
    assert np.array_equal(levels > 0, est > tol)
    e0, n0 = eps(z)
    ea, na = eps(levels.astype(np.int32))
    e2, n2 = eps(z + 2)
    assert ea < e0, (e0, ea, e2)
    assert na < n2
