"""GPU parity of the target-dependent width sigma(x) (Sec. 2.3, eq. sigma2)
against the oracle: sigma(x) and its gradient, Phi and grad Phi with the
grad-sigma term in all three precisions, the chart solve, and the treecode
far field on a sigma(x) mesh.  Tolerances as for per-triangle sigma."""
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
def graded(lsm, oracle_mod):
    """Graded torus, 48 x 16 cells (1,536 triangles, 6x6 sources = 55,296
    nodes), sigma(x) with the defaults; 3,000 targets within 3 sigma_j."""
    m = synth.torus(1.0, 0.3, 48, 16, 8.0, 0.05, 51)
    m.sigma = None
    x = synth.targets_near_surface(synth.torus(1.0, 0.3, 48, 16, 8.0, 0.05, 51), 3000, synth.rng(52), 3.0)
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    s0 = oracle_mod.sigma0_default(dmax)
    sg, gs = oracle_mod.sigma_x(c, sj, s0, x)
    y, nw, _ = oracle_mod.sources(m.verts, m.tris, sj, 6, 0)
    phi, grad = oracle_mod.phi_grad_sigx(y, nw, x, sg, gs)
    return dict(m=m, x=x, c=c, sj=sj, s0=s0, sg=sg, gs=gs, y=y, nw=nw, phi=phi, grad=grad)


def test_sigma_x_matches_oracle(lsm, graded):
    ctx = lsm.Context(0)
    mesh = ctx.upload_sigma_x(graded["m"].verts, graded["m"].tris, n_gl=6)
    assert abs(mesh.sigma0 - graded["s0"]) < 1e-15 * graded["s0"]
    sg, gs = mesh.eval_sigma(graded["x"])
    assert np.abs(sg - graded["sg"]).max() <= 1e-13 * graded["sg"].max()
    assert np.abs(gs - graded["gs"]).max() <= 1e-12 * np.abs(graded["gs"]).max()


@pytest.mark.parametrize("prec,tphi,tgrad", [("FP64", 1e-12, 1e-12), ("FF", 1e-12, 1e-7), ("MIXED", 1e-7, 1e-7)])
def test_phi_grad_sigma_x_matches_oracle(lsm, graded, prec, tphi, tgrad):
    ctx = lsm.Context(0)
    mesh = ctx.upload_sigma_x(graded["m"].verts, graded["m"].tris, n_gl=6)
    phi, grad = mesh.eval_phi_grad(graded["x"], getattr(lsm, prec))
    smin = graded["sj"].min()
    assert np.abs(phi - graded["phi"]).max() <= tphi
    assert np.abs(grad - graded["grad"]).max() <= tgrad / smin


@pytest.mark.parametrize("prec,block", [("FF", 64), ("FF", 128), ("MIXED", 64), ("MIXED", 128), ("MIXED", 256)])
def test_phi_grad_sigma_x_target_tiles(lsm, graded, prec, block):
    """Every target-tile layout of the float-float (64, 128 targets per CTA)
    and mixed (64, 128, 256) kernels in sigma(x) mode against the oracle."""
    opt = {"ff_block": block} if prec == "FF" else {"mixed_block": block}
    ctx = lsm.Context(0, **opt)
    mesh = ctx.upload_sigma_x(graded["m"].verts, graded["m"].tris, n_gl=6)
    phi, grad = mesh.eval_phi_grad(graded["x"], getattr(lsm, prec))
    smin = graded["sj"].min()
    tphi = 1e-12 if prec == "FF" else 1e-7
    assert np.abs(phi - graded["phi"]).max() <= tphi
    assert np.abs(grad - graded["grad"]).max() <= 1e-7 / smin


def test_sigma_x_equal_widths_reduce_to_constant(lsm):
    """Cube: every triangle has the same D_j, so sigma(x) is constant and the
    results equal the per-triangle mesh's with that sigma.  The float-float
    kernel's gradient is FP32 with compensated sums (it only steers Newton),
    and the two meshes run it on differently sized target blocks, so its bar
    is the mixed one."""
    m = synth.cube(1.0, 4)
    ctx = lsm.Context(0)
    mx = ctx.upload_sigma_x(m.verts, m.tris, n_gl=4, subdiv=1)
    sig = 0.5 * np.sqrt(2) / 2.5
    mc = ctx.upload(m.verts, m.tris, np.full(m.m, sig), n_gl=4, subdiv=1)
    x = synth.targets_uniform(2000, -1.5, 1.5, synth.rng(53))
    for prec, tol, gtol in ((lsm.FP64, 1e-13, 1e-11), (lsm.FF, 1e-13, 1e-7), (lsm.MIXED, 5e-8, 5e-6)):
        p1, g1 = mx.eval_phi_grad(x, prec)
        p0, g0 = mc.eval_phi_grad(x, prec)
        assert np.abs(p1 - p0).max() <= tol
        assert np.abs(g1 - g0).max() <= gtol / sig


def test_sigma_x_chart_solve(lsm, oracle_mod, graded):
    """Charts with sigma(x): mixed sweeps then float-float, to 1e-12; nodes
    against the oracle's sigma(x) Newton, and Phi(x) = 1/2 re-evaluated."""
    m = graded["m"]
    ctx = lsm.Context(0)
    mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=6)
    x, h, st, stats = mesh.solve_charts(order=4, tol=1e-12, precision=lsm.MIXED)
    assert stats.n_failed == 0
    x0, hd, _ = oracle_mod.chart_nodes(m.verts, m.tris, graded["sj"], 4)
    sel = np.random.default_rng(54).choice(len(x0), 60, replace=False)
    r = oracle_mod.solve_charts_sigx(graded["y"], graded["nw"], graded["c"], graded["sj"], graded["s0"], x0[sel],
                                     hd[sel], np.repeat(graded["sj"], 16)[sel], tol=1e-13, max_iter=30)
    assert (r["status"] == 0).all()
    assert np.abs(x[sel] - r["x"]).max() < 1e-9
    sg, gs = oracle_mod.sigma_x(graded["c"], graded["sj"], graded["s0"], x[sel])
    po, _ = oracle_mod.phi_grad_sigx(graded["y"], graded["nw"], x[sel], sg, gs)
    assert np.abs(po - 0.5).max() < 1e-12


def test_sigma_x_with_treecodes(lsm, oracle_mod):
    """A sigma(x) mesh above the treecode threshold (graded torus 120 x 32,
    276,480 nodes): mixed and float-float evaluations against the oracle on a
    sample of 100,000 dense targets."""
    m = synth.torus(1.0, 0.3, 120, 32, 20.0, 0.05, 55)
    x = synth.targets_near_surface(m, 100_000, synth.rng(56), 3.0)
    ctx = lsm.Context(0)
    mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=6)
    assert mesh.info()["n_sources"] >= 262_144
    pm, gm = mesh.eval_phi_grad(x, lsm.MIXED)
    pf, gf = mesh.eval_phi_grad(x, lsm.FF)
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    sel = np.random.default_rng(57).choice(len(x), 200, replace=False)
    sg, gs = oracle_mod.sigma_x(c, sj, oracle_mod.sigma0_default(dmax), x[sel])
    y, nw, _ = oracle_mod.sources(m.verts, m.tris, sj, 6, 0)
    po, go = oracle_mod.phi_grad_sigx(y, nw, x[sel], sg, gs)
    assert np.abs(pm[sel] - po).max() <= 1e-7
    assert np.abs(pf[sel] - po).max() <= 1e-12
    assert np.abs(gm[sel] - go).max() <= 1e-7 / sj.min()


def test_sigma_x_target_clusters(lsm, oracle_mod):
    """Target clusters in sigma(x) mode (the float-float treecode's 4,096-target
    clusters, and the mixed treecode's, here of 2,048), whose near
    width is their largest target sigma: against the same trees without
    clusters, Phi within 5e-13 (float-float) and 1e-8 (mixed), the gradients
    within the paths' bars, and the float-float bar against the oracle on
    sampled targets."""
    m = synth.torus(1.0, 0.3, 120, 32, 20.0, 0.05, 55)
    x = synth.targets_near_surface(m, 100_000, synth.rng(58), 3.0)
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    smin = sj.min()
    out = {}
    for name, kw in (("clusters", {"tree_cluster": 2048}), ("plain", {"tree_ff_cluster": -1, "tree_cluster": -1})):
        ctx = lsm.Context(0, **kw)
        mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=6)
        mesh.eval_phi_grad(x[:4096], lsm.FF)       # builds the trees
        mesh.eval_phi_grad(x[:4096], lsm.MIXED)
        ctx.read_stats(reset=True)
        pf, gf = mesh.eval_phi_grad(x, lsm.FF)
        far = ctx.read_stats(reset=True)["kind_pairs_far"][1]
        pm, gm = mesh.eval_phi_grad(x, lsm.MIXED)
        out[name] = (pf, gf, pm, gm, far)
        mesh.free()
        ctx.close()
    (pf, gf, pm, gm, far_c), (pf0, gf0, pm0, gm0, far_p) = out["clusters"], out["plain"]
    assert np.abs(pf - pf0).max() <= 5e-13
    assert np.abs(gf - gf0).max() <= 1e-7 / smin
    assert np.abs(pm - pm0).max() <= 1e-8
    assert np.abs(gm - gm0).max() <= 1e-7 / smin
    assert far_c != far_p, (far_c, far_p)   # the clusters' grids took part of the far field
    sel = np.random.default_rng(59).choice(len(x), 100, replace=False)
    sg, gs = oracle_mod.sigma_x(c, sj, oracle_mod.sigma0_default(dmax), x[sel])
    y, nw, _ = oracle_mod.sources(m.verts, m.tris, sj, 6, 0)
    po, go = oracle_mod.phi_grad_sigx(y, nw, x[sel], sg, gs)
    assert np.abs(pf[sel] - po).max() <= 1e-12
    assert np.abs(pm[sel] - po).max() <= 1e-7


def test_sigma_x_mesh_rejected_by_batch_and_noalloc(lsm):
    m = synth.cube(1.0, 2)
    ctx = lsm.Context(0)
    mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=3)
    with pytest.raises(lsm.LsmError):
        lsm.Batch(ctx, [mesh])
    import ctypes
    x = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    phi = torch.empty(4, dtype=torch.float64, device="cuda")
    rc = ctx._L.lsm_eval_phi_grad_noalloc(mesh._h, ctypes.c_void_p(x.data_ptr()), 4,
                                          ctypes.c_void_p(phi.data_ptr()), None, lsm.FP64, None)
    assert rc != 0
