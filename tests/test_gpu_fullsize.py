"""Full-size parity, in the launch configuration bench.py times.

Graded torus, 30,720 triangles, Duffy 6x6 sources (1,105,920 nodes), 1e6
targets within 3 sigma, order-8 chart nodes (1,105,920) to |Phi - 1/2| <
1e-12: seeded samples of 10,000 targets and 10,000 chart nodes against the
FP64 oracle computed one by one.
Bumped icosphere, level 8 (1,310,720 triangles, 20,971,520 nodes): a
1e5-target evaluation against the float-float path at every target, the FP64
direct sum on 10,240 targets and the oracle on 1,000.
The same torus with the paper's sigma(x): 1,000 targets and 1,000 chart
nodes against the oracle.
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
def torus(lsm, oracle_mod):
    w = synth.torus_c2(1_000_000)
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    src = oracle_mod.sources(m.verts, m.tris, m.sigma, 6, 0)
    return w, ctx, mesh, src


def test_torus_full_evaluation_sampled(lsm, oracle_mod, torus):
    w, ctx, mesh, (y, nw, sg) = torus
    m = w["mesh"]
    x = torch.from_numpy(w["targets"]).cuda()
    sel = np.random.default_rng(7).choice(len(w["targets"]), 10_000, replace=False)
    po, go = oracle_mod.phi_grad(y, nw, sg, w["targets"][sel])
    for prec, tol, gtol in ((lsm.MIXED, 1e-7, 1e-7), (lsm.FF, 1e-12, 1e-7)):
        phi, grad = mesh.eval_phi_grad(x, prec)
        p = phi.cpu().numpy()[sel]
        g = grad.cpu().numpy()[sel]
        assert np.abs(p - po).max() <= tol
        assert np.abs(g - go).max() <= gtol / m.sigma.min()


def test_torus_oriented_trees_against_first_design(lsm, oracle_mod, torus):
    """The default trees (oriented per-axis grids, degree ladder, shape-aware
    opening rule) against the first design (axis-aligned (p+1)^3 grids, one
    degree, |x - c| >= r / theta; mixed (8, 0.4), float-float (13, 0.4)) on
    the full torus: both within the bars on sampled targets, and the default
    evaluates fewer far pairs in both paths."""
    w, ctx, mesh, (y, nw, sg) = torus
    m = w["mesh"]
    x = torch.from_numpy(w["targets"]).cuda()
    sel = np.random.default_rng(17).choice(len(w["targets"]), 64, replace=False)
    po, _ = oracle_mod.phi_grad(y, nw, sg, w["targets"][sel])
    ctx_old = lsm.Context(0, tree_grid=2, tree_degree=8, tree_theta=0.4, tree_ff_degree=13, tree_ff_theta=0.4)
    mesh_old = ctx_old.upload(m.verts, m.tris, m.sigma, n_gl=6)
    far = {}
    for name, c, me in (("new", ctx, mesh), ("old", ctx_old, mesh_old)):
        for prec, tol in ((lsm.MIXED, 1e-7), (lsm.FF, 1e-12)):
            me.eval_phi_grad(x[:4096], prec)   # builds the tree
            c.read_stats(reset=True)
            phi, _ = me.eval_phi_grad(x, prec)
            far[name, prec] = c.read_stats(reset=True)["pairs_far"]
            assert np.abs(phi.cpu().numpy()[sel] - po).max() <= tol, (name, prec)
    assert far["new", lsm.MIXED] < far["old", lsm.MIXED], far
    assert far["new", lsm.FF] < 0.85 * far["old", lsm.FF], far


def test_torus_float_float_against_fp64_path(lsm, torus):
    """The float-float path (with its treecode) against the FP64 path (direct
    sums on the FP64 pipes) on 1,024 sampled targets of the full torus: within
    1e-13 everywhere (about 6e-14 measured, mostly the treecode's
    interpolation; the direct float-float sum stays within 1e-14).  A
    float-pair representation of absolute positions, a tile centre off by
    its pair's rounding, a tile spanning a jump of the Morton curve, or a
    first-order-only refinement of 1/|r| each left single targets 1e-13 to
    7e-13 off."""
    w, ctx, mesh, _ = torus
    sel = np.random.default_rng(7).choice(len(w["targets"]), 1024, replace=False)
    xs = torch.from_numpy(w["targets"][sel]).cuda()
    pf, _ = mesh.eval_phi_grad(xs, lsm.FF)
    pd, _ = mesh.eval_phi_grad(xs, lsm.FP64)
    assert (pf - pd).abs().max().item() <= 1e-13
    info = mesh.info()
    # tiles are cut at jumps of the Morton curve: a few percent more tiles
    full = -(-info["n_sources"] // 128)
    assert full <= info["n_tiles"] <= 1.1 * full


def test_torus_target_clusters_cut_far_pairs(lsm, torus):
    """At the bench's density (10^6 targets) the float-float treecode's target
    clusters take the far nodes of each 4,096-target cluster onto its grid:
    fewer far pairs than the same tree without clusters, Phi within 5e-13."""
    w, ctx, mesh, _ = torus
    m = w["mesh"]
    x = torch.from_numpy(w["targets"]).cuda()
    ctx_p = lsm.Context(0, tree_ff_cluster=-1)
    mesh_p = ctx_p.upload(m.verts, m.tris, m.sigma, n_gl=6)
    far = {}
    phi = {}
    for name, c, me in (("clusters", ctx, mesh), ("plain", ctx_p, mesh_p)):
        me.eval_phi_grad(x[:4096], lsm.FF)
        c.read_stats(reset=True)
        phi[name], _ = me.eval_phi_grad(x, lsm.FF)
        far[name] = c.read_stats(reset=True)["kind_pairs_far"][1]
    assert (phi["clusters"] - phi["plain"]).abs().max().item() <= 5e-13
    assert far["clusters"] < 0.95 * far["plain"], far
    mesh_p.free()
    ctx_p.close()


def test_torus_full_chart_solve_sampled(lsm, oracle_mod, torus):
    w, ctx, mesh, (y, nw, sg) = torus
    x, h, st, stats = mesh.solve_charts(order=8, tol=1e-12, precision=lsm.MIXED, device_out=True)
    assert stats.n_nodes == 1_105_920 and stats.n_failed == 0
    assert bool((st & 255 == 0).all())
    sel = np.random.default_rng(8).choice(stats.n_nodes, 10_000, replace=False)
    po, _ = oracle_mod.phi_grad(y, nw, sg, x.cpu().numpy()[sel])
    assert np.abs(po - 0.5).max() < 1e-12


def test_torus_newton_tree(lsm, oracle_mod, torus):
    """The mixed Newton sweeps' own coarser treecode (degree 5, theta 0.5, the
    default) against the same solve on the mesh's mixed treecode
    (newton_tree_degree=-1): no failed node, the same nodes to 1e-11, fewer
    mixed far pairs, and the oracle's |Phi - 1/2| below 1e-12 at 2,000
    sampled nodes of the default solve."""
    w, ctx, mesh, (y, nw, sg) = torus
    m = w["mesh"]
    ctx_p = lsm.Context(0, newton_tree_degree=-1)
    mesh_p = ctx_p.upload(m.verts, m.tris, m.sigma, n_gl=6)
    out = {}
    for name, c, me in (("newton_tree", ctx, mesh), ("mesh_tree", ctx_p, mesh_p)):
        me.solve_charts(order=4, tol=1e-12, precision=lsm.MIXED, device_out=True)   # builds the trees
        c.read_stats(reset=True)
        x, h, st, stats = me.solve_charts(order=8, tol=1e-12, precision=lsm.MIXED, device_out=True)
        out[name] = (x, stats, c.read_stats(reset=True)["kind_pairs_far"][0])
    (xn, sn, fn), (xp, sp, fp) = out["newton_tree"], out["mesh_tree"]
    assert sn.n_failed == 0 and sp.n_failed == 0
    assert (xn - xp).abs().max().item() < 1e-11
    assert fn < 0.9 * fp, (fn, fp)
    sel = np.random.default_rng(62).choice(sn.n_nodes, 2000, replace=False)
    po, _ = oracle_mod.phi_grad(y, nw, sg, xn.cpu().numpy()[sel])
    assert np.abs(po - 0.5).max() < 1e-12
    mesh_p.free()
    ctx_p.close()


def test_icosphere_full_evaluation_sampled(lsm, oracle_mod):
    """The 2.1e7-node bumped icosphere, mixed path with its treecode at 1e5
    targets, against: the float-float path at all 1e5 targets, the FP64
    direct sum on 10,240 targets (four runs of 2,560 consecutive targets in
    Morton order, so that its blocks are as compact as the full set's), and
    the FP64 oracle on 1,000 targets.  The float-float path is also held to
    the FP64 direct sum there (1e-12)."""
    from paper_1909_13356_gb300 import shard
    w = synth.icosphere_c3(n_targets=100_000)
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4)
    assert mesh.info()["n_sources"] == 20_971_520
    x = torch.from_numpy(w["targets"]).cuda()
    phi, grad = mesh.eval_phi_grad(x, lsm.MIXED)
    pff, gff = mesh.eval_phi_grad(x, lsm.FF)
    assert (phi - pff).abs().max().item() <= 1e-7
    assert (grad - gff).abs().max().item() <= 1e-7 / m.sigma.min()
    order = np.argsort(shard.morton_keys(w["targets"]), kind="stable")
    starts = [k * 25_000 + 256 for k in range(4)]
    sel = np.concatenate([order[s0:s0 + 2560] for s0 in starts])
    sel_d = torch.from_numpy(sel).cuda()
    p64, g64 = mesh.eval_phi_grad(x[sel_d], lsm.FP64)
    assert (phi[sel_d] - p64).abs().max().item() <= 1e-7
    assert (grad[sel_d] - g64).abs().max().item() <= 1e-7 / m.sigma.min()
    assert (pff[sel_d] - p64).abs().max().item() <= 1e-12
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 4, 0)
    so = np.random.default_rng(9).choice(len(w["targets"]), 1000, replace=False)
    po, go = oracle_mod.phi_grad(y, nw, sg, w["targets"][so])
    assert np.abs(phi.cpu().numpy()[so] - po).max() <= 1e-7
    assert np.abs(grad.cpu().numpy()[so] - go).max() <= 1e-7 / m.sigma.min()
    assert np.abs(pff.cpu().numpy()[so] - po).max() <= 1e-12


def test_torus_sigma_x_full_sampled(lsm, oracle_mod):
    """The bench's sigma(x) leg at its full size: the graded torus with the
    paper's target-dependent width (eq. sigma2) in place of per-triangle
    sigma, 10^6 targets, mixed and float-float evaluations against the oracle
    (sigma(x), grad sigma and Phi, grad Phi in FP64, one target at a time) on
    1,000 sampled targets, and the order-8 chart solve to |Phi - 1/2| <
    1e-12 re-evaluated by the oracle at 1,000 sampled nodes."""
    w = synth.torus_c2(1_000_000)
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload_sigma_x(m.verts, m.tris, n_gl=6)
    x = torch.from_numpy(w["targets"]).cuda()
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    s0 = oracle_mod.sigma0_default(dmax)
    y, nw, _ = oracle_mod.sources(m.verts, m.tris, sj, 6, 0)
    sel = np.random.default_rng(60).choice(len(w["targets"]), 1000, replace=False)
    sg, gs = oracle_mod.sigma_x(c, sj, s0, w["targets"][sel])
    po, go = oracle_mod.phi_grad_sigx(y, nw, w["targets"][sel], sg, gs)
    for prec, tol in ((lsm.MIXED, 1e-7), (lsm.FF, 1e-12)):
        phi, grad = mesh.eval_phi_grad(x, prec)
        assert np.abs(phi.cpu().numpy()[sel] - po).max() <= tol
        assert np.abs(grad.cpu().numpy()[sel] - go).max() <= 1e-7 / sj.min()
    xs, h, st, stats = mesh.solve_charts(order=8, tol=1e-12, precision=lsm.MIXED, device_out=True)
    assert stats.n_nodes == 1_105_920 and stats.n_failed == 0
    sel = np.random.default_rng(61).choice(stats.n_nodes, 1000, replace=False)
    xn = xs.cpu().numpy()[sel]
    sg, gs = oracle_mod.sigma_x(c, sj, s0, xn)
    pn, _ = oracle_mod.phi_grad_sigx(y, nw, xn, sg, gs)
    assert np.abs(pn - 0.5).max() < 1e-12
    mesh.free()
    ctx.close()
