"""GPU parity of the mixed path's treecode far field against the FP64 oracle.

The treecode replaces far source tiles by Chebyshev proxies of their tree
nodes; the sum it approximates is the oracle's direct sum over all pairs, so
the bar is the mixed path's: |dPhi| <= 1e-7, |d grad Phi| <= 1e-7 / sigma_min.
Meshes below the default size threshold are pushed onto the treecode with
tree_min_sources=1.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-7


@pytest.fixture(scope="module")
def lsm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as m
    m.load()
    return m


def _eval(lsm, ctx, mesh, x, prec=None):
    phi, grad = mesh.eval_phi_grad(torch.from_numpy(x).cuda(), lsm.MIXED if prec is None else prec)
    return phi.cpu().numpy(), grad.cpu().numpy()


@pytest.fixture(scope="module")
def torus_case(lsm, oracle_mod):
    # graded torus, 120 x 32 cells (7,680 triangles, 276,480 nodes), 6,000
    # targets within 3 sigma
    w = synth.torus_c2(6_000, seed=21, nu=120, nv=32)
    m = w["mesh"]
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 6, 0)
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, w["targets"])
    return dict(w=w, phi=phi_o, grad=grad_o)


def test_torus_tree_matches_oracle(lsm, torus_case):
    w = torus_case["w"]
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    assert mesh.info()["n_sources"] >= 262_144     # above the default threshold
    ctx.read_stats(reset=True)
    phi, grad = _eval(lsm, ctx, mesh, w["targets"])
    st_tree = ctx.read_stats(reset=True)
    assert np.abs(phi - torus_case["phi"]).max() <= TOL32
    assert np.abs(grad - torus_case["grad"]).max() <= TOL32 / m.sigma.min()
    # the direct far field on the same inputs: same answer, more pairs
    ctx_d = lsm.Context(0, tree_min_sources=-1)
    mesh_d = ctx_d.upload(m.verts, m.tris, m.sigma, n_gl=6)
    ctx_d.read_stats(reset=True)
    phi_d, grad_d = _eval(lsm, ctx_d, mesh_d, w["targets"])
    st_dir = ctx_d.read_stats(reset=True)
    assert np.abs(phi_d - torus_case["phi"]).max() <= TOL32
    assert np.abs(phi - phi_d).max() <= TOL32
    # near tiles are the same in both: the treecode only replaces far tiles
    assert st_tree["pairs_near"] == st_dir["pairs_near"]
    assert st_tree["pairs_far"] < st_dir["pairs_far"]


def test_tree_dense_targets_against_direct(lsm):
    """100,000 targets on the same torus (blocks of 256 targets are then
    compact): the treecode against the direct far field, both on the GPU,
    with far fewer pairs."""
    w = synth.torus_c2(100_000, seed=21, nu=120, nv=32)
    m = w["mesh"]
    out = {}
    for name, kw in (("tree", {}), ("direct", {"tree_min_sources": -1})):
        ctx = lsm.Context(0, **kw)
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
        ctx.read_stats(reset=True)
        out[name] = _eval(lsm, ctx, mesh, w["targets"]) + (ctx.read_stats(reset=True),)
    (pt, gt, st_t), (pd, gd, st_d) = out["tree"], out["direct"]
    assert np.abs(pt - pd).max() <= TOL32
    assert np.abs(gt - gd).max() <= TOL32 / m.sigma.min()
    assert st_t["pairs_near"] + st_t["pairs_far"] < 0.6 * (st_d["pairs_near"] + st_d["pairs_far"])


def test_tree_error_falls_with_degree(lsm, torus_case):
    w = torus_case["w"]
    m = w["mesh"]
    errs = []
    for deg in (3, 6, 10):
        ctx = lsm.Context(0, tree_degree=deg, tree_theta=0.45)
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
        phi, _ = _eval(lsm, ctx, mesh, w["targets"])
        errs.append(np.abs(phi - torus_case["phi"]).max())
    assert errs[0] > errs[1] > errs[2], errs
    assert errs[2] <= TOL32


def test_tree_deterministic_and_reused(lsm, torus_case):
    w = torus_case["w"]
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    n0 = ctx.launch_count
    a = _eval(lsm, ctx, mesh, w["targets"])
    n1 = ctx.launch_count
    b = _eval(lsm, ctx, mesh, w["targets"])
    n2 = ctx.launch_count
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # the tree (node boxes level by level, proxy weights) is built by the
    # first call only
    assert (n1 - n0) - (n2 - n1) >= 10


def test_cube_flat_faces_tree(lsm, oracle_mod):
    """Cube faces are planar: oriented node boxes of one face have a zero
    extent across it (raised to 1e-9 of the radius, two points).  Cube
    [-1,1]^3, 16 x 16 squares per face
    (3,072 triangles, 49,152 nodes), sigma = 0.02, 50,000 targets uniform in
    [-1.5,1.5]^3."""
    m = synth.cube(1.0, 16)
    m.sigma = np.full(m.m, 0.02)
    x = synth.targets_uniform(50_000, -1.5, 1.5, synth.rng(31))
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 4, 0)
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, x)
    ctx = lsm.Context(0, tree_min_sources=1)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4)
    ctx.read_stats(reset=True)
    phi, grad = _eval(lsm, ctx, mesh, x)
    st = ctx.read_stats(reset=True)
    assert np.abs(phi - phi_o).max() <= TOL32
    assert np.abs(grad - grad_o).max() <= TOL32 / m.sigma.min()
    # volume targets make wide blocks that few nodes may act on, but proxies
    # act (fewer pairs than the direct sum)
    assert st["pairs_near"] + st["pairs_far"] < len(y) * len(x)


def test_ragged_target_counts_tree(lsm, torus_case):
    """Target counts that leave a partial block, a single target, and a block
    count below the GPU's width (the interaction lists are split)."""
    w = torus_case["w"]
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    for n in (1, 255, 257, 3001):
        phi, grad = _eval(lsm, ctx, mesh, w["targets"][:n])
        assert np.abs(phi - torus_case["phi"][:n]).max() <= TOL32
        assert np.abs(grad - torus_case["grad"][:n]).max() <= TOL32 / m.sigma.min()


def test_chart_solve_with_tree(lsm, oracle_mod):
    """Mixed chart solve on a mesh that uses the treecodes in its mixed sweeps
    and in its float-float record sweep: every node to |Phi - 1/2| < 1e-12,
    re-evaluated by the oracle."""
    w = synth.torus_c2(10, seed=22, nu=120, nv=32)
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    x, h, st, stats = mesh.solve_charts(order=8, tol=1e-12, precision=lsm.MIXED)
    assert stats.n_failed == 0
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 6, 0)
    sel = np.random.default_rng(3).choice(stats.n_nodes, 48, replace=False)
    po, _ = oracle_mod.phi_grad(y, nw, sg, x[sel])
    assert np.abs(po - 0.5).max() < 1e-12


def test_autotune_choice_within_budget(lsm, oracle_mod):
    """The autotuner's choice meets its error budget on its own sample, is no
    slower there than the direct far field, and the mesh then evaluates with
    it: checked against the oracle on a sample of a dense target set."""
    w = synth.torus_c2(100_000, seed=23, nu=120, nv=32)
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    r = mesh.autotune(w["targets"], err_budget=5e-8)
    assert r["candidates"] >= 5 and r["sample_targets"] == 8 * 4096
    assert r["err_phi"] <= 5e-8
    assert r["ms_sample"] <= r["ms_direct"] * 1.05
    # second stage: the near-field radius (within the mixed bound) and the target tile
    assert min(abs(r["cutoff"] - c) for c in (6.4, 6.5, 7.0)) < 1e-12
    assert r["targets_per_block"] in (64, 128, 256)
    phi, grad = _eval(lsm, ctx, mesh, w["targets"])
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 6, 0)
    sel = np.random.default_rng(5).choice(len(w["targets"]), 400, replace=False)
    po, go = oracle_mod.phi_grad(y, nw, sg, w["targets"][sel])
    assert np.abs(phi[sel] - po).max() <= TOL32
    assert np.abs(grad[sel] - go).max() <= TOL32 / m.sigma.min()


def test_autotune_unreachable_budget(lsm, torus_case):
    """A budget below every candidate's error: the most accurate candidate is
    kept, and results stay within the mixed bar."""
    w = torus_case["w"]
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    r = mesh.autotune(w["targets"], err_budget=1e-15)
    assert r["err_phi"] > 1e-15
    phi, _ = _eval(lsm, ctx, mesh, w["targets"])
    assert np.abs(phi - torus_case["phi"]).max() <= TOL32


def test_ff_tree_matches_oracle(lsm, torus_case):
    """Float-float path with its treecode (degree 14, theta 0.45, FP64 proxy
    weights): Phi to the FP64 bar."""
    w = torus_case["w"]
    m = w["mesh"]
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
    phi, grad = _eval(lsm, ctx, mesh, w["targets"], lsm.FF)
    assert np.abs(phi - torus_case["phi"]).max() <= 1e-12
    assert np.abs(grad - torus_case["grad"]).max() <= TOL32 / m.sigma.min()


def test_ff_tree_dense_against_direct(lsm):
    w = synth.torus_c2(100_000, seed=21, nu=120, nv=32)
    m = w["mesh"]
    out = {}
    for name, kw in (("tree", {}), ("direct", {"tree_ff_min_sources": -1})):
        ctx = lsm.Context(0, **kw)
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
        ctx.read_stats(reset=True)
        out[name] = _eval(lsm, ctx, mesh, w["targets"], lsm.FF) + (ctx.read_stats(reset=True),)
    (pt, gt, st_t), (pd, gd, st_d) = out["tree"], out["direct"]
    assert np.abs(pt - pd).max() <= 5e-13
    assert np.abs(gt - gd).max() <= TOL32 / m.sigma.min()
    assert st_t["pairs_near"] == st_d["pairs_near"]
    assert st_t["pairs_far"] < st_d["pairs_far"]


def test_mixed_block_layouts(lsm, torus_case):
    """The mixed kernel with 64 targets per CTA (two threads per target, each
    taking every other pair of sources), 128 (one thread, two sources per
    packed lane pair) and 256 (two targets per thread in the packed lanes):
    all within the mixed bar of the oracle, and smaller target boxes put
    fewer pairs in the near field."""
    w = torus_case["w"]
    m = w["mesh"]
    near = {}
    for blk in (64, 128, 256):
        ctx = lsm.Context(0, mixed_block=blk, tree_degree=8, tree_theta=0.5)
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
        _eval(lsm, ctx, mesh, w["targets"][:4096])    # builds the tree
        ctx.read_stats(reset=True)
        phi, grad = _eval(lsm, ctx, mesh, w["targets"])
        st = ctx.read_stats(reset=True)
        assert np.abs(phi - torus_case["phi"]).max() <= TOL32, blk
        assert np.abs(grad - torus_case["grad"]).max() <= TOL32 / m.sigma.min(), blk
        near[blk] = st["pairs_near"]
    assert near[64] < near[128] < near[256], near
    with pytest.raises(lsm.LsmError):
        lsm.Context(0, mixed_block=32)


def test_ff_block_sizes(lsm, torus_case):
    """The float-float kernel with 64 targets per CTA (two threads per target,
    the default) and with 128: both within the FP64 bar of the oracle, within
    5e-13 of each other, and the smaller target boxes evaluate fewer pairs."""
    w = torus_case["w"]
    m = w["mesh"]
    out = {}
    for blk in (64, 128):
        ctx = lsm.Context(0, ff_block=blk)
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
        _eval(lsm, ctx, mesh, w["targets"][:4096], lsm.FF)    # builds the tree
        ctx.read_stats(reset=True)
        phi, grad = _eval(lsm, ctx, mesh, w["targets"], lsm.FF)
        st = ctx.read_stats(reset=True)
        assert np.abs(phi - torus_case["phi"]).max() <= 1e-12, blk
        assert np.abs(grad - torus_case["grad"]).max() <= TOL32 / m.sigma.min(), blk
        out[blk] = (phi, st["pairs_near"] + st["pairs_far"])
    assert np.abs(out[64][0] - out[128][0]).max() <= 5e-13
    assert out[64][1] < out[128][1], (out[64][1], out[128][1])
    with pytest.raises(lsm.LsmError):
        lsm.Context(0, ff_block=96)


def test_oriented_grids_and_full_grids(lsm, torus_case):
    """Oriented per-axis grids with the degree ladder (the default) and full
    axis-aligned (p+1)^3 grids of one degree: both within the mixed bar and
    the float-float bar against the oracle."""
    w = torus_case["w"]
    m = w["mesh"]
    for grid in (1, 2):
        ctx = lsm.Context(0, tree_grid=grid)
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
        phi, grad = _eval(lsm, ctx, mesh, w["targets"])
        assert np.abs(phi - torus_case["phi"]).max() <= TOL32, grid
        assert np.abs(grad - torus_case["grad"]).max() <= TOL32 / m.sigma.min(), grid
        phi, _ = _eval(lsm, ctx, mesh, w["targets"], lsm.FF)
        assert np.abs(phi - torus_case["phi"]).max() <= 1e-12, grid



def test_ff_target_clusters(lsm, oracle_mod):
    """Target clusters of the float-float treecode (4,096 targets each, the
    default): nodes far from a cluster act on its Chebyshev grid and the
    targets interpolate.  Against the same tree without clusters: within
    5e-13 on Phi; against the oracle on sampled targets: the float-float bar;
    and a chart solve whose record sweeps use clusters stays below 1e-12
    re-evaluated by the oracle.  (At this target density the clusters save
    little; the full-size test checks that they cut the pairs there.)"""
    w = synth.torus_c2(200_000, seed=25, nu=120, nv=32)
    m = w["mesh"]
    out = {}
    for name, kw in (("clusters", {}), ("plain", {"tree_ff_cluster": -1})):
        ctx = lsm.Context(0, **kw)
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=6)
        _eval(lsm, ctx, mesh, w["targets"][:4096], lsm.FF)    # builds the tree
        ctx.read_stats(reset=True)
        out[name] = _eval(lsm, ctx, mesh, w["targets"], lsm.FF) + (ctx.read_stats(reset=True), ctx, mesh)
    (pc, gc, sc, ctx_c, mesh_c), (pp, gp, sp, _, _) = out["clusters"], out["plain"]
    assert np.abs(pc - pp).max() <= 5e-13
    assert np.abs(gc - gp).max() <= TOL32 / m.sigma.min()
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 6, 0)
    sel = np.random.default_rng(26).choice(len(w["targets"]), 300, replace=False)
    po, _ = oracle_mod.phi_grad(y, nw, sg, w["targets"][sel])
    assert np.abs(pc[sel] - po).max() <= 1e-12
    x, h, st, stats = mesh_c.solve_charts(order=8, tol=1e-12, precision=lsm.MIXED)
    assert stats.n_failed == 0
    sel = np.random.default_rng(27).choice(len(h), 300, replace=False)
    pcn, _ = oracle_mod.phi_grad(y, nw, sg, x[sel])
    assert np.abs(pcn - 0.5).max() < 1e-12
