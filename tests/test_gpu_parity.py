"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element on the same seeded inputs.

Tolerances (stated by the workloads, and derived where they are silent):
  FP64 path  |dPhi| <= 1e-12,  |d grad Phi| <= 1e-12 / sigma_min
  mixed path |dPhi| <= 1e-7,   |d grad Phi| <= 1e-7 / sigma_min
  chart node positions: FP64 <= 1e-10, mixed (finished with FP64 steps) <= 1e-9
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32 = 1e-7


@pytest.fixture(scope="module")
def lsm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as m
    m.load()
    return m


@pytest.fixture(scope="module")
def ctx(lsm):
    return lsm.Context(0)


def _oracle_sources(oracle_mod, mesh, n, subdiv=0, sigma=None):
    return oracle_mod.sources(mesh.verts, mesh.tris, mesh.sigma if sigma is None else sigma, n, subdiv)


def _check(phi, grad, phi_o, grad_o, tol, smin):
    ep = np.abs(phi - phi_o).max()
    eg = np.abs(grad - grad_o).max()
    assert ep <= tol, f"Phi error {ep:.3e} > {tol:.1e}"
    assert eg <= tol / smin, f"grad error {eg:.3e} > {tol / smin:.1e}"
    return ep, eg


@pytest.fixture(scope="module")
def cube_case(oracle_mod, ctx):
    w = synth.cube_c1(10_000)
    m = w["mesh"]
    y, nw, sg = _oracle_sources(oracle_mod, m, 4, 1)
    x = w["targets"]
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, x)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4, subdiv=1)
    return dict(w=w, x=x, phi=phi_o, grad=grad_o, mesh=mesh)


def test_cube_fp64_matches_oracle(lsm, cube_case):
    """Cube, 192 triangles, 4x4 rule on 4 children (12,288 nodes), 10,000
    targets in [-1.5,1.5]^3, FP64 path."""
    c = cube_case
    assert c["mesh"].info()["n_sources"] == 12_288
    phi, grad = c["mesh"].eval_phi_grad(c["x"], lsm.FP64)
    _check(phi, grad, c["phi"], c["grad"], TOL64, 0.1)


def test_cube_mixed_matches_oracle(lsm, cube_case):
    c = cube_case
    phi, grad = c["mesh"].eval_phi_grad(c["x"], lsm.MIXED)
    _check(phi, grad, c["phi"], c["grad"], TOL32, 0.1)


@pytest.fixture(scope="module")
def torus_case(oracle_mod, ctx):
    """A graded, jittered torus with per-triangle sigma: 2 x 52 x 14 = 1,456
    triangles, 3x3 rule = 13,104 nodes (103 tiles, the last one ragged),
    3,001 targets within 3 sigma of the surface."""
    m = synth.torus(1.0, 0.3, 52, 14, 20.0, 0.05, seed=21)
    y, nw, sg = _oracle_sources(oracle_mod, m, 3)
    x = synth.targets_near_surface(m, 3001, synth.rng(22), 3.0)
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, x)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=3)
    return dict(m=m, x=x, phi=phi_o, grad=grad_o, mesh=mesh, src=(y, nw, sg))


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
def test_torus_matches_oracle(lsm, torus_case, prec, tol):
    c = torus_case
    phi, grad = c["mesh"].eval_phi_grad(c["x"], prec)
    _check(phi, grad, c["phi"], c["grad"], tol, c["m"].sigma.min())


def test_bumped_icosphere_matches_oracle(lsm, ctx, oracle_mod):
    """Multiscale surface: icosphere level 4 (5,120 triangles) with 200
    Gaussian bumps down to width 0.005, sigma by the area rule, 4x4 rule
    (81,920 nodes), 4,000 targets within 3 sigma; all three precisions."""
    m = synth.bumped_icosphere(4, 200, seed=13)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 4, 0)
    x = synth.targets_near_surface(m, 4000, synth.rng(14), 3.0)
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, x)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4)
    for prec, tol in ((0, TOL64), (1, TOL32)):
        phi, grad = mesh.eval_phi_grad(x, prec)
        _check(phi, grad, phi_o, grad_o, tol, m.sigma.min())
    phi, grad = mesh.eval_phi_grad(x, lsm.FF)
    assert np.abs(phi - phi_o).max() <= TOL64
    assert np.abs(grad - grad_o).max() <= TOL32 / m.sigma.min()


@pytest.mark.parametrize("case", ["cube", "torus"])
def test_float_float_path_reaches_fp64_accuracy_on_phi(lsm, cube_case, torus_case, case):
    """LSM_FF: far tiles in float-float on the FP32 pipes, near tiles in FP64.
    Phi within the FP64 tolerance; grad Phi within the mixed tolerance."""
    c = cube_case if case == "cube" else torus_case
    smin = 0.1 if case == "cube" else c["m"].sigma.min()
    phi, grad = c["mesh"].eval_phi_grad(c["x"], lsm.FF)
    assert np.abs(phi - c["phi"]).max() <= TOL64
    assert np.abs(grad - c["grad"]).max() <= TOL32 / smin


@pytest.mark.parametrize("prec,tol", [(0, TOL64), (1, TOL32)])
def test_device_and_host_pointers_agree(lsm, torus_case, prec, tol):
    c = torus_case
    xd = torch.from_numpy(c["x"]).cuda()
    phi_d, grad_d = c["mesh"].eval_phi_grad(xd, prec)
    torch.cuda.synchronize()
    phi_h, grad_h = c["mesh"].eval_phi_grad(c["x"], prec)
    assert np.array_equal(phi_d.cpu().numpy(), phi_h)
    assert np.array_equal(grad_d.cpu().numpy(), grad_h)


def test_results_are_deterministic(lsm, torus_case):
    c = torus_case
    a = c["mesh"].eval_phi_grad(c["x"], lsm.MIXED)
    b = c["mesh"].eval_phi_grad(c["x"], lsm.MIXED)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_edge_cases(lsm, oracle_mod, torus_case):
    c = torus_case
    y, nw, sg = c["src"]
    # targets exactly on source nodes (rho = 0), a single target, far targets
    x = np.concatenate([y[:7], [[0.0, 0.0, 0.0]], [[1e3, -2e3, 5e2]], [[1.3, 0.0, 0.0]]])
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, x)
    for prec, tol in ((0, TOL64), (1, TOL32)):
        phi, grad = c["mesh"].eval_phi_grad(x, prec)
        _check(phi, grad, phi_o, grad_o, tol, c["m"].sigma.min())
        p1, g1 = c["mesh"].eval_phi_grad(x[8:9], prec)
        assert abs(p1[0] - phi_o[8]) <= tol
    p0, g0 = c["mesh"].eval_phi_grad(np.zeros((0, 3)), lsm.FP64)
    assert p0.shape == (0,)


def test_rejects_bad_meshes_and_arguments(lsm, ctx):
    m = synth.cube(1.0, 2)
    with pytest.raises(lsm.LsmError) as e:
        ctx.upload(m.verts, m.tris[:-1])          # open mesh
    assert e.value.code == -4
    with pytest.raises(lsm.LsmError) as e:
        ctx.upload(m.verts, m.tris[:, ::-1].copy())  # inside-out
    assert e.value.code == -4
    bad = m.tris.copy()
    bad[0, 0] = 10_000
    with pytest.raises(lsm.LsmError) as e:
        ctx.upload(m.verts, bad)
    assert e.value.code == -4
    with pytest.raises(lsm.LsmError) as e:
        ctx.upload(m.verts, m.tris, np.zeros(m.m))  # sigma must be > 0
    assert e.value.code == -4
    mesh = ctx.upload(m.verts, m.tris, np.full(m.m, 0.2))
    with pytest.raises(lsm.LsmError) as e:
        mesh.eval_phi_grad(np.zeros((4, 3)), precision=7)
    assert e.value.code == -1


def test_default_sigma_rule(lsm, ctx, oracle_mod):
    m = synth.torus(1.0, 0.3, 20, 8, 4.0, 0.05, seed=5)
    mesh = ctx.upload(m.verts, m.tris, None, n_gl=2)
    inf = mesh.info()
    s = synth.sigma_half_sqrt2area(m.verts, m.tris)
    assert abs(inf["sigma_min"] - s.min()) < 1e-15 and abs(inf["sigma_max"] - s.max()) < 1e-15
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, None, 2, 0)
    x = synth.targets_near_surface(m, 300, synth.rng(1), 2.0, sigma=s)
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, x)
    phi, grad = mesh.eval_phi_grad(x, lsm.FP64)
    _check(phi, grad, phi_o, grad_o, TOL64, s.min())


# ---------------------------------------------------------------- charts
def test_flat_face_charts_match_closed_form(lsm, ctx, oracle_mod):
    """Chart nodes on triangles interior to the cube faces: the GPU's h equals
    the oracle's h (itself pinned to the 1-D erf-product root)."""
    m = synth.cube(1.0, 4)
    s = np.full(m.m, 0.1)
    mesh = ctx.upload(m.verts, m.tris, s, n_gl=8, subdiv=1)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, s, 8, 1)
    x0, hd, sl = oracle_mod.chart_nodes(m.verts, m.tris, s, 3)
    ref = oracle_mod.solve_charts(y, nw, sg, x0, hd, sl, tol=1e-12)
    for prec, tol in ((0, 1e-11), (1, 1e-10)):
        x, h, st, stats = mesh.solve_charts(order=2, tol=1e-12, precision=prec)   # n = 3
        assert np.all(st == 0), np.unique(st)
        assert np.abs(h - ref["h"]).max() < tol
        assert np.abs(x - ref["x"]).max() < tol
        assert stats.n_converged == len(h) and stats.max_residual < 1e-12


@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-9)])
def test_torus_charts_match_oracle(lsm, oracle_mod, torus_case, prec, tol):
    c = torus_case
    m = c["m"]
    y, nw, sg = c["src"]
    x0, hd, sl = oracle_mod.chart_nodes(m.verts, m.tris, m.sigma, 2)
    x, h, st, stats = c["mesh"].solve_charts(order=0, tol=1e-12, precision=prec)    # n = 2
    assert np.all(st & 255 == 0)
    sel = np.arange(0, len(x0), 7)
    ref = oracle_mod.solve_charts(y, nw, sg, x0[sel], hd[sel], sl[sel], tol=1e-12)
    assert np.all(ref["status"] & 255 == 0)
    assert np.abs(x[sel] - ref["x"]).max() < tol
    phi, _ = oracle_mod.phi_grad(y, nw, sg, x[sel])
    assert np.abs(phi - 0.5).max() < 1e-11
    if prec == 1:
        assert stats.evals_fp32 > 0 and stats.evals_fp64 > 0


def test_newton_reports_failures_per_node(lsm, ctx):
    m = synth.cube(1.0, 2)
    mesh = ctx.upload(m.verts, m.tris, np.full(m.m, 0.2), n_gl=3)
    x, h, st, stats = mesh.solve_charts(order=0, tol=1e-14, max_iter=1)
    assert np.all(st & 255 == lsm.NODE_MAXITER)
    assert stats.n_failed == len(st) and stats.iterations == 1
