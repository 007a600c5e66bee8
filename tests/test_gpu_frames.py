"""GPU parity of the chart local coordinates and the Gauss flux check
(Sec. 3.3, Sec. 5) against the oracle, on the same solved charts.

The frames and the flux are FP64 elementwise arithmetic over the chart
nodes: the bar is FP64 rounding (1e-12 relative on x_u, x_v, da; 1e-13 on
eps0, a sum of O(1) magnitude).
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
def sphere(lsm):
    """Icosphere level 2 (320 triangles), sigma by the workloads' rule, 4x4
    sources, order-8 charts solved on the FP64 path to 1e-13."""
    m = synth.icosphere(2)
    ctx = lsm.Context(0)
    mesh = ctx.upload(m.verts, m.tris, None, n_gl=4)
    x, h, st, stats = mesh.solve_charts(order=8, tol=1e-13, precision=lsm.FP64)
    assert stats.n_failed == 0
    _, g = mesh.eval_phi_grad(x, lsm.FP64)
    return m, ctx, mesh, x, h, g


def test_frames_match_oracle(lsm, oracle_mod, sphere):
    m, ctx, mesh, x, h, g = sphere
    xu, xv, jac = mesh.chart_frames(8, h, g)
    ou, ov, oj = oracle_mod.chart_frames(m.verts, m.tris, h, g, n=6)
    scale = np.abs(ou).max()
    assert np.abs(xu - ou).max() <= 1e-12 * scale
    assert np.abs(xv - ov).max() <= 1e-12 * scale
    assert np.abs(jac - oj).max() <= 1e-12 * np.abs(oj).max()
    # tangent to the level set
    assert np.abs(np.sum(xu * g, axis=1)).max() <= 1e-10 * scale * np.abs(g).max()


def test_gauss_flux_matches_oracle_and_closes(lsm, oracle_mod, sphere):
    m, ctx, mesh, x, h, g = sphere
    _, _, jac = mesh.chart_frames(8, h, g)
    for x0 in ((0.05, -0.1, 0.02), (0.0, 0.0, 0.0), (0.3, 0.2, -0.1)):
        e = mesh.gauss_flux(8, x, g, jac, x0)
        eo = oracle_mod.gauss_flux(x, g, jac, x0, n=6)
        assert abs(e - eo) <= 1e-13
        assert abs(e) < 1e-9
    e_out = mesh.gauss_flux(8, x, g, jac, (3.0, 0.0, 0.0))
    assert abs(e_out - 1.0) < 1e-9


def test_frames_and_flux_device_pointers(lsm, sphere):
    m, ctx, mesh, x, h, g = sphere
    xu, xv, jac = mesh.chart_frames(8, h, g)
    dxu, dxv, djac = mesh.chart_frames(8, torch.from_numpy(h).cuda(), torch.from_numpy(g).cuda())
    assert np.array_equal(dxu.cpu().numpy(), xu) and np.array_equal(djac.cpu().numpy(), jac)
    e = mesh.gauss_flux(8, x, g, jac, (0.0, 0.0, 0.0))
    ed = mesh.gauss_flux(8, torch.from_numpy(x).cuda(), torch.from_numpy(g).cuda(), djac, (0.0, 0.0, 0.0))
    assert e == ed


def test_flux_with_mixed_solve_and_ff_gradient(lsm, sphere):
    """The production path: mixed chart solve to 1e-12, grad Phi from the
    float-float path (its gradient carries the mixed accuracy, 1e-7 relative),
    which sets the floor of eps0."""
    m, ctx, mesh, x64, h64, g64 = sphere
    x, h, st, stats = mesh.solve_charts(order=8, tol=1e-12, precision=lsm.MIXED)
    assert stats.n_failed == 0
    _, gff = mesh.eval_phi_grad(x, lsm.FF)
    _, _, jac = mesh.chart_frames(8, h, gff)
    e_ff = mesh.gauss_flux(8, x, gff, jac, (0.0, 0.0, 0.0))
    _, _, jac64 = mesh.chart_frames(8, h64, g64)
    e_64 = mesh.gauss_flux(8, x64, g64, jac64, (0.0, 0.0, 0.0))
    assert abs(e_64) < 1e-6
    assert abs(e_ff) < 1e-6
    assert np.abs(h - h64).max() < 1e-9


def test_frames_bad_arguments(lsm, sphere):
    m, ctx, mesh, x, h, g = sphere
    with pytest.raises(lsm.LsmError):
        mesh.chart_frames(-2, h, g)
