"""Failure detection on the GPU without a GPU fault.

Every wait of a pair kernel on its staged source tile is bounded.  A test
hook (lsm_test_inject_wait_timeout) makes each kernel arm its first stage's
barrier without issuing the copy, so the wait runs out with nothing in
flight.  The call must report LSM_E_TIMEOUT (synchronous, host pointers) or
leave NaN and report it at lsm_check_error (asynchronous, device pointers),
and the context must stay usable: the next call matches the call before.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TIMEOUT = -6


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as lsm
    ctx = lsm.Context(0, tree_min_sources=20_000, tree_ff_min_sources=20_000)
    m = synth.torus(1.0, 0.3, 60, 16, 20.0, 0.05, seed=71)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4)   # 30,720 nodes: treecode lists
    x = synth.targets_near_surface(m, 3000, synth.rng(72), 3.0)
    return lsm, ctx, m, mesh, x


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_timeout_is_reported_and_context_recovers(setup, prec):
    lsm, ctx, m, mesh, x = setup
    phi0, grad0 = mesh.eval_phi_grad(x, prec)
    ctx.inject_wait_timeout(True)
    try:
        with pytest.raises(lsm.LsmError) as e:
            mesh.eval_phi_grad(x, prec)
        assert e.value.code == TIMEOUT
        assert "wait limit" in str(e.value)
        # device pointers: the call returns at once, the results are NaN and
        # the error word is read by lsm_check_error
        xd = torch.from_numpy(x).cuda()
        phi, _ = mesh.eval_phi_grad(xd, prec)
        torch.cuda.synchronize()
        assert torch.isnan(phi).all()
        with pytest.raises(lsm.LsmError) as e:
            ctx.check_error()
        assert e.value.code == TIMEOUT
    finally:
        ctx.inject_wait_timeout(False)
    ctx.check_error()   # cleared
    phi1, grad1 = mesh.eval_phi_grad(x, prec)
    assert np.array_equal(phi1, phi0) and np.array_equal(grad1, grad0)


def test_timeout_in_chart_solve(setup):
    """Newton under the hook: nodes see NaN (status non-finite) and the solve
    reports the timeout; the next solve converges as before."""
    lsm, ctx, m, mesh, x = setup
    ref = mesh.solve_charts(order=4, tol=1e-12, precision=lsm.MIXED)
    ctx.inject_wait_timeout(True)
    try:
        with pytest.raises(lsm.LsmError) as e:
            mesh.solve_charts(order=4, tol=1e-12, precision=lsm.MIXED)
        assert e.value.code == TIMEOUT
    finally:
        ctx.inject_wait_timeout(False)
    xc, h, st, stats = mesh.solve_charts(order=4, tol=1e-12, precision=lsm.MIXED)
    assert np.all(st & 255 == 0)
    assert np.array_equal(xc, ref[0])


def test_context_closed_before_its_meshes(setup):
    """Objects freed in any order (as a garbage collector may do with cycles):
    closing a context first frees its meshes, batches and servers; freeing
    them afterwards is a no-op, and later calls on a new context see no error
    left behind."""
    lsm, _, m, _, x = setup
    ctx2 = lsm.Context(0)
    mesh2 = ctx2.upload(m.verts, m.tris, m.sigma, n_gl=3)
    b2 = lsm.Batch(ctx2, [mesh2])
    srv = lsm.Server(ctx2, slots=2)
    ctx2.close()
    mesh2.free()
    b2.free()
    srv.close()
    ctx3 = lsm.Context(0)
    mesh3 = ctx3.upload(m.verts, m.tris, m.sigma, n_gl=3)
    phi, _ = mesh3.eval_phi_grad(x[:500], lsm.MIXED)
    assert np.isfinite(phi).all()
    ctx3.check_error()
    mesh3.free()
    ctx3.close()
