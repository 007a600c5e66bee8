"""The no-allocation entry point, lsm_eval_phi_grad_noalloc.

Some callers cannot call cudaMalloc while they run: a latency-critical loop
in which an allocation or a free could synchronise the device, or a process
whose device memory another allocator has already reserved in full.  For them
the library evaluates Phi and grad Phi with its scratch in one fixed 8 MiB
device array.  This file checks, through the C ABI, that it returns what
lsm_eval_phi_grad returns (within the tolerances of the other GPU tests) on
calls in a row, that the last of them matches the oracle, that it refuses
sizes beyond its limit, and that a bounded wait that runs out is reported.  It builds
its own context and mesh, so it runs the same alone or after the other tests.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MAX_TARGETS = 16384


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as lsm
    L = lsm.load()
    ctx = lsm.Context(0)
    m = synth.torus(1.0, 0.3, 52, 14, 20.0, 0.05, seed=31)
    mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=3)
    return lsm, L, ctx, m, mesh


def _noalloc(L, mesh, x, prec):
    n = x.shape[0]
    phi = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
    grad = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    rc = L.lsm_eval_phi_grad_noalloc(mesh._h, ctypes.c_void_p(x.data_ptr()), n,
                                     ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                     prec, ctypes.c_void_p(st))
    return rc, phi, grad


@pytest.mark.parametrize("prec,tol", [(0, 1e-12), (1, 1e-7)])
def test_noalloc_matches_eval_on_two_calls(setup, oracle_mod, prec, tol):
    """Calls in a row of growing, then shrinking size: the shared array keeps
    the previous call's contents, and the split planes move with n, so a
    smaller call after the largest would read stale partials if any element
    were read before being written."""
    lsm, L, ctx, m, mesh = setup
    smin = m.sigma.min()
    for call, (n, seed) in enumerate(((3001, 40), (MAX_TARGETS, 41), (777, 42))):
        x = torch.from_numpy(synth.targets_near_surface(m, n, synth.rng(seed), 3.0)).cuda()
        rc, phi, grad = _noalloc(L, mesh, x, prec)
        assert rc == 0, ctx._L.lsm_last_error(ctx._h)
        ref_phi, ref_grad = mesh.eval_phi_grad(x, prec)
        torch.cuda.synchronize()
        assert torch.isfinite(phi).all() and torch.isfinite(grad).all()
        ep = (phi - ref_phi).abs().max().item()
        eg = (grad - ref_grad).abs().max().item()
        assert ep <= tol, (call, ep)
        assert eg <= tol / smin, (call, eg)
    # the last call against the FP64 oracle on a subset of its targets
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 3, 0)
    xs = x[:96].cpu().numpy()
    phi_o, grad_o = oracle_mod.phi_grad(y, nw, sg, xs)
    assert np.abs(phi[:96].cpu().numpy() - phi_o).max() <= tol
    assert np.abs(grad[:96].cpu().numpy() - grad_o).max() <= tol / smin
    ctx.check_error()   # no bounded wait ran out


def test_noalloc_reports_a_lost_stage(setup):
    """A wait that runs out (test hook: the first stage is armed without a
    copy) leaves NaN in the targets concerned and is reported by
    lsm_check_error; the next call is clean."""
    lsm, L, ctx, m, mesh = setup
    x = torch.from_numpy(synth.targets_near_surface(m, 500, synth.rng(43), 3.0)).cuda()
    ctx.inject_wait_timeout(True)
    try:
        rc, phi, _ = _noalloc(L, mesh, x, 1)
        assert rc == 0   # asynchronous: reported below
        torch.cuda.synchronize()
        assert torch.isnan(phi).all()
        with pytest.raises(lsm.LsmError) as e:
            ctx.check_error()
        assert e.value.code == -6
    finally:
        ctx.inject_wait_timeout(False)
    rc, phi, _ = _noalloc(L, mesh, x, 1)
    assert rc == 0
    torch.cuda.synchronize()
    assert torch.isfinite(phi).all()
    ctx.check_error()


def test_noalloc_rejects_sizes_beyond_its_scratch(setup):
    lsm, L, ctx, m, mesh = setup
    x = torch.zeros((MAX_TARGETS + 1, 3), dtype=torch.float64, device="cuda")
    rc, _, _ = _noalloc(L, mesh, x, 1)
    assert rc == -1
    assert b"16384" in ctx._L.lsm_last_error(ctx._h)
    xh = np.zeros((4, 3))
    out = np.zeros(4)
    rc = L.lsm_eval_phi_grad_noalloc(mesh._h, xh.ctypes.data_as(ctypes.c_void_p), 4,
                                     out.ctypes.data_as(ctypes.c_void_p), None, 1, None)
    assert rc == -1
