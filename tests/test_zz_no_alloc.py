"""The no-allocation entry point, lsm_eval_phi_grad_noalloc.

Some callers cannot call cudaMalloc while they run: a latency-critical loop
in which an allocation or a free could synchronise the device, or a process
whose device memory another allocator has already reserved in full.  For them
the library evaluates Phi and grad Phi with its scratch in one fixed 8 MiB
device array.  This file checks, through the C ABI, that it returns what
lsm_eval_phi_grad returns (within the tolerances of the other GPU tests) on
two calls in a row, and that it refuses sizes beyond its limit.  It builds
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
def test_noalloc_matches_eval_on_two_calls(setup, prec, tol):
    lsm, L, ctx, m, mesh = setup
    smin = m.sigma.min()
    for call, (n, seed) in enumerate(((3001, 40), (MAX_TARGETS, 41))):
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
