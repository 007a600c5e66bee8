"""FP64 CPU oracle for the smoothed level-set function (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product library never does, and
this package never imports the product library: the two share nothing but
the seeded input arrays produced by ``synth``.

The arithmetic lives in ``oracle.c`` (plain C, FP64, direct summation over all
pairs).  This module compiles it with gcc on first use and wraps it with
ctypes; every wrapper names the paper passage its C function follows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

ST_CONVERGED = 0
ST_MAXITER = 1
ST_ZERODERIV = 2
ST_NONFINITE = 3
ST_CLAMPED_BIT = 256


def build(force: bool = False) -> str:
    """Compile oracle.c into a shared library (gcc, OpenMP, no fast-math)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            I64 = ctypes.c_int64
            lib.or_gauss_legendre01.argtypes = [ctypes.c_int, P, P]
            lib.or_simplex_rule.argtypes = [ctypes.c_int, ctypes.c_int, P, P, P]
            lib.or_geometry.argtypes = [I64, P, I64, P, P, P, P, P, P, P]
            lib.or_sources.argtypes = [I64, P, I64, P, P, P, ctypes.c_int, P, P, P, P, P, P]
            lib.or_radial.argtypes = [ctypes.c_double, ctypes.c_double, P, P]
            lib.or_phi_grad.argtypes = [I64, P, P, P, I64, P, P, P, ctypes.c_int]
            lib.or_chart_nodes.argtypes = [P, I64, P, P, P, ctypes.c_int, P, P, P, P, P]
            lib.or_solve_charts.argtypes = [I64, P, P, P, I64, P, P, P, ctypes.c_double,
                                            ctypes.c_int, P, P, P, P, P, ctypes.c_int]
            lib.or_chart_frames.argtypes = [P, I64, P, P, ctypes.c_int, P, P, P, P, P, P, P]
            lib.or_gauss_flux.argtypes = [I64, ctypes.c_int, P, P, P, P, P]
            lib.or_gauss_flux.restype = ctypes.c_double
            lib.or_sigma_sources.argtypes = [P, I64, P, ctypes.c_double, P, P]
            lib.or_sigma_sources.restype = ctypes.c_double
            lib.or_sigma_x.argtypes = [I64, P, P, ctypes.c_double, I64, P, P, P]
            lib.or_phi_grad_sigx.argtypes = [I64, P, P, I64, P, P, P, P, P, ctypes.c_int]
            lib.or_solve_charts_sigx.argtypes = [I64, P, P, I64, P, P, ctypes.c_double, I64, P, P, P,
                                                 ctypes.c_double, ctypes.c_int, P, P, P, P, P, ctypes.c_int]
            lib.or_radial_G.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.or_radial_G.restype = ctypes.c_double
            lib.or_phi_grad_hess.argtypes = [I64, P, P, P, I64, P, P, P, P, ctypes.c_int]
            lib.or_chart_second.argtypes = [P, I64, P, P, ctypes.c_int, P, P, P, P, P, P, P, P, P, P]
            lib.or_chart_nodes_at.argtypes = [P, P, P, P, I64, P, P, P, P, P]
            lib.or_chart_frames_at.argtypes = [P, P, P, I64, P, P, P, P, P, P, P]
            lib.or_gauss_flux_w.argtypes = [I64, P, P, P, P, P]
            lib.or_gauss_flux_w.restype = ctypes.c_double
            lib.or_geometry_quad.argtypes = [I64, P, I64, P, P, ctypes.c_int, P, P, P, P, P]
            lib.or_sources_quad.argtypes = [P, I64, P, P, ctypes.c_int, P, P, P, P, P, P]
            lib.or_chart_nodes_quad_at.argtypes = [P, P, P, P, I64, P, P, P, P, P]
            lib.or_chart_frames_quad_at.argtypes = [P, P, P, I64, P, P, P, P, P, P, P]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def gauss_legendre01(n: int):
    """n-point Gauss-Legendre nodes and weights on [0,1]."""
    x = np.empty(n)
    w = np.empty(n)
    if _load().or_gauss_legendre01(n, _p(x), _p(w)) != 0:
        raise ValueError("bad n")
    return x, w


def simplex_rule(n: int, subdiv: int = 0):
    """Duffy-collapsed n x n Gauss-Legendre rule on the standard simplex,
    composite over ``subdiv`` midpoint splits (Sec. 4.3 and 4.5)."""
    cnt = n * n * 4 ** subdiv
    u, v, w = np.empty(cnt), np.empty(cnt), np.empty(cnt)
    m = _load().or_simplex_rule(n, subdiv, _p(u), _p(v), _p(w))
    if m != cnt:
        raise ValueError("bad rule parameters")
    return u, v, w


def geometry(verts, tris, sigma=None):
    """Per-triangle T_u, T_v, N (eq. tparam), sigma_j, and the vertex
    pseudonormals H(P) (eq. mkvertexpn)."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    nv, m = len(verts), len(tris)
    tu, tv, nrm = np.empty((m, 3)), np.empty((m, 3)), np.empty((m, 3))
    sig = np.empty(m)
    vpn = np.empty((nv, 3))
    sig_in = _f64(sigma) if sigma is not None else None
    rc = _load().or_geometry(nv, _p(verts), m, _p(tris),
                             _p(sig_in) if sig_in is not None else None,
                             _p(tu), _p(tv), _p(nrm), _p(sig), _p(vpn))
    if rc != 0:
        raise ValueError("a vertex has no incident triangle")
    return dict(tu=tu, tv=tv, nrm=nrm, sigma=sig, vpn=vpn)


def sources(verts, tris, sigma=None, n: int = 4, subdiv: int = 0):
    """Source nodes y, nw = w |N| N_hat and sigma of the discrete sum
    (eq. discrete_int) for the n x n Duffy rule with ``subdiv`` splits."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    geo = geometry(verts, tris, sigma)
    ru, rv, rw = simplex_rule(n, subdiv)
    m, nq = len(tris), len(ru)
    y, nw, sg = np.empty((m * nq, 3)), np.empty((m * nq, 3)), np.empty(m * nq)
    _load().or_sources(len(verts), _p(verts), m, _p(tris), _p(geo["nrm"]), _p(geo["sigma"]),
                       nq, _p(ru), _p(rv), _p(rw), _p(y), _p(nw), _p(sg))
    return y, nw, sg


def radial(rho: float, sigma: float):
    """Radial factors f(rho) and F(rho) = f'(rho)/rho of the pair kernel."""
    f = ctypes.c_double()
    F = ctypes.c_double()
    _load().or_radial(float(rho), float(sigma), ctypes.byref(f), ctypes.byref(F))
    return f.value, F.value


def phi_grad(y, nw, sig, x, nthreads: int = 0):
    """Phi and grad Phi at targets x by the full direct sum (eq. discrete_int,
    eq. gradPhi with corrected sign)."""
    y, nw, sig, x = _f64(y), _f64(nw), _f64(sig), _f64(x)
    nt = len(x)
    phi = np.empty(nt)
    grad = np.empty((nt, 3))
    _load().or_phi_grad(len(y), _p(y), _p(nw), _p(sig), nt, _p(x), _p(phi), _p(grad), nthreads)
    return phi, grad


def chart_nodes(verts, tris, sigma=None, n: int = 6):
    """Chart nodes x0 = T^j(u_i,v_i), directions H^j(u_i,v_i) (eq. mkpseudovec)
    and the triangle's sigma, for the n x n Duffy chart rule."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    geo = geometry(verts, tris, sigma)
    cu, cv, _ = simplex_rule(n, 0)
    m, npn = len(tris), len(cu)
    x0, hd, sl = np.empty((m * npn, 3)), np.empty((m * npn, 3)), np.empty(m * npn)
    _load().or_chart_nodes(_p(verts), m, _p(tris), _p(geo["vpn"]), _p(geo["sigma"]), npn,
                           _p(cu), _p(cv), _p(x0), _p(hd), _p(sl))
    return x0, hd, sl


def solve_charts(y, nw, sig, x0, hdir, sloc, tol: float = 1e-12, max_iter: int = 20,
                 nthreads: int = 0):
    """Newton's method for h at each chart node (eq. newtoneq), h0 = 0."""
    y, nw, sig = _f64(y), _f64(nw), _f64(sig)
    x0, hdir, sloc = _f64(x0), _f64(hdir), _f64(sloc)
    n = len(x0)
    xo, ho = np.empty((n, 3)), np.empty(n)
    st, it = np.empty(n, dtype=np.int32), np.empty(n, dtype=np.int32)
    dh = np.empty(n)
    _load().or_solve_charts(len(y), _p(y), _p(nw), _p(sig), n, _p(x0), _p(hdir), _p(sloc),
                            float(tol), int(max_iter), _p(xo), _p(ho), _p(st), _p(it), _p(dh),
                            nthreads)
    return dict(x=xo, h=ho, status=st, iters=it, last_dh=dh)


def chart_frames(verts, tris, h, grad, sigma=None, n: int = 6, uv=None):
    """Local coordinates x_u, x_v and the area density |x_u x x_v| at the chart
    nodes of the n x n Duffy chart rule (eq. u_vector, U_vector_2, v_vector,
    v_vector_2, da), from the solved h and grad Phi at each node.  uv = (cu,
    cv) replaces the rule's points (the same points on every triangle)."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    geo = geometry(verts, tris, sigma)
    if uv is None:
        cu, cv, _ = simplex_rule(n, 0)
    else:
        cu, cv = _f64(uv[0]), _f64(uv[1])
    h, grad = _f64(h), _f64(grad)
    m, npn = len(tris), len(cu)
    assert h.shape == (m * npn,) and grad.shape == (m * npn, 3)
    xu, xv, jac = np.empty((m * npn, 3)), np.empty((m * npn, 3)), np.empty(m * npn)
    _load().or_chart_frames(_p(verts), m, _p(tris), _p(geo["vpn"]), npn, _p(cu), _p(cv), _p(h), _p(grad),
                            _p(xu), _p(xv), _p(jac))
    return xu, xv, jac


def gauss_flux(x, grad, jac, x0, n: int = 6) -> float:
    """Gauss flux error eps0 of the charts (Sec. 5) about the point x0, with
    the n x n Duffy chart rule as quadrature on every triangle."""
    _, _, cw = simplex_rule(n, 0)
    x, grad, jac = _f64(x), _f64(grad), _f64(jac)
    x0 = _f64(np.asarray(x0, dtype=np.float64).reshape(3))
    assert len(x) % len(cw) == 0
    return _load().or_gauss_flux(len(x), len(cw), _p(cw), _p(x), _p(grad), _p(jac), _p(x0))


SIGMA_LAMBDA = 2.5


def sigma0_default(dmax: float) -> float:
    """sigma0 such that a centroid one diameter away has weight 1/2 (the
    influence the paper states for its choice, Sec. 2.3)."""
    return dmax / np.sqrt(2.0 * np.log(2.0))


def sigma_sources(verts, tris, lam: float = SIGMA_LAMBDA):
    """Centroids c_j, sigma_j = D_j / lambda (D_j: diameter of the smallest
    enclosing ball) and max_j D_j (Sec. 2.3)."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    m = len(tris)
    c, sj = np.empty((m, 3)), np.empty(m)
    dmax = _load().or_sigma_sources(_p(verts), m, _p(tris), float(lam), _p(c), _p(sj))
    return c, sj, dmax


def sigma_x(c, sj, sigma0: float, x):
    """sigma(x) and grad sigma(x) at targets x [n, 3] (eq. sigma2)."""
    c, sj, x = _f64(c), _f64(sj), _f64(x)
    n = len(x)
    sig, gs = np.empty(n), np.empty((n, 3))
    _load().or_sigma_x(len(c), _p(c), _p(sj), float(sigma0), n, _p(x), _p(sig), _p(gs))
    return sig, gs


def phi_grad_sigx(y, nw, x, sig, gsig, nthreads: int = 0):
    """Phi and grad Phi with the targets' sigma (eq. kerpsi with sigma(x), eq.
    gradPhi including the grad-sigma term, sign corrected)."""
    y, nw, x, sig, gsig = _f64(y), _f64(nw), _f64(x), _f64(sig), _f64(gsig)
    nt = len(x)
    phi, grad = np.empty(nt), np.empty((nt, 3))
    _load().or_phi_grad_sigx(len(y), _p(y), _p(nw), nt, _p(x), _p(sig), _p(gsig), _p(phi), _p(grad), nthreads)
    return phi, grad


def solve_charts_sigx(y, nw, c, sj, sigma0, x0, hdir, sloc, tol: float = 1e-12, max_iter: int = 20,
                      nthreads: int = 0):
    """Newton's method for h at each chart node (eq. newtoneq) with sigma(x)."""
    y, nw, c, sj = _f64(y), _f64(nw), _f64(c), _f64(sj)
    x0, hdir, sloc = _f64(x0), _f64(hdir), _f64(sloc)
    n = len(x0)
    xo, ho = np.empty((n, 3)), np.empty(n)
    st, it = np.empty(n, dtype=np.int32), np.empty(n, dtype=np.int32)
    dh = np.empty(n)
    _load().or_solve_charts_sigx(len(y), _p(y), _p(nw), len(c), _p(c), _p(sj), float(sigma0), n, _p(x0), _p(hdir),
                                 _p(sloc), float(tol), int(max_iter), _p(xo), _p(ho), _p(st), _p(it), _p(dh),
                                 nthreads)
    return dict(x=xo, h=ho, status=st, iters=it, last_dh=dh)


def radial_G(rho: float, sigma: float) -> float:
    """Third radial factor G = F'(rho)/rho of the pair kernel."""
    return _load().or_radial_G(float(rho), float(sigma))


def phi_grad_hess(y, nw, sig, x, nthreads: int = 0):
    """Phi, grad Phi and the Hessian [n, 6] = (xx, xy, xz, yy, yz, zz) by
    direct summation (per-triangle sigma)."""
    y, nw, sig, x = _f64(y), _f64(nw), _f64(sig), _f64(x)
    nt = len(x)
    phi, grad, hess = np.empty(nt), np.empty((nt, 3)), np.empty((nt, 6))
    _load().or_phi_grad_hess(len(y), _p(y), _p(nw), _p(sig), nt, _p(x), _p(phi), _p(grad), _p(hess), nthreads)
    return phi, grad, hess


def chart_second(verts, tris, h, grad, hess, sigma=None, n: int = 6, uv=None):
    """Second derivatives x_uu, x_uv, x_vv [N, 3] of the solved charts and the
    mean (sum of principal curvatures) and Gaussian curvatures [N] of the
    level set at the nodes (eq. uu_vector and its analogues)."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    geo = geometry(verts, tris, sigma)
    if uv is None:
        cu, cv, _ = simplex_rule(n, 0)
    else:
        cu, cv = _f64(uv[0]), _f64(uv[1])
    h, grad, hess = _f64(h), _f64(grad), _f64(hess)
    m, npn = len(tris), len(cu)
    N = m * npn
    assert h.shape == (N,) and grad.shape == (N, 3) and hess.shape == (N, 6)
    uu, uv_, vv = np.empty((N, 3)), np.empty((N, 3)), np.empty((N, 3))
    km, kg = np.empty(N), np.empty(N)
    _load().or_chart_second(_p(verts), m, _p(tris), _p(geo["vpn"]), npn, _p(cu), _p(cv), _p(h), _p(grad),
                            _p(hess), _p(uu), _p(uv_), _p(vv), _p(km), _p(kg))
    return uu, uv_, vv, km, kg


def refined_nodes(m: int, n: int, levels):
    """Chart nodes of triangles refined 1 -> 4 levels[j] times (Sec. 3.4): for
    each triangle in order, the n x n Duffy rule composited over its 4^L
    midpoint children, as parent coordinates (u, v) and weights (summing to
    1/2 per triangle).  Returns tri [N], uv [N, 2], w [N]."""
    levels = np.asarray(levels, dtype=np.int64)
    assert levels.shape == (m,)
    rules = {}
    tri, uv, w = [], [], []
    for j in range(m):
        L = int(levels[j])
        if L not in rules:
            rules[L] = simplex_rule(n, L)
        u, v, ww = rules[L]
        tri.append(np.full(len(u), j, dtype=np.int32))
        uv.append(np.stack([u, v], 1))
        w.append(ww)
    return np.concatenate(tri), np.concatenate(uv), np.concatenate(w)


def chart_nodes_at(verts, tris, tri, uv, sigma=None):
    """x0 = T(u, v), H(u, v) and sigma of the triangle at explicit nodes."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    geo = geometry(verts, tris, sigma)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    uv = _f64(uv)
    n = len(tri)
    x0, hd, sl = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    _load().or_chart_nodes_at(_p(verts), _p(tris), _p(geo["vpn"]), _p(geo["sigma"]), n, _p(tri), _p(uv),
                              _p(x0), _p(hd), _p(sl))
    return x0, hd, sl


def chart_frames_at(verts, tris, tri, uv, h, grad, sigma=None):
    """chart_frames at explicit nodes (triangle, parent (u, v))."""
    verts = _f64(verts)
    tris = np.ascontiguousarray(tris, dtype=np.int32)
    geo = geometry(verts, tris, sigma)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    uv, h, grad = _f64(uv), _f64(h), _f64(grad)
    n = len(tri)
    xu, xv, jac = np.empty((n, 3)), np.empty((n, 3)), np.empty(n)
    _load().or_chart_frames_at(_p(verts), _p(tris), _p(geo["vpn"]), n, _p(tri), _p(uv), _p(h), _p(grad),
                               _p(xu), _p(xv), _p(jac))
    return xu, xv, jac


def gauss_flux_w(x, grad, jac, w, x0) -> float:
    """Gauss flux error with a quadrature weight per node (Sec. 5)."""
    x, grad, jac, w = _f64(x), _f64(grad), _f64(jac), _f64(w)
    x0 = _f64(np.asarray(x0, dtype=np.float64).reshape(3))
    return _load().or_gauss_flux_w(len(x), _p(w), _p(x), _p(grad), _p(jac), _p(x0))


# ---------------------------------------------------------------- quadratic patches
def geometry_quad(verts, tris6, sigma=None, n: int = 4, subdiv: int = 0):
    """sigma_j (0.5 sqrt(2 area_j), the curved patch's area by the n x n
    rule, or the given sigma) and the corner vertex pseudonormals of a mesh of
    6-node quadratic patches (corners P1..P3, then the nodes of edges 1-2,
    2-3, 3-1)."""
    verts = _f64(verts)
    tris6 = np.ascontiguousarray(tris6, dtype=np.int32)
    nv, m = len(verts), len(tris6)
    ru, rv, rw = simplex_rule(n, subdiv)
    sig = np.empty(m)
    vpn = np.empty((nv, 3))
    sig_in = _f64(sigma) if sigma is not None else None
    rc = _load().or_geometry_quad(nv, _p(verts), m, _p(tris6), _p(sig_in) if sig_in is not None else None,
                                  len(ru), _p(ru), _p(rv), _p(rw), _p(sig), _p(vpn))
    if rc != 0:
        raise ValueError("a corner vertex has zero total angle")
    return dict(sigma=sig, vpn=vpn)


def sources_quad(verts, tris6, sigma=None, n: int = 4, subdiv: int = 0):
    """Source nodes on quadratic patches: y = T(u_k, v_k), nw = w_k (T_u x T_v)."""
    verts = _f64(verts)
    tris6 = np.ascontiguousarray(tris6, dtype=np.int32)
    geo = geometry_quad(verts, tris6, sigma, n, subdiv)
    ru, rv, rw = simplex_rule(n, subdiv)
    m, nq = len(tris6), len(ru)
    y, nw, sg = np.empty((m * nq, 3)), np.empty((m * nq, 3)), np.empty(m * nq)
    _load().or_sources_quad(_p(verts), m, _p(tris6), _p(geo["sigma"]), nq, _p(ru), _p(rv), _p(rw), _p(y),
                            _p(nw), _p(sg))
    return y, nw, sg


def chart_nodes_quad_at(verts, tris6, tri, uv, sigma=None, n: int = 4, subdiv: int = 0):
    """x0 = T(u, v) on the quadratic patch, H(u, v) linear in its corner
    pseudonormals, and sigma of the patch (sigma by the n x n source rule's
    area when not given)."""
    verts = _f64(verts)
    tris6 = np.ascontiguousarray(tris6, dtype=np.int32)
    geo = geometry_quad(verts, tris6, sigma, n, subdiv)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    uv = _f64(uv)
    k = len(tri)
    x0, hd, sl = np.empty((k, 3)), np.empty((k, 3)), np.empty(k)
    _load().or_chart_nodes_quad_at(_p(verts), _p(tris6), _p(geo["vpn"]), _p(geo["sigma"]), k, _p(tri), _p(uv),
                                   _p(x0), _p(hd), _p(sl))
    return x0, hd, sl


def chart_frames_quad_at(verts, tris6, tri, uv, h, grad, n: int = 4, subdiv: int = 0):
    """x_u, x_v and |x_u x x_v| of charts on quadratic patches at explicit nodes."""
    verts = _f64(verts)
    tris6 = np.ascontiguousarray(tris6, dtype=np.int32)
    geo = geometry_quad(verts, tris6, None, n, subdiv)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    uv, h, grad = _f64(uv), _f64(h), _f64(grad)
    k = len(tri)
    xu, xv, jac = np.empty((k, 3)), np.empty((k, 3)), np.empty(k)
    _load().or_chart_frames_quad_at(_p(verts), _p(tris6), _p(geo["vpn"]), k, _p(tri), _p(uv), _p(h), _p(grad),
                                    _p(xu), _p(xv), _p(jac))
    return xu, xv, jac
