"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a limit, a library routine, brute-force volume quadrature, finite
differences, or a value printed in the paper.  A plausible mistake in the
oracle (a dropped term, a wrong sign, a transposed operand, a wrong weight)
fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy.optimize import brentq
from scipy.special import erf

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
SQ2 = math.sqrt(2.0)


def box_phi(x, a, s):
    """Constant-sigma Gaussian convolution of the box [-a,a]^3 (eq. basemodelg)."""
    t = 0.5 * (erf((a - x) / (SQ2 * s)) + erf((a + x) / (SQ2 * s)))
    return np.prod(t, axis=1)


def box_grad(x, a, s):
    t = 0.5 * (erf((a - x) / (SQ2 * s)) + erf((a + x) / (SQ2 * s)))
    c = 1.0 / (math.sqrt(2.0 * math.pi) * s)
    dt = c * (np.exp(-(a + x) ** 2 / (2 * s * s)) - np.exp(-(a - x) ** 2 / (2 * s * s)))
    g = np.empty_like(x)
    for i in range(3):
        o = [k for k in range(3) if k != i]
        g[:, i] = dt[:, i] * t[:, o[0]] * t[:, o[1]]
    return g


# ---------------------------------------------------------------- rules
def test_gauss_legendre_matches_library(oracle_mod):
    for n in (1, 2, 3, 4, 6, 8, 12, 16):
        x, w = oracle_mod.gauss_legendre01(n)
        z, wz = np.polynomial.legendre.leggauss(n)
        np.testing.assert_allclose(x, np.sort(0.5 * (z + 1.0)), atol=1e-15)
        np.testing.assert_allclose(w, 0.5 * wz[np.argsort(z)], atol=1e-15)


@pytest.mark.parametrize("n,subdiv", [(1, 0), (3, 0), (4, 1), (6, 0), (5, 2)])
def test_simplex_rule_exact_on_monomials(oracle_mod, n, subdiv):
    u, v, w = oracle_mod.simplex_rule(n, subdiv)
    assert len(u) == n * n * 4 ** subdiv
    assert np.all(u >= 0) and np.all(v >= 0) and np.all(u + v <= 1 + 1e-15)
    assert abs(w.sum() - 0.5) < 1e-15
    # int_{T0} u^a v^b = a! b! / (a+b+2)!, exact for a+b <= 2n-2
    for a in range(0, 2 * n - 1):
        for b in range(0, 2 * n - 1 - a):
            exact = math.factorial(a) * math.factorial(b) / math.factorial(a + b + 2)
            assert abs((w * u ** a * v ** b).sum() - exact) < 1e-15 * max(1.0, 1.0 / exact) * 10


# ---------------------------------------------------------------- kernel
def _golden_series():
    num, den = [], []
    with open(os.path.join(GOLDEN, "kerpsi_series.txt")) as fh:
        for ln in fh:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            a, b = ln.split()
            if a in ("accuracy", "umax"):
                continue
            num.append(float(a))
            den.append(float(b))
    return np.array(num) / np.array(den)


def test_small_u_series_matches_paper_coefficients(oracle_mod):
    """eq. kerpsi_asymp: f = (2/3 - 2u^2/5 + u^4/7 - u^6/27 + u^8/132) / (4 sqrt(2 pi^3) sigma^3)
    to about 1e-13 relative for u < 0.1."""
    c = _golden_series()
    sig = 0.37
    for u in np.linspace(0.0, 0.1, 23):
        rho = u * SQ2 * sig
        f, _ = oracle_mod.radial(rho, sig)
        p = sum(c[k] * u ** (2 * k) for k in range(5))
        ref = p / (4.0 * math.sqrt(2.0 * math.pi ** 3) * sig ** 3)
        assert abs(f - ref) <= 3e-13 * abs(ref)


def test_series_and_closed_form_agree_on_overlap(oracle_mod):
    """The oracle switches from series to closed form at u = 0.5; compare each
    side with the closed forms evaluated here with scipy's erf (P8)."""
    sig = 0.05
    for u in np.linspace(0.3, 0.75, 40):
        rho = u * SQ2 * sig
        f, F = oracle_mod.radial(rho, sig)
        g = erf(u) - 2.0 * u / math.sqrt(math.pi) * math.exp(-u * u)
        f_ref = g / (4 * math.pi * rho ** 3)
        F_ref = (math.sqrt(2 / math.pi) * (rho / sig) ** 3 * math.exp(-u * u) - 3 * g) / (4 * math.pi * rho ** 5)
        assert abs(f - f_ref) <= 1e-13 * abs(f_ref)
        assert abs(F - F_ref) <= 1e-11 * abs(F_ref)


def test_radial_derivative_is_consistent(oracle_mod):
    """F = f'(rho)/rho, by Richardson-extrapolated central differences of f."""
    sig = 0.2
    for u in (0.05, 0.2, 0.45, 0.55, 1.0, 2.5, 6.0):
        rho = u * SQ2 * sig
        h = 1e-3 * rho
        d1 = (oracle_mod.radial(rho + h, sig)[0] - oracle_mod.radial(rho - h, sig)[0]) / (2 * h)
        d2 = (oracle_mod.radial(rho + h / 2, sig)[0] - oracle_mod.radial(rho - h / 2, sig)[0]) / h
        d = (4 * d2 - d1) / 3
        F = oracle_mod.radial(rho, sig)[1]
        assert abs(d / rho - F) <= 1e-8 * abs(F)


def test_laplace_limit_beyond_8_sigma(oracle_mod):
    """Sec. 4.4: beyond 8 sigma the kernel is the Laplace double layer
    (eq. kerapprox) to near double precision.  The neglected relative part is
    erfc(u) + (2u/sqrt pi) e^{-u^2}, below 1e-13 at 8 sigma."""
    txt = open(os.path.join(GOLDEN, "cutoff_8sigma.txt")).read().split()
    eb = float(txt[txt.index("erf_bound") + 1])
    xb = float(txt[txt.index("exp_bound") + 1])
    assert 1 - erf(8 / SQ2) <= eb and math.exp(-32) <= xb
    sig = 0.01
    for c in (8.0, 9.0, 12.0, 40.0):
        rho = c * sig
        f, F = oracle_mod.radial(rho, sig)
        tail = math.erfc(c / SQ2) + c * math.sqrt(2 / math.pi) * math.exp(-c * c / 2)
        assert abs(f * 4 * math.pi * rho ** 3 - 1.0) <= tail + 1e-15
        assert tail < 1e-13
        # the gradient's radial factor keeps a (rho/sigma)^3 e^{-u^2} term: at
        # 8 sigma it is still 5e-12 relative, which bounds the FP64 cutoff error
        ftail = 3 * tail + math.sqrt(2 / math.pi) * c ** 3 * math.exp(-c * c / 2)
        assert abs(F * 4 * math.pi * rho ** 5 + 3.0) <= ftail + 1e-14


# ---------------------------------------------------------------- Phi
@pytest.fixture(scope="module")
def c1_fine(oracle_mod):
    w = synth.cube_c1(400)
    m = w["mesh"]
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 8, 2)
    phi, gr = oracle_mod.phi_grad(y, nw, sg, w["targets"])
    return w, phi, gr


def test_box_closed_form_phi_and_grad(c1_fine):
    """P1: the cube's discrete sum converges to the separable erf product
    (eq. basemodelg with V = [-1,1]^3, sigma = 0.1) and its gradient."""
    w, phi, gr = c1_fine
    x = w["targets"]
    assert np.abs(phi - box_phi(x, 1.0, 0.1)).max() < 1e-12
    assert np.abs(gr - box_grad(x, 1.0, 0.1)).max() < 1e-11


def test_box_spectral_convergence(oracle_mod):
    """P1, convergence: the C1 rule (4x4 on 4 children) is accurate to about
    1e-5; refining the rule drives the error toward rounding."""
    w = synth.cube_c1(300)
    m, x = w["mesh"], w["targets"]
    ex = box_phi(x, 1.0, 0.1)
    errs = []
    for n, sd in ((4, 1), (6, 1), (8, 1), (8, 2)):
        y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, n, sd)
        phi, _ = oracle_mod.phi_grad(y, nw, sg, x)
        errs.append(np.abs(phi - ex).max())
    assert errs[0] < 5e-5
    assert errs[0] > errs[1] > errs[2] > errs[3]
    assert errs[3] < 1e-12


def _solid_angle(x, verts, tris):
    """Van Oosterom-Strackee signed solid angle of each triangle seen from x."""
    a = verts[tris[:, 0]] - x
    b = verts[tris[:, 1]] - x
    c = verts[tris[:, 2]] - x
    la, lb, lc = (np.linalg.norm(v, axis=1) for v in (a, b, c))
    num = np.einsum("ij,ij->i", a, np.cross(b, c))
    den = la * lb * lc + np.einsum("ij,ij->i", a, b) * lc + np.einsum("ij,ij->i", a, c) * lb \
        + np.einsum("ij,ij->i", b, c) * la
    return 2.0 * np.arctan2(num, den)


def test_sigma_to_zero_is_solid_angle(oracle_mod):
    """P2: as sigma -> 0, Phi off the surface is sum(solid angle)/(4 pi):
    1 inside, 0 outside (Sec. 5, Gauss flux).  Per-triangle sigma varies."""
    g = synth.rng(11)
    m = synth.icosphere(1)
    sig = g.uniform(5e-4, 2e-3, m.m)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, sig, 10, 3)
    x = np.concatenate([g.uniform(-0.5, 0.5, (6, 3)), g.normal(size=(6, 3))])
    x[6:] *= (1.6 / np.linalg.norm(x[6:], axis=1))[:, None]
    phi, _ = oracle_mod.phi_grad(y, nw, sg, x)
    ref = np.array([_solid_angle(p, m.verts, m.tris).sum() / (4 * math.pi) for p in x])
    np.testing.assert_allclose(ref[:6], 1.0, atol=1e-12)
    np.testing.assert_allclose(ref[6:], 0.0, atol=1e-12)
    assert np.abs(phi - ref).max() < 1e-9


def _tet_volume_rule(P, n):
    """Tensor Gauss-Legendre rule on a tetrahedron by collapsing the unit cube."""
    z, wz = np.polynomial.legendre.leggauss(n)
    t, wt = 0.5 * (z + 1), 0.5 * wz
    A, B, C = np.meshgrid(t, t, t, indexing="ij")
    W = (wt[:, None, None] * wt[None, :, None] * wt[None, None, :])
    s1 = A
    s2 = A * B
    s3 = A * B * C
    jac = A * A * B
    bary1 = s1 - s2
    bary2 = s2 - s3
    bary3 = s3
    pts = (P[0][None, :] + bary1.ravel()[:, None] * (P[1] - P[0]) + bary2.ravel()[:, None] * (P[2] - P[0])
           + bary3.ravel()[:, None] * (P[3] - P[0]))
    vol6 = abs(np.linalg.det(np.stack([P[1] - P[0], P[2] - P[0], P[3] - P[0]])))
    return pts, (W * jac).ravel() * vol6


def test_tetrahedron_volume_quadrature(oracle_mod):
    """P5: the boundary form (eq. surf) equals brute-force volume quadrature of
    the Gaussian convolution (eq. basemodelg) on a tetrahedron, for Phi and
    grad Phi (grad G = -(x - x') G / sigma^2)."""
    P = np.array([[0.0, 0.0, 0.0], [1.0, 0.1, 0.0], [0.2, 0.9, 0.1], [0.3, 0.2, 0.8]])
    tris = np.array([[0, 2, 1], [0, 1, 3], [1, 2, 3], [0, 3, 2]], dtype=np.int32)
    s = 0.25
    y, nw, sg = oracle_mod.sources(P, tris, np.full(4, s), 14, 2)
    x = np.array([[0.35, 0.3, 0.25], [0.0, 0.0, 0.0], [0.9, 0.9, 0.9], [-0.3, 0.5, 0.2],
                  [0.5, 0.05, 0.0]])
    phi, gr = oracle_mod.phi_grad(y, nw, sg, x)
    pts, wv = _tet_volume_rule(P, 40)
    for i, xi in enumerate(x):
        d = xi[None, :] - pts
        G = np.exp(-(d ** 2).sum(1) / (2 * s * s)) / (2 * math.pi * s * s) ** 1.5
        assert abs((wv * G).sum() - phi[i]) < 1e-11
        gref = -(wv[:, None] * d * G[:, None]).sum(0) / (s * s)
        assert np.abs(gref - gr[i]).max() < 1e-10


def _ball_phi(rho, R, s):
    rho = np.asarray(rho, dtype=np.float64)
    out = np.empty_like(rho)
    z = rho < 1e-8
    r = rho[~z]
    out[~z] = 0.5 * (erf((R - r) / (SQ2 * s)) + erf((R + r) / (SQ2 * s))) + \
        s / (r * math.sqrt(2 * math.pi)) * (np.exp(-(R + r) ** 2 / (2 * s * s)) - np.exp(-(R - r) ** 2 / (2 * s * s)))
    out[z] = erf(R / (SQ2 * s)) - math.sqrt(2 / math.pi) * (R / s) * math.exp(-R * R / (2 * s * s))
    return out


def test_ball_closed_form_on_icosphere(oracle_mod):
    """P4 (approximate): a fine icosphere with constant sigma approaches the
    Gaussian convolution of the unit ball, up to the O(h^2) geometric error."""
    s = 0.15
    rr = np.array([0.4, 0.8, 0.95, 1.0, 1.05, 1.3])
    x = np.stack([rr / math.sqrt(3)] * 3, axis=1)
    errs = []
    for level in (3, 4, 5):
        m = synth.icosphere(level)
        y, nw, sg = oracle_mod.sources(m.verts, m.tris, np.full(m.m, s), 3, 0)
        phi, _ = oracle_mod.phi_grad(y, nw, sg, x)
        errs.append(np.abs(phi - _ball_phi(rr, 1.0, s)).max())
    # each level halves the edge: the inscribed polyhedron's error drops ~4x
    assert 3.0 < errs[0] / errs[1] < 5.0 and 3.0 < errs[1] / errs[2] < 5.0
    assert errs[2] < 6e-4


def test_limits_deep_inside_and_far_outside(oracle_mod):
    """P6: Phi -> 1 deep inside, -> 0 far outside; Laplace limit far away."""
    m = synth.cube(1.0, 3)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, np.full(m.m, 0.05), 8, 1)
    phi, gr = oracle_mod.phi_grad(y, nw, sg, np.array([[0.0, 0.0, 0.0], [0.2, -0.1, 0.3],
                                                       [30.0, 0.0, 0.0], [0, -25.0, 10.0]]))
    assert abs(phi[0] - 1) < 1e-13 and abs(phi[1] - 1) < 1e-13
    assert abs(phi[2]) < 1e-12 and abs(phi[3]) < 1e-12
    assert np.abs(gr).max() < 1e-10


def test_gradient_by_finite_differences(oracle_mod):
    """P7: grad Phi against Richardson-extrapolated central differences of Phi,
    on a jittered graded torus with per-triangle sigma (pins the sign of the
    second term of eq. gradPhi for variable sigma)."""
    m = synth.torus(1.0, 0.3, 24, 8, 5.0, 0.05, seed=7)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 3, 0)
    g = synth.rng(12)
    x = synth.targets_near_surface(m, 12, g, 2.0)
    _, gr = oracle_mod.phi_grad(y, nw, sg, x)
    h = 2e-4
    fd = np.empty_like(gr)
    for i in range(3):
        e = np.zeros(3)
        e[i] = 1.0
        d1 = (oracle_mod.phi_grad(y, nw, sg, x + h * e)[0] - oracle_mod.phi_grad(y, nw, sg, x - h * e)[0]) / (2 * h)
        d2 = (oracle_mod.phi_grad(y, nw, sg, x + h / 2 * e)[0] - oracle_mod.phi_grad(y, nw, sg, x - h / 2 * e)[0]) / h
        fd[:, i] = (4 * d2 - d1) / 3
    assert np.abs(fd - gr).max() < 1e-7 * np.abs(gr).max()


# ---------------------------------------------------------------- geometry
def test_sigma_rule_and_pseudonormals(oracle_mod):
    """Default sigma rule (0.5 sqrt(2 area)); pseudonormals (eq. mkvertexpn) of
    a cube: n_hat at face-interior vertices, (n1+n2+n3)/3 at corners (each face
    contributes a total angle pi/2), (n1+n2)/2 on edges."""
    m = synth.cube(1.0, 4)
    geo = oracle_mod.geometry(m.verts, m.tris, None)
    np.testing.assert_allclose(geo["sigma"], synth.sigma_half_sqrt2area(m.verts, m.tris), rtol=1e-15)
    v = m.verts
    nb = (np.abs(np.abs(v) - 1.0) < 1e-12).sum(1)
    for i in range(len(v)):
        n = np.where(np.abs(np.abs(v[i]) - 1.0) < 1e-12, np.sign(v[i]), 0.0)
        np.testing.assert_allclose(geo["vpn"][i], n / nb[i], atol=1e-15)


def test_chart_nodes_on_flat_face_match_closed_form_root(oracle_mod):
    """P3: on triangles interior to a cube face H = n_hat, so Newton's root
    h solves Phi_box(x0 + h n_hat) = 1/2 (a 1-D root of the erf product); the
    oracle's h agrees with brentq on the closed form to quadrature error."""
    m = synth.cube(1.0, 4)
    s = 0.1
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, np.full(m.m, s), 8, 2)
    x0, hd, sl = oracle_mod.chart_nodes(m.verts, m.tris, np.full(m.m, s), 3)
    v = m.verts
    inner = np.all(np.abs(v) < 1 - 1e-9, axis=1) | (np.sum(np.abs(np.abs(v) - 1) < 1e-9, axis=1) == 1)
    tri_ok = np.all(inner[m.tris], axis=1)
    sel = np.repeat(tri_ok, 9)
    x0, hd, sl = x0[sel][:40], hd[sel][:40], sl[sel][:40]
    out = oracle_mod.solve_charts(y, nw, sg, x0, hd, sl, tol=1e-13, max_iter=20)
    assert np.all(out["status"] == oracle_mod.ST_CONVERGED)
    for i in range(len(x0)):
        n = hd[i]
        assert abs(np.linalg.norm(n) - 1) < 1e-14
        root = brentq(lambda h: box_phi((x0[i] + h * n)[None, :], 1.0, s)[0] - 0.5, -0.3, 0.3, xtol=1e-16)
        assert abs(out["h"][i] - root) < 1e-12


def test_newton_reaches_half_level_on_torus(oracle_mod):
    """Chart positions on a curved mesh: parity unpinned beyond Phi(x) = 1/2,
    which is re-evaluated here by the direct sum."""
    m = synth.torus(1.0, 0.3, 24, 8, 5.0, 0.05, seed=9)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, m.sigma, 3, 0)
    x0, hd, sl = oracle_mod.chart_nodes(m.verts, m.tris, m.sigma, 2)
    out = oracle_mod.solve_charts(y, nw, sg, x0[:64], hd[:64], sl[:64], tol=1e-12)
    assert np.all(out["status"] == 0)
    phi, _ = oracle_mod.phi_grad(y, nw, sg, out["x"])
    assert np.abs(phi - 0.5).max() < 1e-12
    assert np.all(out["iters"] <= 8)


def test_newton_reports_nonconvergence(oracle_mod):
    """A capped solve reports MAXITER per node instead of failing (the paper's
    failure mode, Sec. 5, must be reported, not crash)."""
    m = synth.cube(1.0, 2)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, np.full(m.m, 0.2), 3, 0)
    x0, hd, sl = oracle_mod.chart_nodes(m.verts, m.tris, np.full(m.m, 0.2), 2)
    out = oracle_mod.solve_charts(y, nw, sg, x0, hd, sl, tol=1e-14, max_iter=1)
    assert np.all((out["status"] & 255) == oracle_mod.ST_MAXITER)
    assert np.all(out["iters"] == 1)


# ---------------------------------------------------------------- local coordinates and Gauss flux

def _exact_sphere_charts(n):
    """Unit sphere charted by radial projection of an icosphere's flat
    triangles: positions, derivatives in (u, v) and |x_u x x_v| written out
    from the projection x = T/|T| (no oracle code involved)."""
    m = synth.icosphere(2)
    V = m.verts / np.linalg.norm(m.verts, axis=1)[:, None]
    cu, cv, _ = _rule(n)
    P1, P2, P3 = V[m.tris[:, 0]], V[m.tris[:, 1]], V[m.tris[:, 2]]
    Tu, Tv = P2 - P1, P3 - P1
    T = P1[:, None, :] + cu[None, :, None] * Tu[:, None, :] + cv[None, :, None] * Tv[:, None, :]
    nT = np.linalg.norm(T, axis=2)[..., None]
    xu = Tu[:, None, :] / nT - T * np.sum(T * Tu[:, None, :], axis=2)[..., None] / nT ** 3
    xv = Tv[:, None, :] / nT - T * np.sum(T * Tv[:, None, :], axis=2)[..., None] / nT ** 3
    jac = np.linalg.norm(np.cross(xu, xv), axis=2)
    return (T / nT).reshape(-1, 3), jac.ravel()


def _rule(n):
    """Duffy n x n rule on the reference triangle, written out with numpy's
    Gauss-Legendre (u = xi (1 - eta), v = xi eta, w = w_xi w_eta xi)."""
    g, wg = np.polynomial.legendre.leggauss(n)
    g, wg = 0.5 * (g + 1), 0.5 * wg
    xi, eta = np.meshgrid(g, g, indexing="ij")
    wx, we = np.meshgrid(wg, wg, indexing="ij")
    return (xi * (1 - eta)).ravel(), (xi * eta).ravel(), (wx * we * xi).ravel()


def test_gauss_flux_exact_sphere(oracle_mod):
    """Sec. 5: eps0 = 1 + flux of grad 1/(4 pi |x0 - x|) through a closed
    surface is 0 for x0 inside and 1 outside; on an exactly charted sphere
    the chart quadrature converges spectrally to those values."""
    # the oracle's chart rule is the same Duffy rule (pinned above); check
    # the point order used by the flux weights
    u, v, w = oracle_mod.simplex_rule(8, 0)
    cu, cv, cw = _rule(8)
    assert np.allclose(u, cu) and np.allclose(v, cv) and np.allclose(w, cw)
    errs = []
    for n in (3, 5, 8):
        x, jac = _exact_sphere_charts(n)
        # outward normal is x; the oracle takes it as -grad Phi / |grad Phi|
        e_in = [oracle_mod.gauss_flux(x, -x, jac, x0, n=n) for x0 in ((0.1, -0.2, 0.05), (0.0, 0.0, 0.0))]
        e_out = oracle_mod.gauss_flux(x, -x, jac, (2.0, 0.3, 0.0), n=n)
        errs.append(max(abs(e) for e in e_in))
        assert abs(e_out - 1.0) < 1e-6
    assert errs[0] > 1e3 * errs[1] and errs[1] > 1e3 * errs[2]
    assert errs[2] < 1e-13


@pytest.fixture(scope="module")
def small_sphere_charts(oracle_mod):
    """Icosphere level 1 (80 triangles), sigma by the workloads' rule, 4x4
    sources; charts solved to 1e-14 at the rule points."""
    m = synth.icosphere(1)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, None, 4, 0)
    geo = oracle_mod.geometry(m.verts, m.tris, None)
    return m, (y, nw, sg), geo


def _solve_at(oracle_mod, m, src, geo, j, u, v):
    """Chart point of triangle j at (u, v): Newton on h along H(u, v)."""
    P = m.verts[m.tris[j]]
    Hn = geo["vpn"][m.tris[j]]
    x0 = P[0] + u * (P[1] - P[0]) + v * (P[2] - P[0])
    H = Hn[0] + u * (Hn[1] - Hn[0]) + v * (Hn[2] - Hn[0])
    r = oracle_mod.solve_charts(*src, x0[None], H[None], geo["sigma"][j:j + 1], tol=1e-14, max_iter=40)
    assert r["status"][0] == 0
    return r["x"][0], r["h"][0]


def test_chart_frames_match_finite_differences(oracle_mod, small_sphere_charts):
    """eq. u_vector / U_vector_2 (and v): x_u, x_v from the solved h and grad
    Phi equal central differences of the solved chart x(u, v) = T + h H."""
    m, src, geo = small_sphere_charts
    d = 1e-4
    for j, u, v in ((3, 0.2, 0.3), (41, 0.55, 0.1), (77, 0.1, 0.7)):
        x, h = _solve_at(oracle_mod, m, src, geo, j, u, v)
        _, g = oracle_mod.phi_grad(*src, x[None])
        xu, xv, jac = oracle_mod.chart_frames(m.verts, m.tris, np.full(m.m, h), np.tile(g, (m.m, 1)),
                                              uv=(np.array([u]), np.array([v])))
        fu = (_solve_at(oracle_mod, m, src, geo, j, u + d, v)[0] - _solve_at(oracle_mod, m, src, geo, j, u - d, v)[0]) / (2 * d)
        fv = (_solve_at(oracle_mod, m, src, geo, j, u, v + d)[0] - _solve_at(oracle_mod, m, src, geo, j, u, v - d)[0]) / (2 * d)
        scale = np.linalg.norm(fu) + np.linalg.norm(fv)
        assert np.abs(xu[j] - fu).max() < 1e-7 * scale
        assert np.abs(xv[j] - fv).max() < 1e-7 * scale
        assert abs(jac[j] - np.linalg.norm(np.cross(fu, fv))) < 1e-7 * scale ** 2
        # the frame is tangent to the level set
        assert abs(xu[j] @ g[0]) < 1e-9 * np.linalg.norm(xu[j]) * np.linalg.norm(g[0])


def test_gauss_flux_of_solved_charts_converges(oracle_mod, small_sphere_charts):
    """End to end: charts solved on the level set, their frames and the flux
    about an interior point.  Adjacent charts meet exactly on shared edges,
    so eps0 falls with the chart rule's order."""
    m, src, geo = small_sphere_charts
    out = []
    for n in (3, 5, 7):
        x0, hd, sl = oracle_mod.chart_nodes(m.verts, m.tris, None, n)
        r = oracle_mod.solve_charts(*src, x0, hd, sl, tol=1e-14, max_iter=40)
        assert (r["status"] == 0).all()
        _, g = oracle_mod.phi_grad(*src, r["x"])
        _, _, jac = oracle_mod.chart_frames(m.verts, m.tris, r["h"], g, n=n)
        out.append(abs(oracle_mod.gauss_flux(r["x"], g, jac, (0.05, -0.1, 0.02), n=n)))
    # measured: 1.4e-5, 4.7e-9, 9.9e-12
    assert out[0] > 100 * out[1] and out[1] > 100 * out[2]
    assert out[2] < 1e-10


# ---------------------------------------------------------------- target-dependent sigma (eq. sigma2)

def test_enclosing_ball_diameters(oracle_mod):
    """D_j: longest edge for right and obtuse triangles, the circumdiameter
    abc/(2 area) for acute ones (closed forms written out here)."""
    P = np.array([[0, 0, 0], [1, 0, 0], [0.5, np.sqrt(3) / 2, 0],        # equilateral, side 1
                  [0, 0, 1], [3, 0, 1], [0, 4, 1],                        # right, 3-4-5
                  [0, 0, 2], [4, 0, 2], [1, 0.5, 2],                      # obtuse
                  [0, 0, 3], [2, 0, 3], [0.8, 1.5, 3]], dtype=float)      # acute scalene
    T = np.arange(12, dtype=np.int32).reshape(4, 3)
    _, sj, dmax = oracle_mod.sigma_sources(P, T, lam=1.0)
    a, b, c = np.linalg.norm(P[10] - P[9]), np.linalg.norm(P[11] - P[10]), np.linalg.norm(P[11] - P[9])
    area = 0.5 * np.linalg.norm(np.cross(P[10] - P[9], P[11] - P[9]))
    want = [2 / np.sqrt(3), 5.0, 4.0, a * b * c / (2 * area)]
    assert np.allclose(sj, want, rtol=1e-14, atol=0)
    assert dmax == max(want)


def _graded_small():
    m = synth.torus(1.0, 0.3, 24, 8, 8.0, 0.05, 7)
    return m


def test_sigma_x_constant_when_all_equal(oracle_mod):
    m = synth.cube(1.0, 4)                    # every triangle right isosceles, legs 0.5
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    assert np.allclose(sj, 0.5 * np.sqrt(2) / 2.5, rtol=1e-15)
    x = synth.targets_uniform(50, -1.5, 1.5, synth.rng(41))
    s, gs = oracle_mod.sigma_x(c, sj, oracle_mod.sigma0_default(dmax), x)
    assert np.allclose(s, sj[0], rtol=1e-14)
    assert np.abs(gs).max() < 1e-12


def test_sigma_x_gradient_finite_differences(oracle_mod):
    m = _graded_small()
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    s0 = oracle_mod.sigma0_default(dmax)
    x = synth.targets_near_surface(m, 20, synth.rng(42), 3.0)
    _, gs = oracle_mod.sigma_x(c, sj, s0, x)
    d = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = d
        fd = (oracle_mod.sigma_x(c, sj, s0, x + e)[0] - oracle_mod.sigma_x(c, sj, s0, x - e)[0]) / (2 * d)
        assert np.abs(fd - gs[:, k]).max() < 1e-8 * (np.abs(gs).max() + 1e-3)
    # sigma varies on this graded mesh
    assert np.ptp(sj) > 0.5 * sj.mean()


def test_sigma_x_phi_reduces_to_constant_sigma(oracle_mod):
    """With every sigma_j equal, sigma(x) is that constant and the sigma(x)
    sum is the constant-sigma sum (pinned to the box's erf product above)."""
    m = synth.cube(1.0, 4)
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    x = synth.targets_uniform(200, -1.5, 1.5, synth.rng(43))
    s, gs = oracle_mod.sigma_x(c, sj, oracle_mod.sigma0_default(dmax), x)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, np.full(m.m, sj[0]), 4, 1)
    p1, g1 = oracle_mod.phi_grad_sigx(y, nw, x, s, gs)
    p0, g0 = oracle_mod.phi_grad(y, nw, sg, x)
    assert np.abs(p1 - p0).max() < 1e-13
    assert np.abs(g1 - g0).max() < 1e-11


def test_sigma_x_grad_phi_finite_differences(oracle_mod):
    """eq. gradPhi with sigma(x): its third term, (dPhi/dsigma) grad sigma
    with the corrected sign, is needed to match central differences of Phi."""
    m = _graded_small()
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    s0 = oracle_mod.sigma0_default(dmax)
    y, nw, _ = oracle_mod.sources(m.verts, m.tris, None, 6, 0)
    x = synth.targets_near_surface(m, 12, synth.rng(44), 2.0)

    def phi_at(p):
        s, gs = oracle_mod.sigma_x(c, sj, s0, p)
        return oracle_mod.phi_grad_sigx(y, nw, p, s, gs)

    _, g = phi_at(x)
    s, gs = oracle_mod.sigma_x(c, sj, s0, x)
    d = 1e-5
    fd = np.empty_like(g)
    for k in range(3):
        e = np.zeros(3)
        e[k] = d
        fd[:, k] = (phi_at(x + e)[0] - phi_at(x - e)[0]) / (2 * d)
    scale = np.abs(g).max()
    assert np.abs(fd - g).max() < 1e-7 * scale
    # without the grad-sigma term (or with the printed sign) the match fails
    dps = np.empty(len(x))
    for t in range(len(x)):
        r = y - x[t]
        u2 = np.sum(r * r, axis=1) / (2 * s[t] ** 2)
        dps[t] = -np.sum(np.sum(nw * r, axis=1) * np.exp(-u2)) / (2 * np.sqrt(2) * np.pi ** 1.5 * s[t] ** 4)
    g_no = g - dps[:, None] * gs
    g_flip = g - 2 * dps[:, None] * gs
    assert np.abs(fd - g_no).max() > 100 * np.abs(fd - g).max()
    assert np.abs(fd - g_flip).max() > 100 * np.abs(fd - g).max()


def test_sigma_x_charts_converge(oracle_mod):
    m = _graded_small()
    c, sj, dmax = oracle_mod.sigma_sources(m.verts, m.tris)
    s0 = oracle_mod.sigma0_default(dmax)
    y, nw, _ = oracle_mod.sources(m.verts, m.tris, None, 6, 0)
    x0, hd, _ = oracle_mod.chart_nodes(m.verts, m.tris, None, 4)
    sel = np.arange(0, len(x0), 37)
    sloc = np.repeat(sj, 16)[sel]
    r = oracle_mod.solve_charts_sigx(y, nw, c, sj, s0, x0[sel], hd[sel], sloc, tol=1e-13, max_iter=30)
    assert (r["status"] == 0).all()
    s, gs = oracle_mod.sigma_x(c, sj, s0, r["x"])
    p, _ = oracle_mod.phi_grad_sigx(y, nw, r["x"], s, gs)
    assert np.abs(p - 0.5).max() < 1e-13


# ---------------------------------------------------------------- Hessian and curvatures

def test_radial_G_is_derivative_of_F(oracle_mod):
    """G = F'(rho)/rho on both branches (series below u = 1, closed form
    above), and its Laplace limit 15/(4 pi rho^7)."""
    s = 0.1
    a = 1 / (np.sqrt(2) * s)
    for u in (0.05, 0.3, 0.7, 0.99, 1.01, 1.5, 3.0, 6.0):
        rho = u / a
        d = 1e-5 * rho
        F = lambda r: oracle_mod.radial(r, s)[1]
        fd = (8 * (F(rho + d) - F(rho - d)) - (F(rho + 2 * d) - F(rho - 2 * d))) / (12 * d) / rho
        G = oracle_mod.radial_G(rho, s)
        assert abs(fd / G - 1) < 1e-8, (u, fd, G)
    rho = 9.0 / a
    assert abs(oracle_mod.radial_G(rho, s) * 4 * np.pi * rho ** 7 / 15 - 1) < 1e-14


def test_hessian_box_closed_form(oracle_mod):
    """Second derivatives of the box's erf product (P1 differentiated twice)."""
    from scipy.special import erf as serf
    m = synth.cube(1.0, 4)
    sig = 0.1
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, np.full(m.m, sig), 8, 2)
    x = synth.targets_uniform(20, -1.3, 1.3, synth.rng(61))
    _, _, H = oracle_mod.phi_grad_hess(y, nw, sg, x)
    A, c = 1.0, np.sqrt(2) * sig
    ph = lambda t: 0.5 * (serf((A - t) / c) + serf((A + t) / c))
    d1 = lambda t: (np.exp(-(A + t) ** 2 / (2 * sig ** 2)) - np.exp(-(A - t) ** 2 / (2 * sig ** 2))) / (
        np.sqrt(2 * np.pi) * sig)
    d2 = lambda t: (-(A - t) * np.exp(-(A - t) ** 2 / (2 * sig ** 2)) -
                    (A + t) * np.exp(-(A + t) ** 2 / (2 * sig ** 2))) / (np.sqrt(2 * np.pi) * sig ** 3)
    P = [ph(x[:, i]) for i in range(3)]
    D1 = [d1(x[:, i]) for i in range(3)]
    D2 = [d2(x[:, i]) for i in range(3)]
    Hc = np.stack([D2[0] * P[1] * P[2], D1[0] * D1[1] * P[2], D1[0] * P[1] * D1[2],
                   P[0] * D2[1] * P[2], P[0] * D1[1] * D1[2], P[0] * P[1] * D2[2]], 1)
    assert np.abs(H - Hc).max() < 1e-11 * np.abs(Hc).max()


def test_hessian_finite_differences_of_gradient(oracle_mod):
    m = _graded_small()
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, None, 6, 0)
    x = synth.targets_near_surface(m, 12, synth.rng(62), 2.0)
    _, g, H = oracle_mod.phi_grad_hess(y, nw, sg, x)
    _, g0 = oracle_mod.phi_grad(y, nw, sg, x)
    assert np.abs(g - g0).max() < 1e-12 * np.abs(g0).max()
    d = 1e-5
    cols = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = d
        cols.append((oracle_mod.phi_grad(y, nw, sg, x + e)[1] - oracle_mod.phi_grad(y, nw, sg, x - e)[1]) / (2 * d))
    Hfd = np.stack([cols[0][:, 0], cols[1][:, 0], cols[2][:, 0], cols[1][:, 1], cols[2][:, 1], cols[2][:, 2]], 1)
    assert np.abs(H - Hfd).max() < 1e-7 * np.abs(H).max()
    # and the matrix FD is symmetric as the formula says
    assert np.abs(cols[0][:, 1] - cols[1][:, 0]).max() < 1e-7 * np.abs(H).max()


def test_chart_second_derivatives_match_finite_differences(oracle_mod, small_sphere_charts):
    """eq. uu_vector (and its uv, vv analogues): x_uu, x_uv equal central
    differences of the frames x_u of Newton-solved charts."""
    m, src, geo = small_sphere_charts
    y, nw, sg = src
    d = 1e-4

    def frame_at(j, u, v):
        x, h = _solve_at(oracle_mod, m, src, geo, j, u, v)
        _, g = oracle_mod.phi_grad(y, nw, sg, x[None])
        xu, xv, _ = oracle_mod.chart_frames(m.verts, m.tris, np.full(m.m, h), np.tile(g, (m.m, 1)),
                                            uv=(np.array([u]), np.array([v])))
        return x, h, g[0], xu[j], xv[j]

    for j, u, v in ((3, 0.2, 0.3), (41, 0.55, 0.1)):
        x, h, g, _, _ = frame_at(j, u, v)
        _, _, H = oracle_mod.phi_grad_hess(y, nw, sg, x[None])
        uu, uv, vv, km, kg = oracle_mod.chart_second(m.verts, m.tris, np.full(m.m, h), np.tile(g, (m.m, 1)),
                                                     np.tile(H[0], (m.m, 1)), uv=(np.array([u]), np.array([v])))
        fuu = (frame_at(j, u + d, v)[3] - frame_at(j, u - d, v)[3]) / (2 * d)
        fuv = (frame_at(j, u, v + d)[3] - frame_at(j, u, v - d)[3]) / (2 * d)
        fvv = (frame_at(j, u, v + d)[4] - frame_at(j, u, v - d)[4]) / (2 * d)
        scale = np.abs(fuu).max() + np.abs(fvv).max() + 1e-3
        assert np.abs(uu[j] - fuu).max() < 1e-6 * scale
        assert np.abs(uv[j] - fuv).max() < 1e-6 * scale
        assert np.abs(vv[j] - fvv).max() < 1e-6 * scale
        # the chart curvature equals the level set's, div(-grad Phi / |grad Phi|)
        S = np.array([[H[0, 0], H[0, 1], H[0, 2]], [H[0, 1], H[0, 3], H[0, 4]], [H[0, 2], H[0, 4], H[0, 5]]])
        gn = np.linalg.norm(g)
        kdiv = -(np.trace(S) * gn ** 2 - g @ S @ g) / gn ** 3
        assert abs(km[j] - kdiv) < 1e-9 * abs(kdiv)


def _gauss_bonnet(oracle_mod, m, n, src):
    y, nw, sg = src
    x0, hd, sl = oracle_mod.chart_nodes(m.verts, m.tris, None, n)
    r = oracle_mod.solve_charts(y, nw, sg, x0, hd, sl, tol=1e-14, max_iter=40)
    assert (r["status"] == 0).all()
    _, g, H = oracle_mod.phi_grad_hess(y, nw, sg, r["x"])
    _, _, jac = oracle_mod.chart_frames(m.verts, m.tris, r["h"], g, n=n)
    _, _, _, km, kg = oracle_mod.chart_second(m.verts, m.tris, r["h"], g, H, n=n)
    _, _, cw = oracle_mod.simplex_rule(n, 0)
    return float(np.sum(np.tile(cw, m.m) * jac * kg))


def test_gauss_bonnet_sphere_and_torus(oracle_mod, small_sphere_charts):
    """Gauss-Bonnet: the Gaussian curvature of the charts integrates to
    2 pi chi, 4 pi on a sphere and 0 on a torus, with the chart rule's error
    falling as its order grows."""
    m, src, geo = small_sphere_charts
    # measured: 2.0e-3, 6.7e-6, 5.5e-10 at n = 3, 5, 7
    errs = [abs(_gauss_bonnet(oracle_mod, m, n, src) - 4 * np.pi) for n in (3, 5, 7)]
    assert errs[0] > 10 * errs[1] and errs[1] > 10 * errs[2]
    assert errs[2] < 1e-6
    t = synth.torus(1.0, 0.4, 24, 10, 1.0, 0.0, 63)
    st = oracle_mod.sources(t.verts, t.tris, None, 6, 0)
    # measured: 2.9e-5 at n = 5, 2.8e-7 at n = 7
    assert abs(_gauss_bonnet(oracle_mod, t, 7, st)) < 5e-6


# ---------------------------------------------------------------- refinement (Sec. 3.4)

def _refined_eps(oracle_mod, m, src, n, levels):
    y, nw, sg = src
    tri, uv, w = oracle_mod.refined_nodes(m.m, n, levels)
    assert np.allclose(np.bincount(tri, weights=w, minlength=m.m), 0.5, rtol=1e-13)
    x0, hd, sl = oracle_mod.chart_nodes_at(m.verts, m.tris, tri, uv)
    r = oracle_mod.solve_charts(y, nw, sg, x0, hd, sl, tol=1e-14, max_iter=40)
    assert (r["status"] == 0).all()
    _, g = oracle_mod.phi_grad(y, nw, sg, r["x"])
    _, _, jac = oracle_mod.chart_frames_at(m.verts, m.tris, tri, uv, r["h"], g)
    return oracle_mod.gauss_flux_w(r["x"], g, jac, w, (0.05, -0.1, 0.02))


def test_refinement_converges_and_stays_closed(oracle_mod, small_sphere_charts):
    """1 -> 4 refinement of every triangle shrinks the flux error about 2^(2n)
    per level; refining a random subset (non-conforming) keeps the charts
    closed: its error stays between the unrefined and refined ones."""
    m, src, geo = small_sphere_charts
    n = 3
    e = [abs(_refined_eps(oracle_mod, m, src, n, np.full(m.m, L))) for L in (0, 1, 2)]
    # measured: 1.4e-5, 1.8e-7, 2.6e-9
    assert e[0] > 30 * e[1] and e[1] > 30 * e[2]
    mix = np.random.default_rng(64).integers(0, 2, m.m)
    em = abs(_refined_eps(oracle_mod, m, src, n, mix))
    assert e[1] < em < e[0]


def test_refined_midpoint_meets_unrefined_neighbour(oracle_mod, small_sphere_charts):
    """The midpoint of an edge shared by a refined and an unrefined triangle:
    the chart point solved from either triangle's map is the same (T and the
    linear H agree along the shared edge)."""
    m, src, geo = small_sphere_charts
    y, nw, sg = src
    T = m.tris
    j = 5
    a, b = T[j][0], T[j][1]
    k = next(i for i in range(m.m) if i != j and a in T[i] and b in T[i])

    def uv_of(i, p, q):
        """parent (u, v) of the midpoint of edge (p, q) of triangle i"""
        loc = [list(T[i]).index(p), list(T[i]).index(q)]
        bary = np.zeros(3)
        bary[loc] = 0.5
        return np.array([[bary[1], bary[2]]])

    xs = []
    for i in (j, k):
        x0, hd, sl = oracle_mod.chart_nodes_at(m.verts, m.tris, np.array([i]), uv_of(i, a, b))
        r = oracle_mod.solve_charts(y, nw, sg, x0, hd, sl, tol=1e-15, max_iter=40)
        xs.append(r["x"][0])
    assert np.abs(xs[0] - xs[1]).max() < 1e-13


# ---------------------------------------------------------------- quadratic (curved) skeletons
def test_quadratic_with_straight_edges_is_the_flat_mesh(oracle_mod):
    """6-node patches whose edge nodes sit at the edge midpoints are the flat
    triangles (the quadratic basis reproduces the affine map of eq. tparam):
    sources, sigma rule, pseudonormals, chart nodes and frames all equal the
    flat oracle's."""
    m = synth.cube(1.0, 2)
    q = synth.quadratic_from_flat(m, 0.5)
    sig = np.linspace(0.15, 0.25, m.m)
    y, nw, sg = oracle_mod.sources(m.verts, m.tris, sig, 4, 1)
    yq, nwq, sgq = oracle_mod.sources_quad(q.verts, q.tris6, sig, 4, 1)
    assert np.abs(yq - y).max() < 1e-15 and np.abs(nwq - nw).max() < 1e-15 and np.array_equal(sgq, sg)
    geo = oracle_mod.geometry(m.verts, m.tris, None)
    gq = oracle_mod.geometry_quad(q.verts, q.tris6, None, 4, 1)
    assert np.abs(gq["sigma"] - geo["sigma"]).max() < 1e-15
    assert np.abs(gq["vpn"][:m.nv] - geo["vpn"]).max() < 1e-15
    tri, uv, w = oracle_mod.refined_nodes(m.m, 3, np.zeros(m.m))
    a = oracle_mod.chart_nodes_at(m.verts, m.tris, tri, uv)
    b = oracle_mod.chart_nodes_quad_at(q.verts, q.tris6, tri, uv)
    for p, r in zip(a, b):
        assert np.abs(p - r).max() < 1e-15
    g = np.random.default_rng(5)
    h, grad = g.normal(size=len(tri)) * 0.1, g.normal(size=(len(tri), 3))
    fa = oracle_mod.chart_frames_at(m.verts, m.tris, tri, uv, h, grad)
    fb = oracle_mod.chart_frames_quad_at(q.verts, q.tris6, tri, uv, h, grad)
    for p, r in zip(fa, fb):
        assert np.abs(p - r).max() < 1e-13


def test_quadratic_reparametrised_cube_is_the_box(oracle_mod):
    """The cube's flat faces with a non-affine parametrisation: every edge node
    at 0.4 of its edge, so T_u, T_v and |N| vary over each patch.  The surface
    is still the cube, so the discrete sum converges to the box's erf product
    (P1) as the rule is refined; the corner tangents keep the edges'
    directions, so the pseudonormals equal the flat cube's; and (1/3) sum
    nw . y is the cube's volume."""
    m = synth.cube(1.0, 4)
    q = synth.quadratic_from_flat(m, 0.4)
    s = 0.1
    x = synth.cube_c1(300)["targets"]
    ex = box_phi(x, 1.0, s)
    errs = []
    for n, sd in ((4, 1), (8, 1), (8, 2)):
        y, nw, sg = oracle_mod.sources_quad(q.verts, q.tris6, np.full(m.m, s), n, sd)
        phi, gr = oracle_mod.phi_grad(y, nw, sg, x)
        errs.append(np.abs(phi - ex).max())
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-11
    assert np.abs(gr - box_grad(x, 1.0, s)).max() < 1e-9
    assert abs((nw * y).sum() / 3.0 - 8.0) < 1e-13
    geo = oracle_mod.geometry(m.verts, m.tris, None)
    gq = oracle_mod.geometry_quad(q.verts, q.tris6, None, 4, 0)
    assert np.abs(gq["vpn"][:m.nv] - geo["vpn"]).max() < 1e-14


def test_quadratic_sphere_converges_faster_than_flat(oracle_mod):
    """Quadratic patches with every node on the unit sphere: the enclosed
    volume (1/3) sum nw . y and the constant-sigma sum at points near the
    surface (against the ball's closed form, P4) converge at a higher order in
    the edge length than the flat icosphere's (second order)."""
    s = 0.15
    rr = np.array([0.8, 0.95, 1.0, 1.05])
    x = np.stack([rr / math.sqrt(3)] * 3, axis=1)
    vq, vf, bq, bf = [], [], [], []
    for level in (1, 2, 3):
        q = synth.quadratic_icosphere(level)
        y, nw, sg = oracle_mod.sources_quad(q.verts, q.tris6, np.full(q.m, s), 6, 0)
        vq.append(abs((nw * y).sum() / 3.0 - 4.0 * math.pi / 3.0))
        bq.append(np.abs(oracle_mod.phi_grad(y, nw, sg, x)[0] - _ball_phi(rr, 1.0, s)).max())
        f = synth.icosphere(level)
        y, nw, sg = oracle_mod.sources(f.verts, f.tris, np.full(f.m, s), 6, 0)
        vf.append(abs((nw * y).sum() / 3.0 - 4.0 * math.pi / 3.0))
        bf.append(np.abs(oracle_mod.phi_grad(y, nw, sg, x)[0] - _ball_phi(rr, 1.0, s)).max())
    for e in (vf, bf):   # flat: second order
        assert 3.0 < e[0] / e[1] < 5.0 and 3.0 < e[1] / e[2] < 5.0
    for e in (vq, bq):   # quadratic: at least third order, and far smaller
        assert e[0] / e[1] > 7.0 and e[1] / e[2] > 7.0
    assert vq[2] < 0.05 * vf[2] and bq[2] < 0.05 * bf[2]


def _quad_solve_at(oracle_mod, q, src, tri, uv, tol=1e-14):
    x0, hd, sl = oracle_mod.chart_nodes_quad_at(q.verts, q.tris6, tri, uv)
    r = oracle_mod.solve_charts(*src, x0, hd, sl, tol=tol, max_iter=40)
    assert (r["status"] == 0).all()
    return r


def test_quadratic_chart_frames_match_finite_differences(oracle_mod):
    """eq. u_vector / U_vector_2 on a curved patch (T_u, T_v vary with u, v):
    x_u, x_v equal central differences of the solved chart x(u, v)."""
    q = synth.quadratic_icosphere(1)
    src = oracle_mod.sources_quad(q.verts, q.tris6, None, 4, 0)
    d = 1e-4
    for j, u, v in ((3, 0.2, 0.3), (41, 0.55, 0.1), (77, 0.1, 0.7)):
        tri = np.array([j] * 5, dtype=np.int32)
        uv = np.array([[u, v], [u + d, v], [u - d, v], [u, v + d], [u, v - d]])
        r = _quad_solve_at(oracle_mod, q, src, tri, uv)
        _, g = oracle_mod.phi_grad(*src, r["x"][:1])
        xu, xv, jac = oracle_mod.chart_frames_quad_at(q.verts, q.tris6, tri[:1], uv[:1], r["h"][:1], g)
        fu = (r["x"][1] - r["x"][2]) / (2 * d)
        fv = (r["x"][3] - r["x"][4]) / (2 * d)
        scale = np.linalg.norm(fu) + np.linalg.norm(fv)
        assert np.abs(xu[0] - fu).max() < 1e-7 * scale
        assert np.abs(xv[0] - fv).max() < 1e-7 * scale
        assert abs(jac[0] - np.linalg.norm(np.cross(fu, fv))) < 1e-7 * scale ** 2


def test_quadratic_charts_close_and_flux_converges(oracle_mod):
    """Charts on quadratic patches: the node at an edge's midpoint solved from
    either neighbouring patch is the same point (T and the linear H agree on
    the shared curved edge), and the Gauss flux error eps0 falls with the
    chart order."""
    q = synth.quadratic_icosphere(1)
    src = oracle_mod.sources_quad(q.verts, q.tris6, None, 4, 0)
    T = q.tris6
    j = 5
    a, b = T[j][0], T[j][1]
    k = next(i for i in range(q.m) if i != j and a in T[i][:3] and b in T[i][:3])

    def uv_of(i, p, r):
        loc = [list(T[i][:3]).index(p), list(T[i][:3]).index(r)]
        bary = np.zeros(3)
        bary[loc] = 0.5
        return np.array([[bary[1], bary[2]]])

    xs = [_quad_solve_at(oracle_mod, q, src, np.array([i], dtype=np.int32), uv_of(i, a, b), 1e-15)["x"][0]
          for i in (j, k)]
    assert np.abs(xs[0] - xs[1]).max() < 1e-13
    out = []
    for n in (3, 5, 7):
        tri, uv, w = oracle_mod.refined_nodes(q.m, n, np.zeros(q.m))
        r = _quad_solve_at(oracle_mod, q, src, tri, uv)
        _, g = oracle_mod.phi_grad(*src, r["x"])
        _, _, jac = oracle_mod.chart_frames_quad_at(q.verts, q.tris6, tri, uv, r["h"], g)
        out.append(abs(oracle_mod.gauss_flux_w(r["x"], g, jac, w, (0.05, -0.1, 0.02))))
    assert out[0] > 100 * out[1] and out[1] > 100 * out[2]
    assert out[2] < 1e-10
