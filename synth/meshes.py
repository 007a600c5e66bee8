"""Mesh and target generators (input construction only; see package doc)."""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def rng(seed: int) -> np.random.Generator:
    """Philox counter-based generator for a workload seed."""
    return np.random.Generator(np.random.Philox(key=int(seed)))


@dataclass
class Mesh:
    """A closed triangulated surface, counter-clockwise seen from outside.

    verts: float64 [nv, 3]; tris: int32 [m, 3]; sigma: float64 [m] (the
    per-triangle smoothing width the workload asks for, or None)."""

    verts: np.ndarray
    tris: np.ndarray
    sigma: np.ndarray | None = None
    name: str = ""

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def m(self) -> int:
        return int(self.tris.shape[0])


def _areas(verts, tris):
    p1, p2, p3 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    return 0.5 * np.linalg.norm(np.cross(p2 - p1, p3 - p1), axis=1)


def sigma_half_sqrt2area(verts, tris) -> np.ndarray:
    """The workloads' sigma rule: sigma_j = 0.5 * sqrt(2 * area_j)."""
    return 0.5 * np.sqrt(2.0 * _areas(verts, tris))


def _grid_tris(idx: np.ndarray) -> np.ndarray:
    """Two triangles per cell of a vertex-index grid idx[i, j]; cell corners
    (i,j),(i+1,j),(i+1,j+1),(i,j+1) are counter-clockwise in the (i, j) plane."""
    a = idx[:-1, :-1].ravel()
    b = idx[1:, :-1].ravel()
    c = idx[1:, 1:].ravel()
    d = idx[:-1, 1:].ravel()
    t1 = np.stack([a, b, c], axis=1)
    t2 = np.stack([a, c, d], axis=1)
    return np.stack([t1, t2], axis=1).reshape(-1, 3).astype(np.int32)


def cube(a: float = 1.0, k: int = 4) -> Mesh:
    """Axis-aligned cube [-a, a]^3, each face a k x k grid of squares with two
    triangles each (12 k^2 triangles), conforming and watertight."""
    lut = {}
    verts = []

    def vid(p):
        key = tuple(int(c) for c in p)
        if key not in lut:
            lut[key] = len(verts)
            verts.append(key)
        return lut[key]

    tris = []
    for d in range(3):
        for s in (-1, 1):
            d1, d2 = (d + 1) % 3, (d + 2) % 3
            if s < 0:
                d1, d2 = d2, d1
            idx = np.empty((k + 1, k + 1), dtype=np.int64)
            for i in range(k + 1):
                for j in range(k + 1):
                    p = [0, 0, 0]
                    p[d] = k if s > 0 else 0
                    p[d1] = i
                    p[d2] = j
                    idx[i, j] = vid(p)
            tris.append(_grid_tris(idx))
    v = np.asarray(verts, dtype=np.float64) * (2.0 * a / k) - a
    return Mesh(v, np.concatenate(tris).astype(np.int32), None, f"cube_k{k}")


def _shortest_incident_edge(verts, tris):
    e = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    ln = np.linalg.norm(verts[e[:, 0]] - verts[e[:, 1]], axis=1)
    out = np.full(len(verts), np.inf)
    np.minimum.at(out, e[:, 0], ln)
    np.minimum.at(out, e[:, 1], ln)
    return out


def _jitter(verts, tris, frac, g: np.random.Generator):
    if frac <= 0:
        return verts
    le = _shortest_incident_edge(verts, tris)
    d = g.uniform(-1.0, 1.0, size=verts.shape) * (frac * le)[:, None]
    return verts + d


def torus(R: float = 1.0, r: float = 0.3, nu: int = 240, nv: int = 64, grading: float = 20.0,
          jitter: float = 0.05, seed: int = 2) -> Mesh:
    """Torus of radii (R, r) from a (u, v) grid of nu x nv cells (2 nu nv
    triangles).  The u-spacing follows a symmetric geometric ramp: it grows by
    a constant ratio over the first nu/2 cells up to `grading` times the
    smallest cell, then mirrors back, so the periodic seam has no jump.
    Vertices are jittered by a uniform vector in [-1,1]^3 times `jitter` times
    the shortest incident edge."""
    g = rng(seed)
    half = nu // 2
    q = grading ** (1.0 / max(half - 1, 1))
    sp = q ** np.arange(half)
    sp = np.concatenate([sp, sp[::-1]])[:nu]
    if len(sp) < nu:
        sp = np.concatenate([sp, sp[-1:]])
    uu = np.concatenate([[0.0], np.cumsum(sp)])[:-1] / sp.sum() * 2.0 * np.pi
    vv = np.arange(nv) / nv * 2.0 * np.pi
    U, V = np.meshgrid(uu, vv, indexing="ij")
    A = R + r * np.cos(V)
    P = np.stack([A * np.cos(U), A * np.sin(U), r * np.sin(V)], axis=-1).reshape(-1, 3)
    idx = np.arange(nu * nv).reshape(nu, nv)
    idx = np.concatenate([idx, idx[:1]], axis=0)
    idx = np.concatenate([idx, idx[:, :1]], axis=1)
    tris = _grid_tris(idx)
    P = _jitter(P, tris, jitter, g)
    return Mesh(P, tris, sigma_half_sqrt2area(P, tris), f"torus_{nu}x{nv}")


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v, f


def icosphere(level: int) -> Mesh:
    """Unit icosphere: icosahedron split `level` times into four midpoint
    children, new vertices projected to the sphere (20 * 4^level triangles)."""
    v, f = _icosahedron()
    for _ in range(level):
        nv = len(v)
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        key = np.minimum(e[:, 0], e[:, 1]) * (nv + 1) + np.maximum(e[:, 0], e[:, 1])
        uk, inv = np.unique(key, return_inverse=True)
        a = uk // (nv + 1)
        b = uk % (nv + 1)
        mid = v[a] + v[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        v = np.concatenate([v, mid])
        m = len(f)
        ab = nv + inv[:m]
        bc = nv + inv[m:2 * m]
        ca = nv + inv[2 * m:]
        f = np.concatenate([
            np.stack([f[:, 0], ab, ca], 1),
            np.stack([ab, f[:, 1], bc], 1),
            np.stack([ca, bc, f[:, 2]], 1),
            np.stack([ab, bc, ca], 1),
        ])
    return Mesh(v, f.astype(np.int32), None, f"icosphere_l{level}")


def bumped_icosphere(level: int = 8, nbumps: int = 200, seed: int = 3) -> Mesh:
    """Icosphere displaced radially by Gaussian bumps: r(p) = 1 + sum_k h_k
    exp(-|p - c_k|^2 / (2 w_k^2)) with centres c_k uniform on the sphere,
    widths log-uniform in [0.005, 0.2] and heights uniform in [-0.1, 0.1]."""
    g = rng(seed)
    base = icosphere(level)
    c = g.normal(size=(nbumps, 3))
    c /= np.linalg.norm(c, axis=1, keepdims=True)
    w = np.exp(g.uniform(np.log(0.005), np.log(0.2), size=nbumps))
    h = g.uniform(-0.1, 0.1, size=nbumps)
    p = base.verts
    rad = np.ones(len(p))
    for k0 in range(0, nbumps, 16):
        d2 = ((p[:, None, :] - c[None, k0:k0 + 16, :]) ** 2).sum(-1)
        rad += (h[None, k0:k0 + 16] * np.exp(-d2 / (2.0 * w[None, k0:k0 + 16] ** 2))).sum(1)
    P = p * rad[:, None]
    return Mesh(P, base.tris, sigma_half_sqrt2area(P, base.tris), f"bumped_icosphere_l{level}")


def _latlong_sphere(T: int):
    nl1 = max(2, int(round((T / 4.0) ** 0.5)))          # rings = n_lat - 1
    nlon = max(3, int(round(T / (2.0 * nl1))))
    th = np.pi * np.arange(1, nl1 + 1) / (nl1 + 1)
    ph = 2.0 * np.pi * np.arange(nlon) / nlon
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    ring = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1).reshape(-1, 3)
    v = np.concatenate([[[0.0, 0.0, 1.0]], ring, [[0.0, 0.0, -1.0]]])
    N, S = 0, len(v) - 1
    idx = 1 + np.arange(nl1 * nlon).reshape(nl1, nlon)
    idx = np.concatenate([idx, idx[:, :1]], axis=1)
    mid = _grid_tris(idx)
    j = np.arange(nlon)
    top = np.stack([np.full(nlon, N), idx[0, j], idx[0, j + 1]], 1)
    bot = np.stack([idx[-1, j], np.full(nlon, S), idx[-1, j + 1]], 1)
    return v, np.concatenate([top, mid, bot]).astype(np.int32)


def _random_rotation(g: np.random.Generator):
    q = g.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def ellipsoid(T: int, g: np.random.Generator, jitter: float = 0.05, center=None) -> Mesh:
    """Latitude-longitude sphere with about T triangles (T = 2 n_lon (n_lat-1)),
    scaled by axes uniform in [0.5, 2], rotated by a uniform random rotation
    and jittered like the torus."""
    v, f = _latlong_sphere(T)
    ax = g.uniform(0.5, 2.0, size=3)
    Rm = _random_rotation(g)
    v = (v * ax[None, :]) @ Rm.T
    v = _jitter(v, f, jitter, g)
    if center is not None:
        v = v + np.asarray(center)[None, :]
    return Mesh(v, f, sigma_half_sqrt2area(v, f), f"ellipsoid_T{len(f)}")


def targets_uniform(n: int, lo: float, hi: float, g: np.random.Generator) -> np.ndarray:
    """n points uniform in the cube [lo, hi]^3."""
    return g.uniform(lo, hi, size=(n, 3))


def targets_near_surface(mesh: Mesh, n: int, g: np.random.Generator, width: float = 3.0,
                         sigma=None) -> np.ndarray:
    """n points within `width` sigma of the surface: a triangle chosen
    uniformly by index, a uniform point in it, and an offset along its unit
    normal uniform in [-width sigma_j, width sigma_j]."""
    sig = mesh.sigma if sigma is None else np.asarray(sigma)
    j = g.integers(0, mesh.m, size=n)
    r1 = g.uniform(size=n)
    r2 = g.uniform(size=n)
    s = np.sqrt(r1)
    b1, b2 = s * (1.0 - r2), s * r2
    p1 = mesh.verts[mesh.tris[j, 0]]
    p2 = mesh.verts[mesh.tris[j, 1]]
    p3 = mesh.verts[mesh.tris[j, 2]]
    nn = np.cross(p2 - p1, p3 - p1)
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    off = g.uniform(-width, width, size=n) * sig[j]
    return p1 + b1[:, None] * (p2 - p1) + b2[:, None] * (p3 - p1) + off[:, None] * nn


# ---------------------------------------------------------------- quadratic patches
@dataclass
class QuadMesh:
    """A closed surface of 6-node quadratic (curvilinear) triangles.

    verts: float64 [nv, 3]; tris6: int32 [m, 6], the corners P1, P2, P3
    (counter-clockwise seen from outside) then the nodes on the edges P1-P2,
    P2-P3, P3-P1; neighbouring patches share an edge's node.  sigma: float64
    [m] or None."""

    verts: np.ndarray
    tris6: np.ndarray
    sigma: np.ndarray | None = None
    name: str = ""

    @property
    def nv(self) -> int:
        return int(self.verts.shape[0])

    @property
    def m(self) -> int:
        return int(self.tris6.shape[0])


def quadratic_from_flat(mesh: Mesh, t: float = 0.5, project=None, name: str = "") -> QuadMesh:
    """Quadratic patches on a flat mesh's triangles: one node per edge at
    P_a + t (P_b - P_a), a < b the edge's vertex indices (so both patches on
    an edge share the node), optionally mapped by `project` (for instance onto
    the surface the flat mesh approximates).  t = 0.5 without projection gives
    the flat mesh itself; t != 0.5 keeps every patch flat but parametrised
    non-affinely (valid for 1/4 < t < 3/4)."""
    v, f = mesh.verts, mesh.tris
    nv = len(v)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    key = lo.astype(np.int64) * (nv + 1) + hi
    uk, inv = np.unique(key, return_inverse=True)
    a, b = uk // (nv + 1), uk % (nv + 1)
    mid = v[a] + t * (v[b] - v[a])
    if project is not None:
        mid = project(mid)
    m = len(f)
    t6 = np.stack([f[:, 0], f[:, 1], f[:, 2], nv + inv[:m], nv + inv[m:2 * m], nv + inv[2 * m:]], 1)
    return QuadMesh(np.concatenate([v, mid]), t6.astype(np.int32), None, name or f"quadratic_{mesh.name}")


def quadratic_icosphere(level: int) -> QuadMesh:
    """Unit sphere from quadratic patches: the icosphere's triangles with
    their edge nodes at the normalised edge midpoints (every node on the
    sphere)."""
    return quadratic_from_flat(icosphere(level), 0.5, lambda p: p / np.linalg.norm(p, axis=1, keepdims=True),
                               f"quadratic_icosphere_l{level}")


def quadratic_torus(R: float = 1.0, r: float = 0.3, nu: int = 24, nv: int = 8) -> QuadMesh:
    """Torus of radii (R, r) from quadratic patches: a uniform (u, v) grid of
    nu x nv cells split into triangles, every node (corners and the edge
    nodes at the parameter midpoints) on the exact torus."""
    def on_torus(U, V):
        A = R + r * np.cos(V)
        return np.stack([A * np.cos(U), A * np.sin(U), r * np.sin(V)], axis=-1)

    uu = np.arange(nu) / nu * 2.0 * np.pi
    vv = np.arange(nv) / nv * 2.0 * np.pi
    U, V = np.meshgrid(uu, vv, indexing="ij")
    P = on_torus(U, V).reshape(-1, 3)
    idx = np.arange(nu * nv).reshape(nu, nv)
    idx = np.concatenate([idx, idx[:1]], axis=0)
    idx = np.concatenate([idx, idx[:, :1]], axis=1)
    f = _grid_tris(idx)
    # parameter coordinates of every corner (unwrapped per triangle) give the
    # edge nodes' parameter midpoints
    iu, iv = np.divmod(np.arange(nu * nv), nv)
    fu, fv = iu[f].astype(np.float64), iv[f].astype(np.float64)
    for c in range(1, 3):   # unwrap the periodic seams relative to the first corner
        fu[:, c] += np.where(fu[:, c] - fu[:, 0] < -nu / 2, nu, 0) - np.where(fu[:, c] - fu[:, 0] > nu / 2, nu, 0)
        fv[:, c] += np.where(fv[:, c] - fv[:, 0] < -nv / 2, nv, 0) - np.where(fv[:, c] - fv[:, 0] > nv / 2, nv, 0)
    nvert = len(P)
    e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
    eu = np.concatenate([fu[:, [0, 1]], fu[:, [1, 2]], fu[:, [2, 0]]]).mean(1)
    ev = np.concatenate([fv[:, [0, 1]], fv[:, [1, 2]], fv[:, [2, 0]]]).mean(1)
    lo, hi = np.minimum(e[:, 0], e[:, 1]), np.maximum(e[:, 0], e[:, 1])
    key = lo.astype(np.int64) * (nvert + 1) + hi
    uk, first, inv = np.unique(key, return_index=True, return_inverse=True)
    mid = on_torus(eu[first] / nu * 2.0 * np.pi, ev[first] / nv * 2.0 * np.pi)
    m = len(f)
    t6 = np.stack([f[:, 0], f[:, 1], f[:, 2], nvert + inv[:m], nvert + inv[m:2 * m], nvert + inv[2 * m:]], 1)
    return QuadMesh(np.concatenate([P, mid]), t6.astype(np.int32), None, f"quadratic_torus_{nu}x{nv}")
