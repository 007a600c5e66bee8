"""The five named workloads, each from its own seed (inputs only)."""
from __future__ import annotations

import numpy as np

from .meshes import (Mesh, bumped_icosphere, cube, ellipsoid, rng, targets_near_surface,
                     targets_uniform, torus)


def cube_c1(n_targets: int = 10_000, seed: int = 1):
    """Cube [-1,1]^3, 4 x 4 squares per face, 2 triangles each (192), constant
    sigma = 0.1; targets uniform in [-1.5, 1.5]^3.  Source rule: Duffy 4 x 4
    on each of the 4 midpoint children of every triangle (12,288 nodes)."""
    m = cube(1.0, 4)
    m.sigma = np.full(m.m, 0.1)
    g = rng(seed)
    x = targets_uniform(n_targets, -1.5, 1.5, g)
    return dict(mesh=m, targets=x, rule=dict(n=4, subdiv=1), name="cube_192tri_sigma0.1")


def torus_c2(n_targets: int = 1_000_000, seed: int = 2, nu: int = 240, nv: int = 64):
    """Graded torus R=1, r=0.3, 240 x 64 cells (30,720 triangles), u-grading
    20, 5% jitter, sigma_j = 0.5 sqrt(2 area_j); targets within 3 sigma of the
    surface.  Source rule Duffy 6 x 6 (1,105,920 nodes); chart order 8 uses the
    6 x 6 chart rule."""
    m = torus(1.0, 0.3, nu, nv, 20.0, 0.05, seed)
    g = rng(seed + 1000)
    x = targets_near_surface(m, n_targets, g, 3.0)
    return dict(mesh=m, targets=x, rule=dict(n=6, subdiv=0), chart_n=6,
                name=f"graded_torus_{2 * nu * nv}tri")


def icosphere_c3(level: int = 8, n_targets: int = 20_000_000, seed: int = 3):
    """Icosphere level 8 (1,310,720 triangles) with 200 Gaussian bumps;
    sigma by the same rule; Duffy 4 x 4 sources (about 2.1e7 nodes); targets
    within 3 sigma."""
    m = bumped_icosphere(level, 200, seed)
    g = rng(seed + 1000)
    x = targets_near_surface(m, n_targets, g, 3.0)
    return dict(mesh=m, targets=x, rule=dict(n=4, subdiv=0), name=f"bumped_icosphere_l{level}")


def ellipsoid_batch_c4(nmesh: int = 512, seed: int = 4, tmin: int = 200, tmax: int = 5000):
    """nmesh ellipsoids, triangle counts log-uniform in [tmin, tmax]; sources
    Duffy 4 x 4; chart order 6 (5 x 5 rule)."""
    g = rng(seed)
    meshes = []
    for _ in range(nmesh):
        T = int(round(np.exp(g.uniform(np.log(tmin), np.log(tmax)))))
        meshes.append(ellipsoid(T, g))
    return dict(meshes=meshes, rule=dict(n=4, subdiv=0), chart_n=5, name=f"ellipsoids_{nmesh}")


def serve_stream_c5(nreq: int = 2000, rate: float = 50.0, seed: int = 5, tmin: float = 1e3,
                    tmax: float = 5e5):
    """Poisson arrivals (mean rate `rate` per second); each request names a
    generator (ellipsoid, graded torus, bumped icosphere) and a triangle count
    log-uniform in [tmin, tmax].  Returns request descriptors; meshes are built
    on demand by make_request_mesh."""
    g = rng(seed)
    t = np.cumsum(g.exponential(1.0 / rate, size=nreq))
    kind = g.integers(0, 3, size=nreq)
    T = np.exp(g.uniform(np.log(tmin), np.log(tmax), size=nreq)).astype(np.int64)
    sub = g.integers(0, 2 ** 31, size=nreq)
    return [dict(arrival=float(t[i]), kind=int(kind[i]), T=int(T[i]), seed=int(sub[i]))
            for i in range(nreq)]


def make_request_mesh(req) -> Mesh:
    """The mesh of one serving request (nearest available size per generator)."""
    g = rng(req["seed"])
    T = req["T"]
    if req["kind"] == 0:
        return ellipsoid(T, g)
    if req["kind"] == 1:
        nv = max(8, int(round((T / 2.0 / 3.75) ** 0.5)))
        nu = max(8, 2 * int(round(T / (2.0 * nv) / 2.0)))
        return torus(1.0, 0.3, nu, nv, 20.0, 0.05, req["seed"])
    level = int(np.clip(round(np.log(max(T, 20) / 20.0) / np.log(4.0)), 1, 7))
    return bumped_icosphere(level, 200, req["seed"])
