"""The seeded input generators: sizes the workloads name, closed and
consistently oriented surfaces, determinism per seed."""
import numpy as np
import pytest

import synth
from synth.workloads import make_request_mesh


def _closed_and_oriented(m):
    t = m.tris.astype(np.int64)
    e = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    k = e[:, 0] * (m.nv + 1) + e[:, 1]
    kr = e[:, 1] * (m.nv + 1) + e[:, 0]
    return len(np.unique(k)) == len(k) and bool(np.all(np.isin(kr, k)))


def _signed_volume(m):
    v, t = m.verts, m.tris
    return np.einsum("ij,ij->i", v[t[:, 0]], np.cross(v[t[:, 1]], v[t[:, 2]])).sum() / 6.0


def test_cube_c1_sizes():
    w = synth.cube_c1()
    assert w["mesh"].m == 192 and w["targets"].shape == (10_000, 3)
    assert abs(_signed_volume(w["mesh"]) - 8.0) < 1e-12
    assert _closed_and_oriented(w["mesh"])
    assert np.all(np.abs(w["targets"]) <= 1.5)


def test_torus_c2_structure():
    m = synth.torus()
    assert m.m == 30_720
    assert _closed_and_oriented(m)
    vol = _signed_volume(m)
    assert abs(vol - 2 * np.pi ** 2 * 1.0 * 0.09) < 0.01
    a = 2 * (m.sigma ** 2)
    assert a.max() / a.min() > 20  # graded by 20 in u, plus jitter


def test_icosphere_counts_and_bumps():
    for L in range(4):
        m = synth.icosphere(L)
        assert m.m == 20 * 4 ** L and _closed_and_oriented(m)
    b = synth.bumped_icosphere(3, 200, seed=3)
    assert _closed_and_oriented(b) and _signed_volume(b) > 0


@pytest.mark.parametrize("T", [200, 1000, 5000])
def test_ellipsoid(T):
    m = synth.ellipsoid(T, synth.rng(4))
    assert abs(m.m - T) / T < 0.05
    assert _closed_and_oriented(m) and _signed_volume(m) > 0


def test_near_surface_targets_within_width():
    m = synth.torus(1.0, 0.3, 24, 8, 5.0, 0.05, seed=1)
    x = synth.targets_near_surface(m, 500, synth.rng(3), 3.0)
    # the distance to the torus' core circle stays within r +- 3 sigma_max (+ jitter)
    d = np.hypot(np.hypot(x[:, 0], x[:, 1]) - 1.0, x[:, 2])
    assert np.all(np.abs(d - 0.3) < 3.2 * m.sigma.max() + 0.05)


def test_determinism_per_seed():
    a = synth.torus_c2(1000)
    b = synth.torus_c2(1000)
    assert np.array_equal(a["mesh"].verts, b["mesh"].verts)
    assert np.array_equal(a["targets"], b["targets"])
    c = synth.torus(seed=3)
    assert not np.array_equal(a["mesh"].verts, c.verts)


def test_serve_stream_requests():
    reqs = synth.serve_stream_c5(50)
    assert len(reqs) == 50 and all(r["arrival"] > 0 for r in reqs)
    assert np.all(np.diff([r["arrival"] for r in reqs]) > 0)
    for r in reqs[:6]:
        r = dict(r, T=min(r["T"], 3000))
        m = make_request_mesh(r)
        assert _closed_and_oriented(m) and _signed_volume(m) > 0
