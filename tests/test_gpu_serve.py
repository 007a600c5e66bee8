"""Serving: requests admitted as slots and HBM budget free up run concurrently
on separate streams; each result equals the same request solved alone, a
failing request reports its error without affecting the others, and a tight
budget serialises admission without changing results."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1909_13356_gb300 as lsm
    ctx = lsm.Context(0)
    g = synth.rng(55)
    ms = [synth.ellipsoid(int(T), g) for T in (300, 900, 500, 1500, 240, 700)]
    ms.append(synth.torus(1.0, 0.3, 40, 12, 20.0, 0.05, seed=56))
    alone = []
    for m in ms:
        mesh = ctx.upload(m.verts, m.tris, m.sigma, n_gl=4)
        alone.append(mesh.solve_charts(order=8, tol=1e-10, precision=lsm.MIXED))
        mesh.free()
    return lsm, ctx, ms, alone


def _check(res, ref):
    x, h, st, stats = ref
    assert res["status"] == 0
    assert np.all(res["node_status"] & 255 == 0)
    assert np.abs(res["x"] - x).max() < 1e-9


def test_served_results_equal_alone(setup):
    lsm, ctx, ms, alone = setup
    srv = lsm.Server(ctx, slots=3)
    tickets = [srv.submit(m.verts, m.tris, m.sigma, n_gl=4, order=8, tol=1e-10) for m in ms]
    results = [srv.result(t) for t in tickets]
    info = srv.info()
    srv.close()
    for r, ref in zip(results, alone):
        _check(r, ref)
    assert info["max_running"] >= 2          # requests overlapped
    assert all(r["t_done_ms"] >= r["t_start_ms"] >= r["t_submit_ms"] for r in results)


def test_tight_budget_serialises_admission(setup):
    lsm, ctx, ms, alone = setup
    srv = lsm.Server(ctx, slots=4, hbm_budget_bytes=1)   # every request is larger than the budget
    tickets = [srv.submit(m.verts, m.tris, m.sigma, n_gl=4, order=8, tol=1e-10) for m in ms[:4]]
    results = [srv.result(t) for t in tickets]
    info = srv.info()
    srv.close()
    assert info["max_running"] == 1
    for r, ref in zip(results, alone[:4]):
        _check(r, ref)


def test_failing_request_is_isolated(setup):
    lsm, ctx, ms, alone = setup
    srv = lsm.Server(ctx, slots=2)
    bad = synth.cube(1.0, 2)
    t_ok = srv.submit(ms[0].verts, ms[0].tris, ms[0].sigma, n_gl=4, order=8, tol=1e-10)
    t_bad = srv.submit(bad.verts, bad.tris[:-1], None, order=8)     # open mesh
    t_ok2 = srv.submit(ms[2].verts, ms[2].tris, ms[2].sigma, n_gl=4, order=8, tol=1e-10)
    r_bad = srv.result(t_bad)
    assert r_bad["status"] == -4
    assert "edge" in r_bad["error"] or "closed" in r_bad["error"] or "mesh" in r_bad["error"], r_bad["error"]
    for t, ref in ((t_ok, alone[0]), (t_ok2, alone[2])):
        r = srv.result(t)
        _check(r, ref)
        assert r["error"] == ""
    srv.close()


def test_failing_requests_keep_their_own_messages(setup):
    """Two kinds of failure running next to good requests on several slots:
    each failed request reports its own message, the good ones none."""
    lsm, ctx, ms, alone = setup
    srv = lsm.Server(ctx, slots=3)
    bad = synth.cube(1.0, 2)
    flipped = bad.tris[:, ::-1].copy()        # inward orientation: negative volume
    tickets = []
    for k in range(3):
        tickets.append(("ok", k, srv.submit(ms[k].verts, ms[k].tris, ms[k].sigma, n_gl=4, order=8, tol=1e-10)))
        tickets.append(("open", k, srv.submit(bad.verts, bad.tris[:-1], None, order=8)))
        tickets.append(("flip", k, srv.submit(bad.verts, flipped, None, order=8)))
    msgs = {}
    for kind, k, t in tickets:
        r = srv.result(t)
        if kind == "ok":
            _check(r, alone[k])
            assert r["error"] == ""
        else:
            assert r["status"] == -4 and r["error"]
            msgs.setdefault(kind, set()).add(r["error"])
    srv.close()
    # every request of a kind got that kind's message, and the kinds differ
    assert len(msgs["open"]) == 1 and len(msgs["flip"]) == 1
    assert msgs["open"] != msgs["flip"]


def test_cancel_takes_queued_requests_off_the_queue(setup):
    """With one slot the later requests wait in the queue; cancelling them
    finalises them as cancelled, the others still run, and a request that has
    already finished cannot be cancelled."""
    lsm, ctx, ms, alone = setup
    srv = lsm.Server(ctx, slots=1)
    tickets = [srv.submit(m.verts, m.tris, m.sigma, n_gl=4, order=8, tol=1e-10) for m in ms[:4]]
    cancelled = [t for t in tickets[2:] if srv.cancel(t)]
    assert cancelled, "the last requests should still have been queued"
    for k, t in enumerate(tickets):
        r = srv.result(t, release=False)
        if t in cancelled:
            assert r["status"] == -7 and "cancel" in r["error"]
        else:
            _check(r, alone[k])
            assert not srv.cancel(t)
    srv.close()
