"""The serving loop (nf_server): continuous batching over concurrent slots.

Each episode's result must be the same alone and in the mix: the forward
(loss, solver iterations) bitwise, since its kernels are deterministic
whatever else runs on the device; the gradient to rounding (the advection
adjoint scatters with float atomics, whose order varies from run to run even
alone). Results must also match the direct episode API; admission must
respect the HBM budget; bad requests fail alone.
"""

import numpy as np
import pytest

import nf_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG = dict(precision="mixed", tol=1e-8, max_iters=2000, cfl_max=8.0, checkpoint_every=2)


def _episodes():
    out = []
    for key, (kind, n) in enumerate([("sphere", 16), ("chamber", 16), ("plate", 16),
                                     ("sphere", 24), ("chamber", 24), ("plate", 20)]):
        if kind == "sphere":
            cfg = I.config_sphere(n)
            cfg["scene"] = dict(cfg["scene"], theta=[0.1 + 0.01 * key, 0.02, -0.01])
            loss = "kinetic_energy"
        elif kind == "chamber":
            cfg = I.config_chamber(n, seed=key, duct_half_cells=2)
            loss = "outflow"
        else:
            cfg = I.config_plate(n, seed=key)
            loss = "kinetic_energy"
        out.append(dict(key=100 + key, grid=cfg["grid"], scene=cfg["scene"], loss=loss))
    return out


def _script(srv, ep):
    """OPEN, 2 frames, 1 frame + adjoint, CLOSE: the tickets in order."""
    return [srv.open(ep["key"], ep["grid"], ep["scene"]),
            srv.step(ep["key"], frames=2),
            srv.step(ep["key"], frames=1, adjoint=True, loss=ep["loss"]),
            srv.close(ep["key"])]


def _collect(srv, tickets):
    return [srv.poll(t, wait_ms=120000) for t in tickets]


def test_each_result_is_the_same_alone_and_in_the_mix(nf):
    eps = _episodes()
    # alone: one slot, one episode at a time
    srv = nf.Server(slots=1, **CFG)
    alone = {}
    for ep in eps:
        res = _collect(srv, _script(srv, ep))
        assert all(r is not None and r["status"] == 0 for r in res), res
        alone[ep["key"]] = res[2]
    srv.close_server()
    # mix: three slots, every request submitted up front, interleaved
    srv = nf.Server(slots=3, **CFG)
    scripts = {ep["key"]: [] for ep in eps}
    for ep in eps:
        scripts[ep["key"]].append(srv.open(ep["key"], ep["grid"], ep["scene"]))
    for ep in eps:
        scripts[ep["key"]].append(srv.step(ep["key"], frames=2))
    for ep in eps:
        scripts[ep["key"]].append(srv.step(ep["key"], frames=1, adjoint=True, loss=ep["loss"]))
    for ep in eps:
        scripts[ep["key"]].append(srv.close(ep["key"]))
    assert srv.drain(wait_ms=300000)
    stats = srv.stats()
    mixed = {k: _collect(srv, t) for k, t in scripts.items()}
    srv.close_server()
    assert stats["completed"] == stats["submitted"] == 4 * len(eps)
    overlap = False
    for ep in eps:
        res = mixed[ep["key"]]
        assert all(r["status"] == 0 for r in res), res
        a, m = alone[ep["key"]], res[2]
        assert m["loss"] == a["loss"]
        assert m["fwd"]["iters"] == a["fwd"]["iters"]
        g_a = np.asarray(a["g_theta"])
        assert np.linalg.norm(m["g_theta"] - g_a) <= 1e-6 * np.linalg.norm(g_a)
    # requests of different episodes were on the device at the same time
    spans = sorted((r["start_ms"], r["end_ms"]) for res in mixed.values() for r in res)
    for (s0, e0), (s1, e1) in zip(spans, spans[1:]):
        overlap |= s1 < e0
    assert overlap


def test_served_result_matches_the_direct_api(nf):
    ep = _episodes()[1]                       # chamber 16^3
    srv = nf.Server(slots=2, **CFG)
    res = _collect(srv, _script(srv, ep))
    srv.close_server()
    ctx = nf.Context(**CFG)
    e = ctx.episode(ep["grid"], ep["scene"])
    e.step(3)
    J, gU = e.loss(ep["loss"], want_grad=True)
    gth, _, _ = e.backward(gU, want_gU0=False)
    e.close()
    ctx.close()
    K = len(ep["scene"]["theta"])
    assert res[2]["loss"] == J
    assert np.linalg.norm(res[2]["g_theta"][:K] - gth) <= 1e-6 * np.linalg.norm(gth)


def test_admission_waits_for_memory_and_respects_the_budget(nf):
    eps = _episodes()[3:]                     # 24^3, 24^3, 20^3 episodes
    probe = nf.Server(slots=1, **CFG)
    t = probe.open(1, eps[0]["grid"], eps[0]["scene"])
    probe.poll(t)
    budget = int(probe.stats()["bytes_reserved"] * 1.5)   # room for one episode
    probe.close_server()
    srv = nf.Server(slots=3, hbm_budget=budget, **CFG)
    scripts = [_script(srv, ep) for ep in eps]
    waiting_seen = srv.stats()["open_waiting"]
    assert srv.drain(wait_ms=300000)
    st = srv.stats()
    results = [_collect(srv, s) for s in scripts]
    srv.close_server()
    assert waiting_seen >= 1
    assert st["bytes_peak"] <= budget
    assert all(r["status"] == 0 for res in results for r in res)
    # one episode at a time: each OPEN starts after the previous CLOSE ended
    for prev, nxt in zip(results, results[1:]):
        assert nxt[0]["start_ms"] >= prev[3]["end_ms"] - 1e-6


def test_bad_requests_fail_alone(nf):
    ep = _episodes()[0]
    srv = nf.Server(slots=2, hbm_budget=1 << 20, **CFG)   # 1 MiB: no episode fits
    t_big = srv.open(1, ep["grid"], ep["scene"])
    t_unknown = srv.step(999, frames=1)
    r_big = srv.poll(t_big)
    r_unknown = srv.poll(t_unknown)
    srv.close_server()
    assert r_big["status"] == 2          # NF_E_OOM: larger than the whole budget
    assert r_unknown["status"] == 1      # NF_E_INVALID: no such episode
    srv = nf.Server(slots=2, **CFG)
    t1 = srv.open(7, ep["grid"], ep["scene"])
    t2 = srv.open(7, ep["grid"], ep["scene"])      # duplicate key
    t3 = srv.step(7, frames=1)
    t4 = srv.close(7)
    res = _collect(srv, [t1, t2, t3, t4])
    srv.close_server()
    assert [r["status"] for r in res] == [0, 1, 0, 0]
