"""The serving loop (nf_server): continuous batching over concurrent slots,
and batched steps of same-size episodes (nf_step_batch).

Each episode's result must be the same alone and in the mix. Without
cross-episode batching the forward (loss, solver iterations) is bitwise
equal, since its kernels are deterministic whatever else runs on the device,
and the gradient equal to rounding (the advection adjoint scatters with
float atomics, whose order varies from run to run even alone). With batching
(one stacked solve for several episodes) every member still meets the solver
tolerance, so its results agree with the solve alone within it. Results must
also match the direct episode API; admission must respect the HBM budget;
bad requests fail alone.
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
    # mix: three slots, every request submitted up front, interleaved (no
    # cross-episode batching here: with it the results agree to the solver
    # tolerance, tested below)
    srv = nf.Server(slots=3, batch=1, **CFG)
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


# ------------------------------------------------------ batched steps ----

def _batch_members(n=16):
    """Same-size episodes with different scenes and openings: a sphere and a
    plate in closed boxes, the chamber with its outlet (CFL substeps), an
    extruded polar-Bezier obstacle and a sphere between an inflow and an
    outflow patch."""
    sph = I.config_sphere(n)
    pla = I.config_plate(n, seed=3)
    cha = I.config_chamber(n, seed=5, duct_half_cells=2)
    g = I.make_grid(n, 0.01)
    ext = I.extruded_scene(4, shapes=1, segments=4, keys=1)
    gin = I.make_grid(n, 0.01, inlet=I.centred_inlet(n, 4, 0.3), outlet=I.centred_outlet(n, 4))
    return [(sph["grid"], sph["scene"], I.gaussian_faces(sph["grid"], 0.1, 1), "kinetic_energy"),
            (pla["grid"], pla["scene"], I.gaussian_faces(pla["grid"], 0.1, 2), "kinetic_energy"),
            (cha["grid"], cha["scene"], I.zero_faces(cha["grid"]), "outflow"),
            (g, ext, I.gaussian_faces(g, 0.1, 3), "kinetic_energy"),
            (gin, I.sphere_scene(v=(0.05, 0.0, 0.0)), I.gaussian_faces(gin, 0.1, 4),
             "kinetic_energy")]


def _start(nf, ctx, members):
    eps = []
    for grid, scene, u0, _ in members:
        e = ctx.episode(grid, scene)
        e.set_velocity([torch.tensor(x, device="cuda") for x in u0], project=True)
        eps.append(e)
    return eps


def _rel(a, b):
    a = np.concatenate([x.ravel() for x in a])
    b = np.concatenate([x.ravel() for x in b])
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol,vtol", [("fp64", 1e-12, 1e-9), ("mixed", 1e-10, 1e-6)])
def test_batched_steps_match_steps_alone(nf, prec, tol, vtol):
    members = _batch_members()
    cfg = dict(precision=prec, tol=tol, max_iters=3000, cfl_max=1.0, checkpoint_every=2)
    ctx_a = nf.Context(**cfg)
    alone = _start(nf, ctx_a, members)
    st_a = [e.step(3) for e in alone]
    ctx_b = nf.Context(**cfg)
    batch = _start(nf, ctx_b, members)
    st_b = ctx_b.step_batch(batch, frames=3)
    assert st_b[2]["steps"] > 3                   # the chamber took substeps
    for (grid, scene, _, loss), ea, eb, sa, sb in zip(members, alone, batch, st_a, st_b):
        assert sb["status"] == 0 and sb["steps"] == sa["steps"]
        assert sb["rel_residual"] <= tol
        ua = [x.cpu().numpy() for x in ea.velocity()]
        ub = [x.cpu().numpy() for x in eb.velocity()]
        assert _rel(ub, ua) <= vtol
        # each member's tape: the adjoint of the batched rollout
        Ja, gUa = ea.loss(loss, want_grad=True)
        Jb, gUb = eb.loss(loss, want_grad=True)
        assert abs(Jb - Ja) <= vtol * abs(Ja)
        ga, _, _ = ea.backward(gUa, want_gU0=False)
        gb, _, _ = eb.backward(gUb, want_gU0=False)
        if len(ga):
            assert np.linalg.norm(gb - ga) <= 1e-5 * np.linalg.norm(ga)
    ctx_a.close()
    ctx_b.close()


def test_batch_member_divergence_leaves_the_others(nf):
    members = _batch_members()[:3]
    cfg = dict(precision="mixed", tol=1e-10, max_iters=3000, checkpoint_every=2)
    ctx = nf.Context(**cfg)
    eps = _start(nf, ctx, members)
    bad = eps[1].velocity(dtype=torch.float32)
    bad[0][3, 4, 5] = float("nan")                 # a fluid face of the plate box
    eps[1].set_velocity(bad, project=False)
    st = ctx.step_batch(eps, frames=2)
    assert [s["status"] for s in st] == [0, 4, 0]
    ref = nf.Context(**cfg)
    alone = _start(nf, ref, [members[0]])[0]
    alone.step(2)
    assert _rel([x.cpu().numpy() for x in eps[0].velocity()],
                [x.cpu().numpy() for x in alone.velocity()]) <= 1e-6
    ctx.close()
    ref.close()


def test_step_batch_refuses_members_of_other_sizes(nf):
    ctx = nf.Context(precision="mixed")
    a = ctx.episode(I.make_grid(16, 0.01), I.sphere_scene())
    b = ctx.episode(I.make_grid(24, 0.01), I.sphere_scene())
    with pytest.raises(nf.NFError) as e:
        ctx.step_batch([a, b], frames=1)
    assert e.value.status == 1
    with pytest.raises(nf.NFError):
        ctx.step_batch([a, a], frames=1)
    ctx.close()


def test_served_batches_match_alone_within_tolerance(nf):
    # the serving mix with cross-episode batching: same-size episodes on a
    # slot step as one batch; each result meets the solver tolerance, so
    # loss and gradient agree with the episode alone within it
    eps = _episodes()
    srv = nf.Server(slots=1, batch=1, **CFG)
    alone = {}
    for ep in eps:
        res = _collect(srv, _script(srv, ep))
        alone[ep["key"]] = res[2]
    srv.close_server()
    srv = nf.Server(slots=2, batch=8, **CFG)
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
    assert stats["batches"] >= 1 and stats["batched_requests"] >= 2
    for ep in eps:
        res = mixed[ep["key"]]
        assert all(r["status"] == 0 for r in res), res
        a, m = alone[ep["key"]], res[2]
        assert abs(m["loss"] - a["loss"]) <= 1e-6 * abs(a["loss"])
        g_a = np.asarray(a["g_theta"])
        assert np.linalg.norm(m["g_theta"] - g_a) <= 1e-4 * np.linalg.norm(g_a)


def test_cancel_drops_the_queued_requests_and_closes_the_episode(nf):
    # one slot: the episode's OPEN runs while its queued steps wait; a cancel
    # completes every step that has not started with NF_E_CANCELED (those
    # that ran before it complete normally: a prefix), then closes the
    # episode, whose memory returns; later requests for the key are invalid
    ep = _episodes()[0]
    srv = nf.Server(slots=1, **CFG)
    t_open = srv.open(ep["key"], ep["grid"], ep["scene"])
    steps = [srv.step(ep["key"], frames=1) for _ in range(6)]
    t_cancel = srv.cancel(ep["key"])
    assert srv.drain(wait_ms=300000)
    assert srv.poll(t_open)["status"] == 0
    status = [srv.poll(t)["status"] for t in steps]
    ran = status.index(8) if 8 in status else len(status)
    assert all(s == 0 for s in status[:ran]) and all(s == 8 for s in status[ran:]), status
    assert srv.poll(t_cancel)["status"] == 0
    st = srv.stats()
    assert st["episodes"] == 0 and st["bytes_reserved"] == 0
    assert srv.poll(srv.step(ep["key"]), wait_ms=60000)["status"] == 1
    srv.close_server()


def test_cancel_of_an_episode_waiting_for_memory(nf):
    # a budget that holds one episode: the second OPEN waits; cancelling it
    # completes the OPEN and its step with NF_E_CANCELED at once, reserves
    # nothing, and leaves the first episode's requests untouched
    eps = _episodes()[3:5]                         # two 24^3 episodes
    probe = nf.Server(slots=1, **CFG)
    probe.poll(probe.open(1, eps[0]["grid"], eps[0]["scene"]))
    budget = int(probe.stats()["bytes_reserved"] * 1.5)
    probe.close_server()
    srv = nf.Server(slots=2, hbm_budget=budget, **CFG)
    a = _script(srv, eps[0])
    b_open = srv.open(eps[1]["key"], eps[1]["grid"], eps[1]["scene"])
    b_step = srv.step(eps[1]["key"], frames=1)
    waiting = srv.stats()["open_waiting"]
    b_cancel = srv.cancel(eps[1]["key"])
    assert srv.poll(b_cancel, wait_ms=60000)["status"] == 0
    assert srv.drain(wait_ms=300000)
    assert waiting >= 1
    assert srv.poll(b_open)["status"] == 8 and srv.poll(b_step)["status"] == 8
    assert all(r["status"] == 0 for r in _collect(srv, a))
    assert srv.stats()["bytes_reserved"] == 0
    srv.close_server()
