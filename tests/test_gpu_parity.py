"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances (velocity relative L2 <= 1e-5, gradient relative error <= 1e-4)
are the spec bars; FP64 runs are additionally held to ~1e-9. Grids
span several multigrid levels and include ragged (non power of two, odd)
sizes. The oracle runs on the host in the same process.
"""

import functools

import numpy as np
import pytest

import nf_inputs as I
from oracle import Grid, advect, mac, project, rasterize
from oracle import step as S

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

VEL_TOL = {"fp64": 1e-9, "mixed": 1e-5, "fp32": 1e-5}
GRAD_TOL = {"fp64": 1e-8, "mixed": 1e-4, "fp32": 1e-4}
SOLVE_TOL = {"fp64": 1e-12, "mixed": 1e-10, "fp32": 1e-6}
# Plain FP32 (no FP64 refinement) stalls short of its 1e-6 tolerance on the
# chamber scenes and at 32^3: its true residual stops falling at the rounding
# floor of FP32 vectors (1.7e-5 on the 16^3 chamber). Those solves report
# NF_E_NOT_CONVERGED (a NotConvergedWarning); the tests accept that for FP32
# alone and hold the residual it did reach to this bound. FP64 and MIXED
# must converge.
FP32_REACHED = 1e-4


def solver_warnings(prec):
    """A context manager recording NotConvergedWarnings, and a check to call
    afterwards with the stats of every call made inside it."""
    import contextlib
    import warnings

    from paper_2405_14903_b300.api import NotConvergedWarning

    rec = []

    @contextlib.contextmanager
    def ctx():
        with warnings.catch_warnings(record=True) as w:
            warnings.simplefilter("always", NotConvergedWarning)
            yield
        rec.extend(x for x in w if issubclass(x.category, NotConvergedWarning))

    def check(*stats):
        if prec != "fp32":
            assert not rec, f"{prec} solve missed its tolerance: {rec[0].message}"
        else:
            for st in stats:
                assert st["rel_residual"] <= FP32_REACHED, st
        return len(rec)

    return ctx, check


def rel(a, b):
    a = np.concatenate([np.ravel(np.asarray(x)) for x in a])
    b = np.concatenate([np.ravel(np.asarray(x)) for x in b])
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def host(ts):
    return [t.detach().cpu().numpy() for t in ts]


def _ragged(radius=0.15):
    # odd-sized, non-cubic box (20 x 12 x 14 cells); the sphere stays clear of
    # the walls (a sphere tangent to a wall leaves near-isolated slivers whose
    # gradient contribution is ill-conditioned)
    g = I.make_grid(20, 0.01, ny=12, nz=14)
    sc = I.sphere_scene(v=(0.1, 0.05, -0.02), centre=(0.5, 0.3, 0.35), radius=radius)
    return dict(I.config_sphere(20, steps=2), grid=g, scene=sc, u0=I.gaussian_faces(g, 0.1, 5))


def _viscous(cfg, nu):
    # explicit viscosity (Eq. viscosity_matrix) with nu h / dx^2 in (0.05, 0.13)
    cfg["grid"]["nu"] = float(nu)
    return cfg


def _corner(cfg):
    # the paper's face-area fractions from corner values (Sec. 2.3.1). A
    # solid surface through grid nodes makes phi = 0 at whole faces' corners,
    # where the rule's fluid test (phi >= 0) is decided by rounding; the
    # chamber's duct walls are moved a quarter cell off the nodes
    cfg["grid"]["fractions"] = "corner"
    if cfg["scene"]["kind"] == "chamber":
        cfg["scene"] = dict(cfg["scene"], duct_half=cfg["scene"]["duct_half"] + 0.25 * cfg["grid"]["dx"])
    return cfg


def _inlet(n=16, steps=3, V=0.3):
    # an inflow patch on the low-x wall and an outlet on the high-x wall,
    # a moving sphere between them; kinetic-energy loss (with a prescribed
    # inflow the outflow is fixed by the geometry)
    cfg = I.config_sphere(n, steps=steps)
    cfg["grid"] = I.make_grid(n, 0.01, inlet=I.centred_inlet(n, 4, V),
                              outlet=I.centred_outlet(n, 4))
    cfg["u0"] = I.gaussian_faces(cfg["grid"], 0.1, 4)
    return cfg


def _slab(n=24, steps=3, V=0.3):
    # the 2D variant (App. D) as a one-cell slab between closed z walls:
    # uniform inflow through the whole low-x wall, the high-x wall open, a
    # moving disc (a sphere through the slab) in the channel
    g = I.make_grid(n, 0.005, nz=1,
                    inlet=dict(axis=0, side=-1, j0=0, k0=0, w=n, h=1, speed=V),
                    outlet=dict(axis=0, side=1, j0=0, k0=0, w=n, h=1))
    sc = I.sphere_scene(v=(0.1, 0.02, 0.0), centre=(0.35, 0.5, 0.5 * g["dx"]), radius=0.12)
    u0 = [np.full(I.face_shape(g, 0), V), np.zeros(I.face_shape(g, 1)),
          np.zeros(I.face_shape(g, 2))]
    return dict(name="slab", grid=g, scene=sc, u0=u0, project_initial=True, steps=steps,
                tol=1e-10, loss="kinetic_energy")


def _extruded(n=12):
    # an extruded polar-Bezier obstacle (App. A): one shape, one key section
    # of four segments, theta = its 8 radii
    g = I.make_grid(n, 0.01)
    return dict(name="extruded", grid=g, scene=I.extruded_scene(4, shapes=1, segments=4, keys=1),
                u0=I.gaussian_faces(g, 0.1, 21), project_initial=True, steps=2, tol=1e-12,
                loss="kinetic_energy")


def _extruded_fixed(n=12):
    # two shapes with two key sections each, CSG union, radii fixed (K = 0),
    # the paper's face-area fractions
    g = I.make_grid(n, 0.01)
    g["fractions"] = "corner"
    sc = I.extruded_scene(5, shapes=2, segments=5, keys=2)
    th, j = sc["theta"], 0
    for shp in sc["shapes"]:
        for k in shp["keys"]:
            k["rho"] = th[j:j + 2 * k["nseg"]]
            j += 2 * k["nseg"]
    sc = dict(sc, theta=[], params="fixed")
    return dict(name="extruded_fixed", grid=g, scene=sc, u0=I.gaussian_faces(g, 0.1, 22),
                project_initial=True, steps=2, tol=1e-12, loss="kinetic_energy")


def _heart(n=12, fractions="corner"):
    # the heart of Sec. 3: a chamber and three tubes, each an extruded
    # polar-Bezier part in its own frame, fluid inside their union; the
    # chamber contracts by k(t) (theta = 4 knots); the outlet tube runs
    # through the high-x patch
    g = I.make_grid(n, 0.01, outlet=I.centred_outlet(n, 2))
    g["fractions"] = fractions
    return dict(name="heart", grid=g, scene=I.heart_scene(7, pulse_period=0.06, outlet=True),
                u0=I.zero_faces(g), project_initial=False, steps=2, tol=1e-13, loss="outflow")


CONFIGS = {
    "sphere": lambda: I.config_sphere(16, steps=3),
    "plate": lambda: I.config_plate(16, steps=3),
    "chamber": lambda: I.config_chamber(16, steps=3, duct_half_cells=2),
    "chamber_sub": lambda: I.config_chamber(24, steps=3, duct_half_cells=3, cfl_max=1.5),
    "ragged_sphere": _ragged,
    "sphere32": lambda: I.config_sphere(32, steps=2),
    "spheres": lambda: dict(I.config_spheres(24, count=8), steps=2),
    "sphere_viscous": lambda: _viscous(I.config_sphere(16, steps=3), 0.05),
    "plate_viscous": lambda: _viscous(I.config_plate(16, steps=3), 0.04),
    "chamber_sub_viscous": lambda: _viscous(
        I.config_chamber(24, steps=3, duct_half_cells=3, cfl_max=1.5), 0.02),
    "sphere_corner": lambda: _corner(I.config_sphere(16, steps=3)),
    "plate_corner": lambda: _corner(I.config_plate(16, steps=3)),
    "chamber_corner": lambda: _corner(I.config_chamber(16, steps=3, duct_half_cells=2)),
    "chamber_sub_corner": lambda: _corner(
        I.config_chamber(24, steps=3, duct_half_cells=3, cfl_max=1.5)),
    "spheres_corner": lambda: _corner(dict(I.config_spheres(24, count=8), steps=2)),
    # radius 3.074 dx: no grid node on the sphere at any step time (r = 3 dx
    # about a node centre puts nodes on it at t = 0)
    "ragged_corner": lambda: _corner(_ragged(radius=0.1537)),
    "sphere_inlet": _inlet,
    "slab": _slab,
    "extruded": _extruded,
    "extruded_corner": lambda: _corner(_extruded()),
    "extruded_fixed": _extruded_fixed,
    "heart": _heart,
    "heart_super": lambda: _heart(fractions="supersample"),
    "slab_corner": lambda: _corner(_slab()),
    "sphere_inlet_corner": lambda: _corner(_inlet()),
}


@functools.lru_cache(maxsize=None)
def oracle_rollout(name):
    cfg = CONFIGS[name]()
    J, gth, info = S.loss_and_grad(cfg, tol=1e-13)
    return cfg, J, gth, info


def make_ctx(nf, prec, solver="mgpcg", cfg=None, **kw):
    kw.setdefault("tol", SOLVE_TOL[prec])
    kw.setdefault("max_iters", 3000)
    if cfg is not None:
        kw.setdefault("cfl_max", cfg.get("cfl_max", 0.0))
    return nf.Context(prec, solver, **kw)


def device_u(cfg, dtype=torch.float64):
    return [torch.tensor(x, device="cuda", dtype=dtype) for x in cfg["u0"]]


# ------------------------------------------------------------ per stage ----

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["sphere", "plate", "chamber", "spheres", "sphere_corner",
                                  "plate_corner", "chamber_corner", "spheres_corner",
                                  "ragged_corner", "extruded", "extruded_corner",
                                  "extruded_fixed", "heart", "heart_super"])
def test_fractions_match_oracle(nf, prec, name):
    cfg = CONFIGS[name]()
    g = Grid(cfg["grid"])
    ctx = make_ctx(nf, prec)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    got = host(ep.fractions())
    ref = rasterize.fractions(g, cfg["scene"], 0.0)
    tol = 1e-13 if prec == "fp64" else 1e-7
    for d in range(3):
        np.testing.assert_allclose(got[d], ref[d], rtol=0, atol=tol)


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("solver", ["cg", "mgpcg"])
@pytest.mark.parametrize("name", ["sphere", "plate", "ragged_sphere", "spheres", "sphere32"])
def test_initial_projection_matches_oracle(nf, prec, solver, name):
    if prec == "fp32" and solver == "cg":
        pytest.skip("plain FP32 CG is not one of the configured paths")
    cfg, _, _, info = oracle_rollout(name)
    ctx = make_ctx(nf, prec, solver)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    ep.set_velocity(device_u(cfg), project=True)
    t0 = info["tapes"][0]
    g = Grid(cfg["grid"])
    GP = mac.grad(g, t0["P"])
    ref = [t0["alpha"][d] * (t0["Uh"][d] - g.c * GP[d]) + (1 - t0["alpha"][d]) * t0["us"][d]
           for d in range(3)]
    assert rel(host(ep.velocity()), ref) <= VEL_TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["sphere", "plate", "chamber", "ragged_sphere",
                                  "sphere_inlet", "slab"])
def test_one_step_stages_match_oracle(nf, prec, name):
    cfg = CONFIGS[name]()
    g = Grid(cfg["grid"])
    ctx = make_ctx(nf, prec)   # single steps of dt (no sub-stepping)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    rng = np.random.default_rng(7)
    U = [0.3 * rng.standard_normal(g.face_shape(d)) for d in range(3)]
    ep.set_velocity([torch.tensor(u, device="cuda") for u in U], project=False)
    ep.step(1)
    U1, tape = S.step(g, cfg["scene"], U, 0, 1e-13)
    assert rel(host(ep.advected()), advect.advect(g, U)) <= VEL_TOL[prec]
    assert rel(host(ep.fractions()), tape["alpha"]) <= 1e-7
    assert rel(host(ep.velocity()), U1) <= VEL_TOL[prec]
    # pressure: gauge-free face differences on faces with alpha > 0
    GP = mac.grad(g, host([ep.pressure()])[0])
    GPr = mac.grad(g, tape["P"])
    for d in range(3):
        m = tape["alpha"][d] > 0
        if not m.any():
            continue          # the slab's z faces are all walls
        scale = np.abs(GPr[d][m]).max()
        assert np.abs(GP[d][m] - GPr[d][m]).max() <= 1e3 * VEL_TOL[prec] * scale


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("nu", [0.03, 0.16])
def test_viscous_step_matches_oracle_face_by_face(nf, prec, nu):
    # ragged 20 x 12 x 14 box: U^ = (I - nu dt/dx^2 G^T G) B(U) U compared
    # face by face (lattice ends at every wall), then the projected velocity;
    # nu = 0.16 gives nu dt / dx^2 = 0.64, past explicit stability, which
    # the step computes as written
    cfg = _ragged()
    cfg["grid"]["nu"] = nu
    g = Grid(cfg["grid"])
    ctx = make_ctx(nf, prec)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    rng = np.random.default_rng(17)
    U = [0.3 * rng.standard_normal(g.face_shape(d)) for d in range(3)]
    ep.set_velocity([torch.tensor(u, device="cuda") for u in U], project=False)
    ep.step(1)
    U1, tape = S.step(g, cfg["scene"], U, 0, 1e-13)
    want = advect.viscosity(g, advect.advect(g, U))
    got = host(ep.advected())
    tol = 1e-12 if prec == "fp64" else 2e-6
    for d in range(3):
        scale = np.abs(want[d]).max()
        np.testing.assert_allclose(got[d], want[d], rtol=0, atol=tol * scale)
    assert rel(host(ep.velocity()), U1) <= VEL_TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_inflow_patch_outflow_equals_inflow(nf, prec):
    # incompressibility with one inflow and one outflow patch: the net flux
    # out equals the prescribed inflow (a rigid sphere adds none), on the
    # GPU as in the oracle's pin
    cfg = _inlet(16, steps=2, V=0.3)
    g = Grid(cfg["grid"])
    ctx = make_ctx(nf, prec)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    ep.set_velocity(device_u(cfg), project=True)
    ep.step(2)
    J = ep.loss("outflow")
    assert abs(J - 0.3 * 16 * g.dx ** 2) <= 1e-6 * J
    # the inlet faces hold the inflow speed exactly
    U = host(ep.velocity())
    i0 = cfg["grid"]["inlet"]
    patch = U[0][i0["k0"]:i0["k0"] + 4, i0["j0"]:i0["j0"] + 4, 0]
    np.testing.assert_allclose(patch, 0.3, rtol=0, atol=1e-7)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_slab_keeps_the_flow_planar_and_the_outflow_equal_to_the_inflow(nf, prec):
    # one-cell slab: u_z stays exactly zero (its faces are the z walls), and
    # with inflow over the whole low-x wall and the high-x wall open the net
    # outflow equals the inflow
    cfg = _slab(24, steps=4)
    g = Grid(cfg["grid"])
    ctx = make_ctx(nf, prec)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    ep.set_velocity(device_u(cfg), project=True)
    ep.step(cfg["steps"])
    U = host(ep.velocity())
    assert not np.any(U[2])
    assert np.abs(U[1]).max() > 1e-3               # the disc deflects the flow
    J = ep.loss("outflow")
    assert abs(J - 0.3 * 24 * g.dx ** 2) <= 1e-6 * J


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_divergence_free_after_step(nf, prec):
    cfg = CONFIGS["plate"]()
    g = Grid(cfg["grid"])
    ctx = make_ctx(nf, prec)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    ep.set_velocity(device_u(cfg), project=True)
    ep.step(2)
    U = host(ep.velocity())
    act = project.active_cells(g, host(ep.fractions()))
    div = np.abs(mac.grad_T(g, U))[act].max()
    scale = max(np.abs(u).max() for u in U)
    assert div <= (1e-10 if prec == "fp64" else 1e-5) * scale


# ------------------------------------------------------ rollout adjoint ----

@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("name", ["sphere", "plate", "chamber", "chamber_sub", "ragged_sphere",
                                  "sphere32", "sphere_viscous", "plate_viscous",
                                  "chamber_sub_viscous", "sphere_corner", "plate_corner",
                                  "chamber_sub_corner", "ragged_corner", "sphere_inlet",
                                  "sphere_inlet_corner", "slab", "slab_corner", "extruded",
                                  "extruded_corner", "extruded_fixed", "heart"])
def test_rollout_loss_and_gradient_match_oracle(nf, prec, name):
    cfg, Jo, gtho, info = oracle_rollout(name)
    ctx = make_ctx(nf, prec, cfg=cfg, checkpoint_every=2)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    recording, check = solver_warnings(prec)
    with recording():
        s0 = ep.set_velocity(device_u(cfg), project=cfg["project_initial"])
        fs = ep.step(cfg["steps"])
        J, gU = ep.loss(cfg["loss"], want_grad=True)
        gth, gU0, st = ep.backward(gU)
    check(s0, fs, st)
    assert abs(J - Jo) <= VEL_TOL[prec] * abs(Jo)
    assert np.linalg.norm(gth - gtho) <= GRAD_TOL[prec] * np.linalg.norm(gtho)
    assert st["steps"] == sum(1 for t in info["tapes"] if t["kind"] == "step")
    scale = max(np.abs(x).max() for x in host(gU))
    if name.startswith(("chamber", "heart")):
        # the outflow is a function of the geometry alone: dJ/dU^0 vanishes
        # up to solver tolerance (oracle and GPU both)
        assert max(np.abs(x).max() for x in host(gU0)) <= 1e-3 * scale
    else:
        assert rel(host(gU0), info["gU0"]) <= GRAD_TOL[prec]


@pytest.mark.parametrize("C", [1, 3, 10])
def test_checkpoint_interval_does_not_change_the_gradient(nf, C):
    cfg, Jo, gtho, _ = oracle_rollout("plate")
    ctx = make_ctx(nf, "mixed", checkpoint_every=C)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    ep.set_velocity(device_u(cfg), project=True)
    ep.step(cfg["steps"])
    _, gU = ep.loss("kinetic_energy", want_grad=True)
    gth, _, _ = ep.backward(gU, want_gU0=False)
    assert np.linalg.norm(gth - gtho) <= 1e-4 * np.linalg.norm(gtho)


def test_forward_is_bitwise_deterministic(nf):
    cfg = CONFIGS["sphere"]()
    ctx = make_ctx(nf, "mixed")
    outs = []
    for _ in range(2):
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        ep.set_velocity(device_u(cfg), project=True)
        ep.step(3)
        outs.append(host(ep.velocity(dtype=torch.float32)))
        ep.close()
    for a, b in zip(*outs):
        assert np.array_equal(a, b)


def test_backward_steps_compose_to_backward(nf):
    cfg, _, gtho, info = oracle_rollout("sphere")
    ctx = make_ctx(nf, "fp64", checkpoint_every=2)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    ep.set_velocity(device_u(cfg), project=True)
    ep.step(cfg["steps"])
    _, gU = ep.loss("kinetic_energy", want_grad=True, dtype=torch.float64)
    total = np.zeros(3)
    g = gU
    for _ in range(cfg["steps"] + 1):          # steps, then the initial projection
        g, gth, _ = ep.backward_step(g)
        total += gth
    np.testing.assert_allclose(total, gtho, rtol=1e-8, atol=1e-12 * np.abs(gtho).max())
    assert rel(host(g), info["gU0"]) <= 1e-8
    with pytest.raises(nf.NFError):
        ep.backward_step(g)


def test_autograd_function_matches_oracle(nf):
    cfg, Jo, gtho, info = oracle_rollout("plate")
    ctx = make_ctx(nf, "mixed")
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    theta = torch.tensor(cfg["scene"]["theta"], dtype=torch.float64, device="cuda", requires_grad=True)
    u0 = [torch.tensor(x, device="cuda", dtype=torch.float32, requires_grad=True) for x in cfg["u0"]]
    J = nf.rollout_loss(ep, theta, u0, cfg["steps"], "kinetic_energy", project=True)
    J.backward()
    assert abs(J.item() - Jo) <= 1e-5 * abs(Jo)
    g = theta.grad.cpu().numpy()
    assert np.linalg.norm(g - gtho) <= 1e-4 * np.linalg.norm(gtho)
    assert rel(host([u.grad for u in u0]), info["gU0"]) <= 1e-4


# ------------------------------------------------ memory kinds, dtypes ----

def test_host_and_device_inputs_agree(nf):
    cfg = CONFIGS["sphere"]()
    ctx = make_ctx(nf, "mixed")
    a = ctx.episode(cfg["grid"], cfg["scene"])
    b = ctx.episode(cfg["grid"], cfg["scene"])
    a.set_velocity(device_u(cfg), project=True)
    b.set_velocity([np.asarray(x, dtype=np.float32) for x in cfg["u0"]], project=True)
    a.step(1)
    b.step(1)
    ua = host(a.velocity(dtype=torch.float32))
    ub = b.velocity(dtype=torch.float32, host=True)
    for x, y in zip(ua, ub):
        assert np.array_equal(x, y)


# ------------------------------------------------------------ statuses ----

def test_iteration_cap_reports_not_converged(nf):
    cfg = CONFIGS["plate"]()
    ctx = make_ctx(nf, "fp64", solver="cg", tol=1e-12, max_iters=3)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    with pytest.warns(nf.NotConvergedWarning):
        st = ep.set_velocity(device_u(cfg), project=True)
    assert st["iters"] <= 3 and st["rel_residual"] > 1e-12


def test_invalid_calls_raise(nf):
    ctx = make_ctx(nf, "mixed")
    with pytest.raises(nf.NFError):
        ctx.episode(I.make_grid(2, 0.01), I.sphere_scene())        # too small
    bad = I.config_chamber(16, duct_half_cells=2)
    g = dict(bad["grid"])
    g["outlet"] = dict(g["outlet"], w=40)
    with pytest.raises(nf.NFError):
        ctx.episode(g, bad["scene"])                                 # outlet outside
    with pytest.raises(nf.NFError):
        ctx.episode(I.make_grid(8, 0.01, nu=-0.1), I.sphere_scene()) # nu < 0
    # an unknown fraction rule, through the C ABI (the binding refuses it first)
    import ctypes
    from paper_2405_14903_b300 import _lib as L
    from paper_2405_14903_b300.api import grid_struct, scene_struct
    gs = grid_struct(I.make_grid(8, 0.01))
    gs.fractions = 7
    ss, _keep = scene_struct(I.sphere_scene())
    eid = ctypes.c_int64()
    assert L.lib.nf_episode_create(ctx.handle, ctypes.byref(gs), ctypes.byref(ss),
                                   ctypes.byref(eid)) == L.NF_E_INVALID
    with pytest.raises(ValueError):
        ctx.episode(dict(I.make_grid(8, 0.01), fractions="marching"), I.sphere_scene())
    cfg = CONFIGS["sphere"]()
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    with pytest.raises(nf.NFError):
        ep.set_params([0.1, 0.2])                                    # wrong K
    gU = [torch.zeros(s, device="cuda") for s in ep.face_shapes]
    with pytest.raises(nf.NFError) as e:
        ep.backward(gU)                                              # nothing recorded
    assert e.value.status == 7
    with pytest.raises(nf.NFError):
        ep.loss("outflow")                                           # no outlet


def test_non_finite_velocity_reports_diverged_and_the_context_recovers(nf):
    # a poisoned input (NaN in one fluid face) made on the host: the
    # projection's residual turns non-finite and the call returns
    # NF_E_DIVERGED instead of iterating; a step from it does the same
    cfg = CONFIGS["sphere"]()
    ctx = make_ctx(nf, "mixed")
    u = device_u(cfg)
    u[0][3, 4, 5] = float("nan")                 # fluid: far from the sphere
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    with pytest.raises(nf.NFError) as e:
        ep.set_velocity(u, project=True)
    assert e.value.status == 4
    ep2 = ctx.episode(cfg["grid"], cfg["scene"])
    ep2.set_velocity(u, project=False)
    with pytest.raises(nf.NFError) as e:
        ep2.step(1)
    assert e.value.status == 4
    ep3 = ctx.episode(cfg["grid"], cfg["scene"])
    ep3.set_velocity(device_u(cfg), project=True)
    ep3.step(1)
    assert all(np.isfinite(x).all() for x in host(ep3.velocity()))


def test_hbm_budget_refuses_admission(nf):
    cfg = CONFIGS["sphere"]()
    ctx = make_ctx(nf, "mixed", hbm_budget=64 << 10)
    with pytest.raises(nf.NFError) as e:
        ctx.episode(cfg["grid"], cfg["scene"])
    assert e.value.status == 2


# ------------------------------------------------------ solver variants ----

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("variant", [
    dict(mg_transfer="trilinear", mg_coarse_weight=1.0),
    dict(mg_transfer="trilinear", mg_coarse_weight=1.0, mg_band_sweeps=1),
    dict(mg_transfer="constant", mg_coarse_weight=1.0, mg_smooth=1),
    dict(mg_transfer="constant", mg_coarse_weight=1.8, mg_coarsest_sweeps=2),
    dict(mg_smooth=2, mg_smooth_coarse=1),
    dict(residual_fp64=False),
], ids=["trilinear", "trilinear_band", "constant_unweighted", "constant_1.8", "coarse_nu1",
        "residual_split_float"])
def test_multigrid_variants_match_oracle(nf, prec, variant):
    # the preconditioner changes the iterations, never the solution
    cfg, Jo, gtho, info = oracle_rollout("chamber_sub")
    ctx = make_ctx(nf, prec, cfg=cfg, checkpoint_every=2, **variant)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    ep.set_velocity(device_u(cfg), project=cfg["project_initial"])
    ep.step(cfg["steps"])
    J, gU = ep.loss(cfg["loss"], want_grad=True)
    gth, _, st = ep.backward(gU)
    assert abs(J - Jo) <= VEL_TOL[prec] * abs(Jo)
    assert np.linalg.norm(gth - gtho) <= GRAD_TOL[prec] * np.linalg.norm(gtho)


# ------------------------------------------- persistent coarse levels ----
# From 48^3 up, coarse levels of at most 64^3 cells lie between the finest
# levels (one launch per phase) and the one-block chain; they run as the
# phases of one cooperative kernel unless mg_persistent is off. Both paths
# do the same per-cell arithmetic, so they take the same iterations.

@functools.lru_cache(maxsize=None)
def oracle_projection(n, kind):
    cfg = I.config_sphere(n, steps=0) if kind == "sphere" else I.config_spheres(n, count=8)
    U, _ = S.initial_projection(Grid(cfg["grid"]), cfg["scene"], cfg["u0"], 1e-12)
    return cfg, U


@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("case", [(64, "sphere"), (48, "spheres")], ids=["sphere64", "spheres48"])
def test_persistent_coarse_levels_match_per_phase_launches_and_oracle(nf, prec, case):
    cfg, U_ref = oracle_projection(*case)
    out = {}
    for persistent in (True, False):
        ctx = make_ctx(nf, prec, mg_persistent=persistent)
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        st = ep.set_velocity(device_u(cfg), project=True)
        out[persistent] = (st, host(ep.velocity()))
        ep.close()
        ctx.close()
    (sp, up), (sn, un) = out[True], out[False]
    assert sp["iters"] == sn["iters"] and sp["outer"] == sn["outer"]
    assert rel(up, un) <= (1e-12 if prec == "fp64" else 1e-6)
    assert rel(up, U_ref) <= VEL_TOL[prec]


# ------------------------------------------------------- bounded waits ----
# Every device wait (the cooperative kernel's grid barriers, the chain's
# mbarrier) gives up after about a second. The test hook makes them wait for
# something that never comes: the solve must end with NF_E_TIMEOUT (status 5)
# within seconds and the context must stay usable.

@pytest.mark.parametrize("persistent", [False, True], ids=["chain_mbarrier", "grid_barrier"])
def test_expired_device_waits_report_timeout_and_the_context_recovers(nf, monkeypatch, persistent):
    import time
    cfg = I.config_sphere(64, steps=0)
    monkeypatch.setenv("NF_TEST_STALL_WAITS", "1")
    ctx = make_ctx(nf, "mixed", mg_persistent=persistent, max_iters=50)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    monkeypatch.delenv("NF_TEST_STALL_WAITS")
    t0 = time.time()
    with pytest.raises(nf.NFError) as e:
        ep.set_velocity(device_u(cfg), project=True)
    assert e.value.status == 5
    assert time.time() - t0 < 60
    ep.close()
    ctx.close()
    ctx = make_ctx(nf, "mixed", mg_persistent=persistent)   # without the hook
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    st = ep.set_velocity(device_u(cfg), project=True)
    assert st["rel_residual"] <= SOLVE_TOL["mixed"]
    ep.close()
    ctx.close()


# -------------------------------------------------------- launch paths ----
# The solver runs its iterations in a device-side conditional-graph loop by
# default, in replayed batches of graphs while profiling, and as direct
# launches with NF_GRAPHS=0. The kernels and their order are the same (the
# other paths only add launches that return at once), so a forward rollout
# gives the same bits and iteration counts on all three. The forward's
# rasterisation runs on a side stream beside the advection except while
# profiling, so the comparison also checks that fork and join order it.

@pytest.mark.parametrize("name,tape", [("chamber_sub", False), ("chamber_sub", True),
                                       ("plate", True), ("sphere32", False)])
def test_launch_paths_give_the_same_bits(nf, monkeypatch, name, tape):
    cfg = CONFIGS[name]()

    def run(profile=False, graphs=True):
        if not graphs:
            monkeypatch.setenv("NF_GRAPHS", "0")
        ctx = make_ctx(nf, "mixed", cfg=cfg, tape_fractions=tape)
        if profile:
            ctx.profile("all")
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        monkeypatch.delenv("NF_GRAPHS", raising=False)
        ep.set_velocity(device_u(cfg), project=cfg["project_initial"])
        st = ep.step(cfg["steps"])
        U = host(ep.velocity())
        ep.close()
        ctx.close()
        return st, U

    (sa, ua), (sb, ub), (sc, uc) = run(), run(profile=True), run(graphs=False)
    assert sa["iters"] == sb["iters"] == sc["iters"] and sa["outer"] == sb["outer"] == sc["outer"]
    for x, y, z in zip(ua, ub, uc):
        assert np.array_equal(x, y) and np.array_equal(x, z)


# ------------------------------------------------ cluster coarse levels ----
# With mg_cluster, from 64^3 up the levels just above an 8^3 chain (32^3
# and 16^3) run as z-slabs on one 8-CTA thread-block cluster. Per cell the
# arithmetic is the per-launch path's, so a projection gives the same bits
# and iterations either way.

@pytest.mark.parametrize("n", [64, 128])
def test_cluster_coarse_levels_give_the_per_launch_bits(nf, n):
    cfg = I.config_chamber(n, steps=1, seed=0, duct_half_cells=max(2, n // 16))
    out = {}
    for cluster in (True, False):
        ctx = make_ctx(nf, "mixed", cfg=cfg, mg_cluster=cluster, tol=1e-8)
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        st = ep.set_velocity(device_u(cfg, torch.float32), project=True)
        fst = ep.step(1)
        out[cluster] = (st, fst, host(ep.velocity()))
        ep.close()
        ctx.close()
    (s1, f1, u1), (s0, f0, u0) = out[True], out[False]
    assert s1["iters"] == s0["iters"] and f1["iters"] == f0["iters"]
    for a, b in zip(u1, u0):
        assert np.array_equal(a, b)


# ------------------------------------------------------------------ dots ----

@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
def test_solver_dot_error_at_256_cubed(nf, dtype):
    # the CG inner products at the size of the precision sweep (256^3 cells):
    # FP32 vectors give exact products and compensated per-thread sums, so
    # the whole dot is within a few FP64 roundings of the exact value
    n = 256 ** 3
    g = torch.Generator(device="cpu").manual_seed(3)
    a = torch.randn(n, generator=g, dtype=torch.float64).to(dtype)
    b = (torch.randn(n, generator=g, dtype=torch.float64) + 0.25).to(dtype)
    ctx = nf.Context("mixed" if dtype == torch.float32 else "fp64")
    got = ctx.dot(a.cuda(), b.cuda())
    ctx.close()
    import math
    ad, bd = a.double().numpy(), b.double().numpy()
    exact = math.fsum((ad * bd).tolist())         # products of floats are exact in FP64
    scale = float(np.abs(ad * bd).sum())
    assert abs(got - exact) <= 1e-12 * scale, (got, exact, scale)


# ------------------------------------------------- fused sweep pairs ----

@pytest.mark.parametrize("prec", ["fp64", "mixed", "fp32"])
@pytest.mark.parametrize("name", ["chamber_sub", "ragged_sphere", "sphere32", "plate64"])
def test_fused_sweep_pairs_give_the_per_launch_bits(nf, prec, name):
    # the red-black pairs as one shared-memory launch each (finest level;
    # every grid level) against one launch per half sweep: the same arithmetic in the same
    # order, so the rollout, its adjoint and the iteration counts agree
    # exactly (ragged sizes, several tiles and z chunks, block edges)
    cfg = I.config_plate(64, steps=2) if name == "plate64" else CONFIGS[name]()
    out = []
    for fused in (0, 1, 2):
        ctx = make_ctx(nf, prec, cfg=cfg, checkpoint_every=2, mg_fused=fused)
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        recording, _ = solver_warnings(prec)
        with recording():
            ep.set_velocity(device_u(cfg), project=cfg["project_initial"])
            fs = ep.step(cfg["steps"])
            J, gU = ep.loss(cfg["loss"], want_grad=True)
            gth, _, bs = ep.backward(gU, want_gU0=False)
        out.append((host(ep.velocity()), J, gth, fs["iters"], bs["iters"]))
        ep.close()
        ctx.close()
    u0, J0, g0, i0, b0 = out[0]
    for u1, J1, g1, i1, b1 in out[1:]:
        assert i0 == i1
        assert J0 == J1
        for a, b in zip(u0, u1):
            assert np.array_equal(a, b)
        # the adjoint's advection scatter uses float atomics, so its
        # right-hand sides (and then an adjoint solve's iteration count, by
        # one) vary from run to run at rounding level, fused or not; plain
        # FP32 solves end where their residual stalls at the rounding floor,
        # which moves the count by a few iterations over the rollout
        assert abs(b1 - b0) <= (2 if prec != "fp32" else max(6, b0 // 20))
        tol = 1e-10 if prec == "fp64" else 1e-5
        assert np.linalg.norm(g1 - g0) <= tol * np.linalg.norm(g0)


# --------------------------------------------------------------- resume ----

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_exported_episode_resumes_bit_for_bit(nf, prec):
    # an episode exported after 3 frames and imported into a fresh one
    # continues exactly as the original: the forward step is deterministic
    # and the frame clock (the geometry's time) is restored
    cfg = I.config_chamber(16, steps=5, duct_half_cells=2, cfl_max=1.0)
    ctx = make_ctx(nf, prec, cfg=cfg)
    a = ctx.episode(cfg["grid"], cfg["scene"])
    a.set_velocity(device_u(cfg), project=False)
    a.step(3)
    state = a.export_state()
    a.step(2)
    b = ctx.episode(cfg["grid"], cfg["scene"])
    b.set_params(np.zeros(8))                          # overwritten by the import
    b.import_state(state)
    b.step(2)
    for x, y in zip(host(a.velocity()), host(b.velocity())):
        assert np.array_equal(x, y)
    # the tape starts at the import: the adjoint reaches back two frames
    J, gU = b.loss("outflow", want_grad=True)
    _, _, st = b.backward(gU, want_gU0=False)
    assert st["steps"] == b.step_index()
    # refused: another grid, a truncated or foreign buffer
    c = ctx.episode(I.make_grid(8, 0.005, outlet=I.centred_outlet(8, 2)),
                    I.config_chamber(8, duct_half_cells=1)["scene"])
    for bad in (state, state[:-8], b"x" * len(state)):
        with pytest.raises(nf.NFError) as e:
            (c if bad is state else b).import_state(bad)
        assert e.value.status == 1


# ------------------------------------------------ overlapped recompute ----

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["chamber_sub", "plate", "sphere_viscous"])
def test_overlapped_recompute_gives_the_sequential_gradient(nf, prec, name):
    # the backward pass recomputing the next checkpoint segment on a second
    # stream (helper thread) while it reverts the current one: the same
    # kernels on the same data, so the loss is bitwise equal and the
    # gradient equal to rounding (float-atomic scatter in the advection
    # adjoint); many segments (checkpoint every 2 steps)
    cfg, Jo, gtho, info = oracle_rollout(name)
    out = []
    for overlap in (False, True):
        ctx = make_ctx(nf, prec, cfg=cfg, checkpoint_every=2, recompute_overlap=overlap)
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        ep.set_velocity(device_u(cfg), project=cfg["project_initial"])
        fs = ep.step(cfg["steps"])
        J, gU = ep.loss(cfg["loss"], want_grad=True)
        gth, gU0, bs = ep.backward(gU)
        out.append((J, gth, host(gU0), bs))
        ep.close()
        ctx.close()
    (J0, g0, u0, b0), (J1, g1, u1, b1) = out
    assert J0 == J1
    assert b1["steps"] == b0["steps"] and b1["solves"] == b0["solves"]
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert np.linalg.norm(g1 - g0) <= tol * np.linalg.norm(g0)
    assert rel(u1, u0) <= tol
    assert np.linalg.norm(g1 - gtho) <= GRAD_TOL[prec] * np.linalg.norm(gtho)



# ---------------------------------------------- integer-bit conversions ----

def _conversion_cases():
    rng = np.random.default_rng(11)
    f32 = np.finfo(np.float32)
    # doubles over and beyond the FP32 range, both signs
    e = rng.integers(-160, 140, 20000)
    v = [rng.uniform(1.0, 2.0, e.size) * np.ldexp(1.0, e) * rng.choice([-1.0, 1.0], e.size)]
    # exact ties between neighbouring floats (round half to even) and their neighbours
    f = rng.uniform(-1e4, 1e4, 5000).astype(np.float32)
    up = np.nextafter(f, np.float32(np.inf))
    mid = (f.astype(np.float64) + up.astype(np.float64)) / 2.0
    v += [mid, np.nextafter(mid, np.inf), np.nextafter(mid, -np.inf), f.astype(np.float64)]
    # range edges: largest float and the tie above it, smallest normal and subnormals
    top = float(f32.max)
    v.append(np.array([0.0, -0.0, np.inf, -np.inf, np.nan, top, -top,
                       top * (1.0 + 2.0 ** -25), top * (1.0 + 2.0 ** -24),
                       float(f32.tiny), float(f32.tiny) * 0.5, float(f32.tiny) * (1 - 2 ** -24),
                       2.0 ** -149, 2.0 ** -150, 2.0 ** -151, 1.0, -1.0, 0.5, 3.0 ** 0.5,
                       np.finfo(np.float64).tiny, np.finfo(np.float64).max]))
    # fractions as the kernels see them: multiples of 1/64 and random values in [0, 1]
    v += [np.arange(65) / 64.0, rng.uniform(0.0, 1.0, 5000)]
    return np.concatenate(v)


def test_integer_bit_conversions_match_the_instructions(nf):
    # the face kernels' FP64 -> FP32 rounding and FP32 -> FP64 widening by
    # integer operations (the conversion instructions run on the slow FP64
    # pipe) against the instructions on the device and against NumPy's
    # round-to-nearest-even casts
    vals = _conversion_cases()
    ctx = nf.Context("mixed", "mgpcg")
    out_f, out_d, bad = ctx.check_conversions(vals)
    ctx.close()
    assert bad == 0
    with np.errstate(over="ignore"):
        ref_f = vals.astype(np.float32)
    nan = np.isnan(ref_f)
    assert np.array_equal(np.isnan(out_f), nan)
    assert np.array_equal(out_f[~nan].view(np.uint32), ref_f[~nan].view(np.uint32))
    ref_d = ref_f.astype(np.float64)
    assert np.array_equal(out_d[~nan].view(np.uint64), ref_d[~nan].view(np.uint64))
