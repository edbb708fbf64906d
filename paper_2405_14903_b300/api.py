"""Python binding of libnf: argument marshalling over the C ABI.

``Context`` wraps ``nf_ctx`` (device, stream, precision and solver
settings); ``Episode`` wraps one simulated grid. Device arrays are torch
tensors (their ``data_ptr`` is passed through); host arrays are NumPy arrays
or CPU tensors. Grid and scene descriptions are the plain dictionaries of
``nf_inputs``. Every call checks the returned status and raises
:class:`NFError` on failure.

Stream ordering: by default a context runs on torch's current stream of its
device, so library work and torch work on the same stream are ordered. The
legacy default stream (handle 0 in torch) is passed as ``cudaStreamLegacy``
because the C ABI reads a null stream as "create a private stream".
"""

from __future__ import annotations

import ctypes as C
import warnings

import numpy as np
import torch

from . import _lib as L

lib = L.lib


class NFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"libnf status {status} ({lib.nf_status_string(status).decode()}): {msg}")
        self.status = status


class NotConvergedWarning(RuntimeWarning):
    pass


def _check(status, ctx=None, allow_not_converged=True):
    if status == L.NF_OK:
        return status
    msg = lib.nf_last_error(ctx).decode() if ctx is not None else ""
    if status == L.NF_E_NOT_CONVERGED and allow_not_converged:
        warnings.warn(f"solver did not reach its tolerance: {msg}", NotConvergedWarning)
        return status
    raise NFError(status, msg)


def grid_struct(desc):
    g = L.Grid()
    g.nx, g.ny, g.nz = desc["nx"], desc["ny"], desc["nz"]
    g.dx, g.dt, g.rho = desc["dx"], desc["dt"], desc.get("rho", 1.0)
    if desc.get("periodic", False):
        raise ValueError("the CUDA path implements closed boxes (walls and an outlet patch)")
    i = desc.get("inlet")
    if i:
        if i["axis"] != 0 or i["side"] not in (-1, 1):
            raise ValueError("inflow patches are on an x wall")
        g.inlet, g.inlet_side = 1, int(i["side"])
        g.inlet_j0, g.inlet_k0, g.inlet_w, g.inlet_h = i["j0"], i["k0"], i["w"], i["h"]
        g.inlet_speed = float(i["speed"])
    g.nu = float(desc.get("nu", 0.0))
    rule = desc.get("fractions", "supersample")
    if rule not in L.FRACTIONS:
        raise ValueError(f"unknown fraction rule {rule!r}")
    g.fractions = L.FRACTIONS[rule]
    o = desc.get("outlet")
    if o:
        if o["axis"] != 0 or o["side"] != 1:
            raise ValueError("outlet patches are on the high-x wall")
        g.outlet, g.outlet_j0, g.outlet_k0, g.outlet_w, g.outlet_h = 1, o["j0"], o["k0"], o["w"], o["h"]
    return g


def scene_struct(sc):
    s = L.Scene()
    kind = sc["kind"]
    if kind not in L.SCENE:
        raise ValueError(f"scene kind {kind!r} is not implemented on the GPU")
    s.kind = L.SCENE[kind]
    th = list(sc.get("theta", []))
    s.K = len(th)
    for k, v in enumerate(th):
        s.theta[k] = v
    consts = []
    keep = None
    if kind == "sphere":
        consts = list(sc["centre"]) + [sc["radius"]]
    elif kind == "chamber":
        consts = list(sc["centre"]) + list(sc["axes"]) + [sc["period"], sc["duct_x0"], sc["duct_half"]]
    elif kind == "plate":
        consts = list(sc["centre"]) + list(sc["half"]) + [sc["period"]]
    elif kind == "spheres":
        keep = np.ascontiguousarray(np.asarray(sc["spheres"], dtype=np.float64).reshape(-1, 4))
        s.spheres = keep.ctypes.data_as(C.POINTER(C.c_double))
        s.nspheres = keep.shape[0]
    elif kind == "extruded":
        keep = extruded_table(sc)
        s.shapes = keep.ctypes.data_as(C.POINTER(C.c_double))
        s.nshape_values = keep.size
        mode = {"radii": 0, "pulse": 1}.get(sc.get("params", "radii"), 2)
        pulse = sc.get("pulse") or {}
        consts = [len(sc["shapes"]), 1.0 if sc["fluid"] == "inside" else 0.0, mode,
                  pulse.get("shape", 0), pulse.get("period", 0.0)]
    for k, v in enumerate(consts):
        s.consts[k] = v
    return s, keep


def extruded_table(sc):
    """The shape table of an ``extruded`` scene description (the layout of
    nf_scene.shapes in nf.h): per shape n keys, N segments, z0, z1, the
    frame (flag, origin, axes), then every key's centre and radii (theta's
    in radii mode, else the key's own)."""
    th = list(sc.get("theta", []))
    radii_mode = sc.get("params", "radii") == "radii"
    out, j = [], 0
    for sh in sc["shapes"]:
        keys = sh["keys"]
        N = int(keys[0]["nseg"])
        if any(int(k["nseg"]) != N for k in keys):
            raise ValueError("every key of a shape has the same number of segments")
        fr = sh.get("frame")
        out += [len(keys), N, float(sh["z0"]), float(sh["z1"]), 1.0 if fr else 0.0]
        out += list(fr["origin"]) if fr else [0.0, 0.0, 0.0]
        out += [float(v) for row in fr["axes"] for v in row] if fr else [1.0, 0, 0, 0, 1.0, 0, 0, 0, 1.0]
        for k in keys:
            out += [float(k["c"][0]), float(k["c"][1])]
            if radii_mode:
                out += th[j:j + 2 * N]
                j += 2 * N
            else:
                out += [float(v) for v in k["rho"]]
    return np.ascontiguousarray(np.asarray(out, dtype=np.float64))


def _ptrs(arrs):
    """(pointer triple, dtype code, memory kind, keep-alive list)."""
    arrs = list(arrs)
    if isinstance(arrs[0], torch.Tensor):
        dt = arrs[0].dtype
        if dt not in (torch.float32, torch.float64):
            raise TypeError("arrays must be float32 or float64")
        ts = [a.contiguous() for a in arrs]
        if not all(t.dtype == dt for t in ts):
            raise TypeError("all components must share a dtype")
        code = L.NF_F64 if dt == torch.float64 else L.NF_F32
        mem = L.NF_MEM_DEVICE if ts[0].is_cuda else L.NF_MEM_HOST
        return L.P3(*[t.data_ptr() for t in ts]), code, mem, ts
    nps = [np.ascontiguousarray(a) for a in arrs]
    dt = nps[0].dtype
    if dt not in (np.float32, np.float64) or not all(a.dtype == dt for a in nps):
        raise TypeError("host arrays must all be float32 or all float64")
    code = L.NF_F64 if dt == np.float64 else L.NF_F32
    return L.P3(*[a.ctypes.data for a in nps]), code, L.NF_MEM_HOST, nps


def loss_noalloc(kind, grid, u, gU=None, stream=None):
    """``nf_loss_noalloc``: the loss of ``Episode.loss`` for the device face
    triple ``u`` (CUDA tensors of one dtype) on ``grid`` (a grid
    description), with no context or episode and nothing allocated, here or
    in the library. ``gU``, if given, is the caller's triple (same shapes and
    dtype) that receives dJ/dU. Runs on torch's current stream (or
    ``stream``) and returns ``J``."""
    arrs = list(u) + (list(gU) if gU is not None else [])
    if len(u) != 3 or (gU is not None and len(gU) != 3):
        raise ValueError("u and gU are face triples (three tensors each)")
    if not all(isinstance(t, torch.Tensor) and t.is_cuda and t.is_contiguous() for t in arrs):
        raise TypeError("u and gU must be contiguous CUDA tensors")
    g = grid_struct(grid)
    # the kernel indexes the arrays by the grid's face shapes: a tensor of
    # another shape, dtype or device would be read or written out of bounds
    shapes = [(g.nz, g.ny, g.nx + 1), (g.nz, g.ny + 1, g.nx), (g.nz + 1, g.ny, g.nx)]
    dev = u[0].device
    for d in range(3):
        if tuple(u[d].shape) != shapes[d]:
            raise ValueError(f"u[{d}] has shape {tuple(u[d].shape)}, the grid's face "
                             f"component {d} is {shapes[d]}")
        if gU is not None and (tuple(gU[d].shape) != shapes[d] or gU[d].dtype != u[d].dtype):
            raise ValueError(f"gU[{d}] must match u[{d}] in shape and dtype")
    if not all(t.device == dev for t in arrs):
        raise ValueError("u and gU must be on one device")
    p, code, _, keep = _ptrs(u)
    pg = _ptrs(gU)[0] if gU is not None else None
    with torch.cuda.device(dev):
        if stream is None:
            stream = torch.cuda.current_stream(dev).cuda_stream or L.CUDA_STREAM_LEGACY
        J = C.c_double()
        _check(lib.nf_loss_noalloc(C.byref(g), L.LOSS[kind], p, pg, code, C.byref(J), stream),
               C.c_void_p())
    return J.value


def _config(precision="mixed", solver="mgpcg", tol=1e-6, max_iters=500,
            inner_tol=1e-3, mg_smooth=2, mg_coarsest=4, advect_order=2,
            checkpoint_every=10, hbm_budget=0, cfl_max=0.0, mg_coarsest_sweeps=8,
            mg_band_sweeps=0, mg_transfer="constant", mg_coarse_weight=1.9,
            mg_smooth_coarse=0, tape_fractions=False, mg_persistent=False,
            mg_cluster=False, residual_fp64=True, mg_fused=0, recompute_overlap=True, device=0,
            stream=0):
    """An ``nf_config`` from keyword arguments (defaults of nf_config_default)."""
    cfg = L.Config()
    _check(lib.nf_config_default(C.byref(cfg)))
    cfg.device = device
    cfg.stream = stream
    cfg.precision = L.PREC[precision]
    cfg.solver = L.SOLVER[solver]
    cfg.tol = tol
    cfg.max_iters = max_iters
    cfg.inner_tol = inner_tol
    cfg.mg_smooth = mg_smooth
    cfg.mg_coarsest = mg_coarsest
    cfg.advect_order = advect_order
    cfg.checkpoint_every = checkpoint_every
    cfg.hbm_budget = int(hbm_budget)
    cfg.cfl_max = float(cfl_max)
    cfg.mg_coarsest_sweeps = int(mg_coarsest_sweeps)
    cfg.mg_band_sweeps = int(mg_band_sweeps)
    cfg.mg_transfer = {"trilinear": 0, "constant": 1}[mg_transfer]
    cfg.mg_coarse_weight = float(mg_coarse_weight)
    cfg.mg_smooth_coarse = int(mg_smooth_coarse)
    cfg.tape_fractions = int(bool(tape_fractions))
    cfg.mg_persistent = int(bool(mg_persistent))
    cfg.mg_cluster = int(bool(mg_cluster))
    cfg.residual_fp64 = int(bool(residual_fp64))
    cfg.mg_fused = int(mg_fused)
    cfg.recompute_overlap = int(bool(recompute_overlap))
    return cfg


class Context:
    """An ``nf_ctx``: one device, one stream, one precision/solver setting."""

    def __init__(self, precision="mixed", solver="mgpcg", device=0, stream=None, **kw):
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
            if not stream:
                stream = L.CUDA_STREAM_LEGACY
        cfg = _config(precision=precision, solver=solver, device=device, stream=stream, **kw)
        self.precision = precision
        self.device = device
        self.config = cfg  # the nf_config the context was created with
        self._h = C.c_void_p()
        _check(lib.nf_create(C.byref(self._h), C.byref(cfg)))
        self.field_dtype = torch.float64 if precision == "fp64" else torch.float32

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            lib.nf_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        _check(lib.nf_synchronize(self._h), self._h)

    def dot(self, a, b):
        """``nf_dot``: <a, b> of two CUDA tensors of one dtype by the solver's
        dot arithmetic (a diagnostic of the CG inner products)."""
        if not (a.is_cuda and b.is_cuda and a.is_contiguous() and b.is_contiguous()
                and a.dtype == b.dtype and a.numel() == b.numel()
                and a.dtype in (torch.float32, torch.float64)):
            raise ValueError("a and b must be contiguous CUDA tensors of one float dtype and size")
        out = C.c_double()
        code = L.NF_F64 if a.dtype == torch.float64 else L.NF_F32
        _check(lib.nf_dot(self._h, a.data_ptr(), b.data_ptr(), a.numel(), code, C.byref(out)),
               self._h)
        return out.value

    def check_conversions(self, values):
        """``nf_check_conversions``: the library's integer-bit FP64 -> FP32
        rounding and FP32 -> FP64 widening on the device, beside the
        conversion instructions. Returns (rounded float32 array, widened
        float64 array, number of mismatching entries)."""
        v = np.ascontiguousarray(np.asarray(values, dtype=np.float64))
        n = v.size
        out_f = np.empty(n, np.float32)
        out_d = np.empty(n, np.float64)
        m = C.c_int64()
        _check(lib.nf_check_conversions(self._h, v.ctypes.data, n, out_f.ctypes.data,
                                        out_d.ctypes.data, C.byref(m)), self._h)
        return out_f, out_d, m.value

    def launches(self):
        n = C.c_int64()
        _check(lib.nf_launch_count(self._h, C.byref(n)), self._h)
        return n.value

    def profile(self, kclass):
        """Time launches of one kernel class (name), 'all', or None to stop."""
        code = -2 if kclass is None else (-1 if kclass == "all" else L.KCLASS.index(kclass))
        _check(lib.nf_profile(self._h, code), self._h)

    def profile_read(self, kclass):
        """(launches, device ms) of a kernel class since :meth:`profile`."""
        n, ms = C.c_int64(), C.c_double()
        _check(lib.nf_profile_read(self._h, L.KCLASS.index(kclass), C.byref(n), C.byref(ms)), self._h)
        return n.value, ms.value

    def episode(self, grid_desc, scene):
        return Episode(self, grid_desc, scene)

    def step_batch(self, episodes, frames=1):
        """``nf_step_batch``: advance same-size episodes of this context
        together, each substep's projections solved as one stacked system;
        returns each member's statistics with its ``status``."""
        n = len(episodes)
        ids = (C.c_int64 * n)(*[e.id for e in episodes])
        st = (L.StepStats * n)()
        stat = (C.c_int * n)()
        rc = lib.nf_step_batch(self._h, ids, n, int(frames), st, stat)
        if rc in (L.NF_E_INVALID, L.NF_E_CUDA, L.NF_E_OOM):
            _check(rc, self._h)
        return [dict(x.as_dict(), status=int(c)) for x, c in zip(st, stat)]


class Episode:
    """One simulated grid (``nf_episode_*``)."""

    def __init__(self, ctx: Context, grid_desc, scene):
        self.ctx = ctx
        self.id = None
        self.grid = dict(grid_desc)
        self.scene = dict(scene)
        g = grid_struct(grid_desc)
        s, keep = scene_struct(scene)
        self.K = s.K
        eid = C.c_int64()
        _check(lib.nf_episode_create(ctx.handle, C.byref(g), C.byref(s), C.byref(eid)), ctx.handle)
        self.id = eid.value
        nx, ny, nz = g.nx, g.ny, g.nz
        self.face_shapes = [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)]
        self.cell_shape = (nz, ny, nx)

    def close(self):
        if self.id is not None and self.ctx.handle:
            lib.nf_episode_destroy(self.ctx.handle, self.id)
        self.id = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def _c(self):
        return self.ctx.handle

    def bytes(self):
        b = C.c_size_t()
        _check(lib.nf_episode_bytes(self._c, self.id, C.byref(b)), self._c)
        return b.value

    def set_params(self, theta):
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64))
        _check(lib.nf_set_params(self._c, self.id, th.ctypes.data_as(C.POINTER(C.c_double)), len(th)), self._c)
        self.scene["theta"] = list(th)

    def set_velocity(self, u, project=False):
        p, code, mem, keep = _ptrs(u)
        st = L.StepStats()
        _check(lib.nf_set_velocity(self._c, self.id, p, code, mem, int(bool(project)), C.byref(st)), self._c)
        return st.as_dict()

    def step(self, n=1):
        st = L.StepStats()
        _check(lib.nf_step(self._c, self.id, int(n), C.byref(st)), self._c)
        return st.as_dict()

    def _faces_out(self, dtype, host):
        if host:
            npdt = np.float64 if dtype == torch.float64 else np.float32
            return [np.empty(s, dtype=npdt) for s in self.face_shapes]
        return [torch.empty(s, dtype=dtype, device=f"cuda:{self.ctx.device}") for s in self.face_shapes]

    def loss(self, kind, want_grad=False, dtype=None):
        J = C.c_double()
        if want_grad:
            gU = self._faces_out(dtype or self.ctx.field_dtype, host=False)
            p, code, mem, _ = _ptrs(gU)
            _check(lib.nf_loss(self._c, self.id, L.LOSS[kind], C.byref(J), p, code, mem), self._c)
            return J.value, gU
        _check(lib.nf_loss(self._c, self.id, L.LOSS[kind], C.byref(J), None, L.NF_F32,
                           L.NF_MEM_DEVICE), self._c)
        return J.value

    def backward(self, gU_final, want_gU0=True, host=False):
        """BPTT through the recorded rollout: (dJ/dtheta, dJ/dU^0, stats)."""
        p, code, mem, keep = _ptrs(gU_final)
        dtype = torch.float64 if code == L.NF_F64 else torch.float32
        out, po = None, None
        if want_gU0:
            out = self._faces_out(dtype, host or mem == L.NF_MEM_HOST)
            po, ocode, omem, okeep = _ptrs(out)
            if ocode != code or omem != mem:
                raise ValueError("gradient input and output must share dtype and memory kind")
        gth = (C.c_double * max(1, self.K))()
        st = L.StepStats()
        _check(lib.nf_backward(self._c, self.id, p, po, code, mem, gth, C.byref(st)), self._c)
        return np.array(gth[:self.K]), out, st.as_dict()

    def backward_step(self, gU_next):
        """Revert one step: (dJ/dU^n, this step's dJ/dtheta, stats)."""
        p, code, mem, keep = _ptrs(gU_next)
        dtype = torch.float64 if code == L.NF_F64 else torch.float32
        out = self._faces_out(dtype, mem == L.NF_MEM_HOST)
        po, *_ = _ptrs(out)
        gth = (C.c_double * max(1, self.K))()
        st = L.StepStats()
        _check(lib.nf_backward_step(self._c, self.id, p, po, code, mem, gth, C.byref(st)), self._c)
        return out, np.array(gth[:self.K]), st.as_dict()

    def _get_faces(self, fn, dtype, host):
        out = self._faces_out(dtype, host)
        p, code, mem, _ = _ptrs(out)
        _check(fn(self._c, self.id, p, code, mem), self._c)
        return out

    def velocity(self, dtype=torch.float64, host=False):
        return self._get_faces(lib.nf_get_velocity, dtype, host)

    def advected(self, dtype=torch.float64, host=False):
        return self._get_faces(lib.nf_get_advected, dtype, host)

    def fractions(self, dtype=torch.float64, host=False):
        return self._get_faces(lib.nf_get_fractions, dtype, host)

    def pressure(self, dtype=torch.float64, host=False):
        code = L.NF_F64 if dtype == torch.float64 else L.NF_F32
        if host:
            out = np.empty(self.cell_shape, dtype=np.float64 if dtype == torch.float64 else np.float32)
            ptr, mem = out.ctypes.data, L.NF_MEM_HOST
        else:
            out = torch.empty(self.cell_shape, dtype=dtype, device=f"cuda:{self.ctx.device}")
            ptr, mem = out.data_ptr(), L.NF_MEM_DEVICE
        _check(lib.nf_get_pressure(self._c, self.id, ptr, code, mem), self._c)
        return out

    def export_state(self):
        """``nf_episode_export``: the resumable state as bytes."""
        n = C.c_size_t()
        _check(lib.nf_episode_export(self._c, self.id, None, C.byref(n)), self._c)
        buf = C.create_string_buffer(n.value)
        _check(lib.nf_episode_export(self._c, self.id, buf, C.byref(n)), self._c)
        return buf.raw[:n.value]

    def import_state(self, state):
        """``nf_episode_import``: continue from bytes of :meth:`export_state`."""
        data = bytes(state)
        _check(lib.nf_episode_import(self._c, self.id, data, len(data)), self._c)

    def step_index(self):
        n = C.c_int()
        _check(lib.nf_get_step(self._c, self.id, C.byref(n)), self._c)
        return n.value


class Server:
    """``nf_server``: continuous batching of many episodes over ``slots``
    concurrent worker streams, admitted under ``hbm_budget`` bytes.

    Episodes are named by client keys. ``open`` / ``step`` / ``close`` queue
    requests and return tickets; ``poll`` returns a result dict (or None on
    timeout). Keyword arguments configure every episode like ``Context``.
    """

    def __init__(self, slots=4, hbm_budget=0, device=0, batch=1, batch_cells=64 ** 3, **cfg_kw):
        cfg = _config(device=device, stream=0, **cfg_kw)
        h = C.c_void_p()
        _check(lib.nf_server_create(C.byref(cfg), int(slots), int(hbm_budget), C.byref(h)),
               C.c_void_p())
        self._h = h
        self._keep = {}
        _check(lib.nf_server_set_batching(h, int(batch), int(batch_cells)), C.c_void_p())

    def _submit(self, req):
        t = C.c_int64()
        _check(lib.nf_server_submit(self._h, C.byref(req), C.byref(t)), C.c_void_p())
        return t.value

    def open(self, key, grid_desc, scene):
        req = L.Request()
        req.kind = L.REQ["open"]
        req.episode = int(key)
        req.grid = grid_struct(grid_desc)
        sc, keep = scene_struct(scene)
        req.scene = sc
        t = self._submit(req)       # the server copies the sphere list
        del keep
        return t

    def step(self, key, frames=1, adjoint=False, loss="outflow"):
        req = L.Request()
        req.kind = L.REQ["step_adjoint" if adjoint else "step"]
        req.episode = int(key)
        req.frames = int(frames)
        req.loss_kind = L.LOSS[loss]
        return self._submit(req)

    def close(self, key):
        req = L.Request()
        req.kind = L.REQ["close"]
        req.episode = int(key)
        return self._submit(req)

    def cancel(self, key):
        """NF_REQ_CANCEL: the episode's requests that have not started
        complete with NF_E_CANCELED, then it closes."""
        req = L.Request()
        req.kind = L.REQ["cancel"]
        req.episode = int(key)
        return self._submit(req)

    def poll(self, ticket, wait_ms=-1):
        r = L.Result()
        st = lib.nf_server_poll(self._h, int(ticket), int(wait_ms), C.byref(r))
        if st == L.NF_E_TIMEOUT:
            return None
        _check(st, C.c_void_p())
        return dict(status=r.status, kind=r.kind, episode=r.episode, loss=r.loss,
                    g_theta=np.array(r.g_theta[:]), fwd=r.fwd.as_dict(), bwd=r.bwd.as_dict(),
                    submit_ms=r.submit_ms, start_ms=r.start_ms, end_ms=r.end_ms,
                    episode_bytes=r.episode_bytes)

    def drain(self, wait_ms=-1):
        st = lib.nf_server_drain(self._h, int(wait_ms))
        return st == L.NF_OK

    def stats(self):
        s = L.ServerStats()
        _check(lib.nf_server_stats_get(self._h, C.byref(s)), C.c_void_p())
        return {k: getattr(s, k) for k, _ in s._fields_}

    def close_server(self):
        if self._h:
            lib.nf_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close_server()
        except Exception:
            pass
