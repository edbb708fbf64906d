"""ctypes declarations of the libnf C ABI (``include/nf.h``).

Argument marshalling only: every step of the method runs in the CUDA
library. Importing this module loads ``libnf.so`` from the package directory
and raises ``ImportError`` if it is missing (there is no fallback).
"""

from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnf.so")

NF_OK, NF_E_INVALID, NF_E_OOM, NF_E_NOT_CONVERGED = 0, 1, 2, 3
NF_E_DIVERGED, NF_E_TIMEOUT, NF_E_CUDA, NF_E_STATE = 4, 5, 6, 7
NF_E_CANCELED = 8
PREC = {"fp64": 0, "fp32": 1, "mixed": 2}
SOLVER = {"cg": 0, "mgpcg": 1}
NF_F32, NF_F64 = 0, 1
NF_MEM_DEVICE, NF_MEM_HOST = 0, 1
SCENE = {"none": 0, "sphere": 1, "chamber": 2, "plate": 3, "spheres": 4, "extruded": 5}
LOSS = {"kinetic_energy": 0, "outflow": 1}
FRACTIONS = {"supersample": 0, "corner": 1}
MAX_PARAMS = 8
CUDA_STREAM_LEGACY = 1   # cudaStreamLegacy: the legacy default stream

KCLASS = ["rasterize", "advect", "rhs", "update", "loss", "adj_gp", "adj_face",
          "adj_advect", "residual64", "axpy64", "cg_init", "apply_dot", "cg_xr",
          "cg_rz", "cg_d", "mg_coarsen", "mg_smooth", "mg_residual", "mg_restrict",
          "mg_prolong", "mg_chain", "cast", "mg_smooth0", "gauge", "mg_mid",
          "viscosity"]


class Config(C.Structure):
    _fields_ = [("device", C.c_int), ("stream", C.c_void_p),
                ("precision", C.c_int), ("solver", C.c_int),
                ("tol", C.c_double), ("max_iters", C.c_int),
                ("inner_tol", C.c_double), ("mg_smooth", C.c_int),
                ("mg_coarsest", C.c_int), ("advect_order", C.c_int),
                ("checkpoint_every", C.c_int), ("hbm_budget", C.c_size_t),
                ("cfl_max", C.c_double), ("mg_coarsest_sweeps", C.c_int),
                ("mg_band_sweeps", C.c_int), ("mg_transfer", C.c_int),
                ("mg_coarse_weight", C.c_double), ("mg_smooth_coarse", C.c_int),
                ("tape_fractions", C.c_int), ("mg_persistent", C.c_int),
                ("mg_cluster", C.c_int), ("residual_fp64", C.c_int), ("mg_fused", C.c_int),
                ("recompute_overlap", C.c_int)]


class Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dx", C.c_double), ("dt", C.c_double), ("rho", C.c_double),
                ("outlet", C.c_int), ("outlet_j0", C.c_int),
                ("outlet_k0", C.c_int), ("outlet_w", C.c_int),
                ("outlet_h", C.c_int), ("nu", C.c_double), ("fractions", C.c_int),
                ("inlet", C.c_int), ("inlet_side", C.c_int), ("inlet_j0", C.c_int),
                ("inlet_k0", C.c_int), ("inlet_w", C.c_int), ("inlet_h", C.c_int),
                ("inlet_speed", C.c_double)]


class Scene(C.Structure):
    _fields_ = [("kind", C.c_int), ("K", C.c_int),
                ("theta", C.c_double * MAX_PARAMS),
                ("consts", C.c_double * 16),
                ("spheres", C.POINTER(C.c_double)), ("nspheres", C.c_int),
                ("shapes", C.POINTER(C.c_double)), ("nshape_values", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("steps", C.c_int), ("solves", C.c_int), ("iters", C.c_int),
                ("max_iters", C.c_int), ("outer", C.c_int),
                ("rel_residual", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Request(C.Structure):
    _fields_ = [("kind", C.c_int), ("episode", C.c_int64), ("grid", Grid),
                ("scene", Scene), ("frames", C.c_int), ("loss_kind", C.c_int)]


class Result(C.Structure):
    _fields_ = [("status", C.c_int), ("kind", C.c_int), ("episode", C.c_int64),
                ("loss", C.c_double), ("g_theta", C.c_double * MAX_PARAMS),
                ("fwd", StepStats), ("bwd", StepStats),
                ("submit_ms", C.c_double), ("start_ms", C.c_double),
                ("end_ms", C.c_double), ("episode_bytes", C.c_size_t)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64),
                ("open_waiting", C.c_int64), ("episodes", C.c_int64),
                ("bytes_reserved", C.c_size_t), ("bytes_peak", C.c_size_t),
                ("budget", C.c_size_t), ("slots", C.c_int),
                ("batches", C.c_int64), ("batched_requests", C.c_int64)]


REQ = {"open": 0, "step": 1, "step_adjoint": 2, "close": 3, "cancel": 4}

P3 = C.c_void_p * 3          # a (x, y, z) triple of array pointers
PP = C.POINTER(C.c_void_p)   # how a triple (or NULL) is passed
_vp = C.c_void_p
_i64 = C.c_int64
_ip = C.POINTER(C.c_int)

# (name, restype, argtypes)
SIGNATURES = [
    ("nf_config_default", C.c_int, [C.POINTER(Config)]),
    ("nf_create", C.c_int, [C.POINTER(_vp), C.POINTER(Config)]),
    ("nf_destroy", C.c_int, [_vp]),
    ("nf_last_error", C.c_char_p, [_vp]),
    ("nf_status_string", C.c_char_p, [C.c_int]),
    ("nf_synchronize", C.c_int, [_vp]),
    ("nf_episode_create", C.c_int, [_vp, C.POINTER(Grid), C.POINTER(Scene), C.POINTER(_i64)]),
    ("nf_episode_destroy", C.c_int, [_vp, _i64]),
    ("nf_episode_bytes", C.c_int, [_vp, _i64, C.POINTER(C.c_size_t)]),
    ("nf_set_params", C.c_int, [_vp, _i64, C.POINTER(C.c_double), C.c_int]),
    ("nf_set_velocity", C.c_int, [_vp, _i64, PP, C.c_int, C.c_int, C.c_int, C.POINTER(StepStats)]),
    ("nf_step", C.c_int, [_vp, _i64, C.c_int, C.POINTER(StepStats)]),
    ("nf_loss", C.c_int, [_vp, _i64, C.c_int, C.POINTER(C.c_double), PP, C.c_int, C.c_int]),
    ("nf_loss_noalloc", C.c_int, [C.POINTER(Grid), C.c_int, PP, PP, C.c_int,
                                  C.POINTER(C.c_double), _vp]),
    ("nf_backward_step", C.c_int, [_vp, _i64, PP, PP, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(StepStats)]),
    ("nf_backward", C.c_int, [_vp, _i64, PP, PP, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(StepStats)]),
    ("nf_get_velocity", C.c_int, [_vp, _i64, PP, C.c_int, C.c_int]),
    ("nf_get_pressure", C.c_int, [_vp, _i64, _vp, C.c_int, C.c_int]),
    ("nf_get_fractions", C.c_int, [_vp, _i64, PP, C.c_int, C.c_int]),
    ("nf_get_advected", C.c_int, [_vp, _i64, PP, C.c_int, C.c_int]),
    ("nf_get_step", C.c_int, [_vp, _i64, _ip]),
    ("nf_episode_export", C.c_int, [_vp, _i64, _vp, C.POINTER(C.c_size_t)]),
    ("nf_episode_import", C.c_int, [_vp, _i64, _vp, C.c_size_t]),
    ("nf_dot", C.c_int, [_vp, _vp, _vp, _i64, C.c_int, C.POINTER(C.c_double)]),
    ("nf_check_conversions", C.c_int, [_vp, _vp, _i64, _vp, _vp, C.POINTER(_i64)]),
    ("nf_launch_count", C.c_int, [_vp, C.POINTER(_i64)]),
    ("nf_profile", C.c_int, [_vp, C.c_int]),
    ("nf_profile_read", C.c_int, [_vp, C.c_int, C.POINTER(_i64), C.POINTER(C.c_double)]),
    ("nf_server_create", C.c_int, [C.POINTER(Config), C.c_int, C.c_size_t, C.POINTER(_vp)]),
    ("nf_server_submit", C.c_int, [_vp, C.POINTER(Request), C.POINTER(_i64)]),
    ("nf_server_poll", C.c_int, [_vp, _i64, C.c_int, C.POINTER(Result)]),
    ("nf_server_drain", C.c_int, [_vp, C.c_int]),
    ("nf_server_stats_get", C.c_int, [_vp, C.POINTER(ServerStats)]),
    ("nf_server_destroy", C.c_int, [_vp]),
    ("nf_server_set_batching", C.c_int, [_vp, C.c_int, _i64]),
    ("nf_step_batch", C.c_int, [_vp, C.POINTER(_i64), C.c_int, C.c_int, C.POINTER(StepStats),
                                C.POINTER(C.c_int)]),
]


def load(path=LIB_PATH):
    if not os.path.exists(path):
        raise ImportError(
            f"libnf.so not found at {path}: build it with "
            "`python paper_2405_14903_b300/build.py` (no CPU fallback exists)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


lib = load()
