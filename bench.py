#!/usr/bin/env python
"""Throughput of the differentiable rollout: cell-steps/s of forward + adjoint.

Workload (one bench step): the pulsing chamber of 128^3 cells with a 16 x 16
outlet patch, 100 time steps of dt = 0.005 (RK2 advection, rasterisation,
MIXED MGPCG projection to relative residual 1e-6), the outflow loss, and the
full adjoint with checkpoints every 10 steps (segments recomputed). value =
128^3 * 100 / seconds per bench step.

Also reported: the end-to-end figure through the public API with host
buffers (``e2e``), the same GPU's plain FP64 CG and FP64 MGPCG paths on a
shorter rollout of the same scene, the roofline of the dominant kernel, the
FP64 CPU oracle on a bounded sample (``cpu_baseline``), and the SM clocks
sampled during the timed region.

``--impl reference`` times the FP64 CPU oracle itself on bounded samples of
the same workload (there is no other reference implementation).

Launch: ``python bench.py [--gpus N] [--steps K] [--warmup W]``; for N > 1
under torchrun every rank runs an independent replica (weak scaling).
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import nf_inputs as I  # noqa: E402

METRIC = "cell-steps/s fwd+adjoint at 128^3 (rel res <= 1e-6)"
UNIT = "cell-steps/s"
HBM_FALLBACK = 6400.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=128)
    ap.add_argument("--rollout", type=int, default=100)
    ap.add_argument("--plain-rollout", type=int, default=10)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip FP64 comparison paths, e2e and the CPU baseline")
    ap.add_argument("--tol", type=float, default=1e-6,
                    help="relative residual of every projection (the metric's 1e-6)")
    ap.add_argument("--inner-tol", type=float, default=1e-3,
                    help="relative tolerance of each FP32 inner solve (MIXED refinement)")
    ap.add_argument("--mg-smooth", type=int, default=2,
                    help="red-black Gauss-Seidel sweeps before and after each coarse correction")
    ap.add_argument("--coarsest-sweeps", type=int, default=8,
                    help="symmetric sweep pairs on the coarsest multigrid level")
    ap.add_argument("--band-sweeps", type=int, default=0,
                    help="extra sweeps on the finest level's boundary band")
    ap.add_argument("--mg-transfer", default="constant", choices=["trilinear", "constant"],
                    help="multigrid prolongation and restriction")
    ap.add_argument("--mg-smooth-coarse", type=int, default=0,
                    help="sweeps on the coarse levels (0: as --mg-smooth)")
    ap.add_argument("--tape-fractions", type=int, default=1,
                    help="1: the tape keeps each step's fractions (no re-rasterising)")
    ap.add_argument("--coarse-weight", type=float, default=1.9,
                    help="scale of the coarse-grid correction")
    ap.add_argument("--mg-cluster", type=int, default=0,
                    help="1: coarse levels above an 8^3 local chain on one thread-block cluster")
    ap.add_argument("--residual-fp64", type=int, default=1,
                    help="1: MIXED refinement residual in FP64 arithmetic (0: split-float)")
    ap.add_argument("--mg-fused", type=int, default=0,
                    help="1: finest-level red-black pairs as one shared-memory launch; "
                         "2: every grid level; 0: one launch per half sweep")
    ap.add_argument("--mg-persistent", type=int, default=0,
                    help="1: coarse levels <= 64^3 and the chain in one cooperative kernel")
    ap.add_argument("--mg-coarsest", type=int, default=4,
                    help="stop coarsening at this many cells per edge")
    ap.add_argument("--nu", type=float, default=0.0,
                    help="kinematic viscosity of the chamber (0: the inviscid metric); "
                         "nu > 0 adds explicit viscosity to every step and its adjoint")
    ap.add_argument("--fractions", default="supersample", choices=["supersample", "corner"],
                    help="face fractions: 4x4x4 ramp subsamples of the face's control volume, "
                         "or the face area from the corner values")
    ap.add_argument("--workload", default="rollout", choices=["rollout", "serving", "precision"],
                    help="rollout: the chamber fwd+adjoint metric; serving: the episode mix")
    ap.add_argument("--serve-count", type=int, default=512, help="episodes in the serving mix")
    ap.add_argument("--serve-rate", type=float, default=0.03,
                    help="Poisson arrival rate of episodes (per ms)")
    ap.add_argument("--serve-requests", type=int, default=2,
                    help="step requests per episode (one frame each)")
    ap.add_argument("--serve-slots", type=int, default=8, help="concurrent worker slots")
    ap.add_argument("--serve-batch", type=int, default=1,
                    help="most same-size episodes stepped as one batch (1: no batching)")
    ap.add_argument("--serve-summary-count", type=int, default=48,
                    help="episodes of the compact serving run in the default bench line")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0, help="admission budget")
    ap.add_argument("--cpu-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-n", type=int, default=64,
                    help="grid of the bounded CPU oracle sample")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK, "fallback"


# ---------------------------------------------------------------- clocks ----

class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------- workloads ----

def chamber(n, steps, seed):
    return I.config_chamber(n, steps=steps, seed=seed, duct_half_cells=max(2, 8 * n // 128))


# Algorithmic bytes per cell of the kernels the roofline may name (FP32
# fields, FP32 fractions on the finest level): what the operation must move.
def alg_bytes_per_cell(kclass, nu):
    if kclass == "mg_smooth0":
        # the method's bytes for one full red-black sweep of the finest level:
        # x read, b read, the three fraction arrays read, x written, each once
        # = 24 B/cell; a launch is a half sweep, so 12 B/cell. (Split into two
        # launches, each half sweep reads every fraction and x of the other
        # colour again: 17.8 B/cell on average over a V-cycle, which is what
        # the kernel moves; the difference is charged to the kernel.)
        return (4 + 4 + 3 * 4 + 4) / 2
    return {
        "apply_dot": 4 + 3 * 4 + 4,            # d, three fraction arrays, q
        "cg_xr": 4 * 4 + 2 * 4,                # x, r, d, q read; x, r written
        "residual64": 8 + 8 + 3 * 4 + 8 + 4,   # b, x (FP64), fractions, r64, r32
    }.get(kclass)


# DRAM bytes per cell of one launch (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture, divided by the level's cells),
# for kernels unchanged since their capture; None otherwise. mg_smooth0: the
# V-cycle's mix of the three half-sweep modes (zero start 26.39 MB, six plain
# 34.78 MB, prolongation folded 35.83 MB; writes stay in L2) at 128^3,
# profiles/k_mg_smooth_chamber128.md.
# viscosity: 25.38 MB read + 0.07 MB written per launch (its output stays in
# L2), profiles/k_viscosity_chamber128.md.
DRAM_BYTES_PER_CELL = {"mg_smooth0": (26.39 + 6 * 34.78 + 35.83) * 1e6 / 8 / 128 ** 3,
                       "viscosity": (25.377792 + 0.066304) * 1e6 / 128 ** 3}


# ------------------------------------------------------ ranks (replicas) ----
# Every rank runs its own episode: no data-path collective. The only
# collectives are the barriers around the timed region and one MAX
# all-reduce of the timed milliseconds.

def ranks_from_env(env=None):
    """(world, rank, local_rank) as torchrun sets them (1, 0, 0 alone)."""
    env = os.environ if env is None else env
    return (int(env.get("WORLD_SIZE", "1")), int(env.get("RANK", "0")),
            int(env.get("LOCAL_RANK", "0")))


def max_over_ranks(ms, world, device="cpu"):
    """The slowest rank's timed milliseconds (the job ends with it)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world, cells, frames, ms_per_step):
    """Cell-steps/s of the whole job: every rank advances cells x frames."""
    return world * cells * frames / (ms_per_step / 1e3)


def run_ours(args, rank, world, local_rank):
    import torch
    torch.cuda.set_device(local_rank)
    import paper_2405_14903_b300 as P
    dev = f"cuda:{local_rank}"
    n, T = args.n, args.rollout
    cfg = chamber(n, T, seed=rank)
    cfg["grid"]["nu"] = float(args.nu)
    cfg["grid"]["fractions"] = args.fractions
    ncell = n ** 3

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    ctx = P.Context("mixed", "mgpcg", tol=args.tol, max_iters=1000, checkpoint_every=10,
                    cfl_max=cfg["cfl_max"], inner_tol=args.inner_tol,
                    mg_smooth=args.mg_smooth, mg_coarsest_sweeps=args.coarsest_sweeps,
                    mg_coarsest=args.mg_coarsest, mg_band_sweeps=args.band_sweeps,
                    mg_transfer=args.mg_transfer, mg_coarse_weight=args.coarse_weight,
                    mg_smooth_coarse=args.mg_smooth_coarse, tape_fractions=bool(args.tape_fractions),
                    mg_persistent=bool(args.mg_persistent),
                    mg_cluster=bool(args.mg_cluster),
                    residual_fp64=bool(args.residual_fp64), mg_fused=args.mg_fused,
                    device=local_rank)
    ep = ctx.episode(cfg["grid"], cfg["scene"])
    u0 = [torch.zeros(s, dtype=torch.float32, device=dev) for s in ep.face_shapes]
    stats = {}

    def one_step():
        ep.set_velocity(u0, project=False)
        fs = ep.step(T)
        J, gU = ep.loss("outflow", want_grad=True)
        gth, _, bs = ep.backward(gU, want_gU0=False)
        stats["fwd"], stats["bwd"] = fs, bs
        return J, gth

    # warm-up; the first one also times every kernel class to find the
    # dominant kernel of the step
    ctx.profile("all")
    one_step()
    torch.cuda.synchronize(dev)
    shares = {k: ctx.profile_read(k) for k in P._lib.KCLASS}
    ctx.profile(None)
    dominant = max(shares, key=lambda k: shares[k][1])
    for _ in range(max(0, args.warmup - 1)):
        one_step()
    torch.cuda.synchronize(dev)

    # timed region (no profiling events: an event pair around each of the
    # ~10^5 smoother launches of a step would slow the step itself)
    roof_class = dominant if alg_bytes_per_cell(dominant, args.mg_smooth) else "mg_smooth0"
    clocks = Clocks(local_rank) if rank == 0 else None
    launches0 = ctx.launches()
    barrier()
    torch.cuda.synchronize(dev)
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J, gth = one_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    ms = e0.elapsed_time(e1)
    launches = ctx.launches() - launches0
    clk = clocks.stop() if clocks else None
    # the roofline kernel's launches, each bracketed by CUDA events on the
    # library's stream (torch's current stream), over one more step of the
    # same workload right after the timed region
    ctx.profile(roof_class)
    one_step()
    torch.cuda.synchronize(dev)
    nl, kms = ctx.profile_read(roof_class)
    ctx.profile(None)
    visc = None
    if args.nu > 0:
        # the viscosity kernel (forward and adjoint launches) over one more step
        ctx.profile("viscosity")
        one_step()
        torch.cuda.synchronize(dev)
        visc = ctx.profile_read("viscosity")
        ctx.profile(None)

    ms_per_step = max_over_ranks(ms, world, dev) / args.steps
    value = whole_job_value(world, ncell, T, ms_per_step)

    out = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
               warmup=args.warmup, ms_per_step=ms_per_step, higher_is_better=True,
               scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
               config=dict(workload=f"pulsing chamber {n}^3, {T} steps dt=0.005, 16x16 outlet, "
                                    "outflow loss; forward rollout + full adjoint",
                           grid=n, rollout_steps=T, checkpoint_every=10, nu=float(args.nu),
                           fractions=args.fractions,
                           cfl_max=cfg["cfl_max"], substeps_executed=int(stats["fwd"]["steps"]),
                           precision="FP32 MGPCG (V-cycle, CG vectors; BF16 coarse-level "
                                     "fractions), CG dots in FP64 (FP64 products and sums), "
                                     f"FP64 refinement (x, b FP64) to rel res {args.tol:g}, its "
                                     "residual in "
                                     + ("FP64 arithmetic" if args.residual_fp64 else
                                        "split-float arithmetic (48-bit, no FP64 instructions)"),
                           inner_tol=args.inner_tol, mg_smooth=args.mg_smooth,
                           mg_coarsest=args.mg_coarsest, coarsest_sweeps=args.coarsest_sweeps,
                           band_sweeps=args.band_sweeps, mg_transfer=args.mg_transfer,
                           coarse_weight=args.coarse_weight,
                           mg_smooth_coarse=args.mg_smooth_coarse,
                           tape_fractions=bool(args.tape_fractions),
                           mg_persistent=bool(args.mg_persistent),
                           mg_cluster=bool(args.mg_cluster),
                           residual_fp64=bool(args.residual_fp64),
                           mg_fused=args.mg_fused,
                           l2="inputs larger than L2 (episode state and tape > 1 GB)",
                           parallelism=f"replicas x{world}"),
               gpu_launches=int(launches), iterations=dict(fwd=stats["fwd"], bwd=stats["bwd"]),
               loss=J, dJ_dtheta=[float(x) for x in gth], clocks=clk)
    if rank != 0:
        return None

    peak, src = peaks()
    per_launch = alg_bytes_per_cell(roof_class, args.mg_smooth) * ncell
    avg_ms = kms / max(nl, 1)
    achieved = per_launch / (avg_ms / 1e3) / 1e9 if nl else None
    out["roofline"] = dict(bound="hbm", kernel=roof_class, achieved=achieved, peak=peak,
                           peak_source=src, unit="GB/s",
                           frac=(achieved / peak) if achieved else None,
                           # the capture was taken at 128^3 (cold cache under ncu)
                           traffic=(DRAM_BYTES_PER_CELL[roof_class] * ncell
                                    if DRAM_BYTES_PER_CELL.get(roof_class) and n == 128
                                    and args.mg_smooth == 2 else None),
                           launches=nl, avg_us=1e3 * avg_ms, alg_bytes_per_launch=per_launch,
                           accounting=("24 B/cell per full red-black sweep (x, b, three "
                                       "fractions read, x written), two launches per sweep"
                                       if roof_class == "mg_smooth0" else "per-cell reads "
                                       "and writes of the operation"),
                           timing="CUDA events around every launch of the kernel, over one "
                                  "step of the same workload run right after the timed region")
    if visc is not None and visc[0]:
        # faces of the three components: one read and one write of each
        nfaces = 3 * (n + 1) * n * n
        vb = 2 * 4 * nfaces
        vms = visc[1] / visc[0]
        va = vb / (vms / 1e3) / 1e9
        out["viscosity_roofline"] = dict(
            bound="hbm", kernel="viscosity", achieved=va, peak=peak, peak_source=src,
            unit="GB/s", frac=va / peak,
            traffic=DRAM_BYTES_PER_CELL["viscosity"] * ncell if n == 128 else None,
            launches=visc[0], avg_us=1e3 * vms,
            alg_bytes_per_launch=vb,
            timing="CUDA events around every launch, over one step after the timed region")
    tot = sum(v[1] for v in shares.values()) or 1.0
    out["kernel_shares"] = {k: round(v[1] / tot, 4) for k, v in
                            sorted(shares.items(), key=lambda kv: -kv[1][1]) if v[1] > 0}
    # average launch time per class in the profiled warm-up step (events
    # around each launch)
    out["kernel_avg_us"] = {k: round(1e3 * v[1] / v[0], 2) for k, v in shares.items() if v[0]}
    if not args.no_extras:
        out["e2e"] = run_e2e(args, torch, cfg, dev, ep)
        out["fp64_plain"] = run_plain(args, P, torch, dev, ctx, ep, value)
        out["cpu_baseline"] = cpu_baseline(args)
        out["cpu_baseline"]["all_cores"] = cpu_baseline_all_cores(args)
        out["serving"] = serving_summary(args)
    ep.close()
    ctx.close()
    return out


def run_e2e(args, torch, cfg, dev, ep):
    """The same metric through the public API with pinned host buffers."""
    T = args.rollout
    u_host = [torch.zeros(s, dtype=torch.float32).pin_memory() for s in ep.face_shapes]
    theta = np.asarray(cfg["scene"]["theta"], dtype=np.float64)
    h2d = sum(u.numel() * 4 for u in u_host) + theta.nbytes

    def one():
        ep.set_params(theta)
        ep.set_velocity(u_host, project=False)
        ep.step(T)
        J, gU = ep.loss("outflow", want_grad=True)
        gth, _, _ = ep.backward(gU, want_gU0=False)      # lands in host memory
        return J, gth

    one()
    torch.cuda.synchronize(dev)
    k = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    for _ in range(k):
        J, gth = one()
    torch.cuda.synchronize(dev)
    dt = (time.perf_counter() - t0) / k
    return dict(value=args.n ** 3 * T / dt, unit=UNIT, h2d_bytes_per_step=int(h2d),
                d2h_bytes_per_step=int(8 + gth.nbytes), ms_per_step=1e3 * dt, steps=k)


def _time_rollout(torch, dev, ep, u0, T, warm_T):
    """Milliseconds (CUDA events) of one forward rollout of T frames plus its
    adjoint, after one untimed rollout of warm_T frames; solver stats."""
    def one(frames):
        ep.set_velocity(u0, project=False)
        fs = ep.step(frames)
        J, gU = ep.loss("outflow", want_grad=True)
        gth, _, bs = ep.backward(gU, want_gU0=False)
        return fs, bs

    one(warm_T)
    torch.cuda.synchronize(dev)
    s = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    fs, bs = one(T)
    e1.record(s)
    torch.cuda.synchronize(dev)
    return e0.elapsed_time(e1), fs, bs


def run_plain(args, P, torch, dev, ours_ctx, ours_ep, ours_value):
    """The same GPU's plain FP64 paths on the same scene, like for like.

    FP64 MGPCG runs the metric's own rollout (the same frames, hence the
    same CFL substeps), so ``value / fp64_mgpcg.value`` compares equal work.
    FP64 CG is too slow for the full rollout inside a bench run (about ten
    minutes); it runs the first ``plain_rollout`` frames, and the configured
    MIXED path is timed on those same frames beside it."""
    res = {}
    Tp = args.plain_rollout
    u32 = [torch.zeros(s, dtype=torch.float32, device=dev) for s in ours_ep.face_shapes]
    ms, fs, bs = _time_rollout(torch, dev, ours_ep, u32, Tp, Tp)
    mixed_short = dict(value=args.n ** 3 * Tp / (ms / 1e3), unit=UNIT, rollout_steps=Tp,
                       substeps=int(fs["steps"]), ms_per_rollout=ms,
                       fwd_iters=fs["iters"], bwd_iters=bs["iters"])
    for solver, T in (("mgpcg", args.rollout), ("cg", Tp)):
        cfg = chamber(args.n, T, seed=0)
        ctx = P.Context("fp64", solver, tol=args.tol, max_iters=20000, checkpoint_every=10,
                        cfl_max=cfg["cfl_max"])
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        u0 = [torch.zeros(s, dtype=torch.float64, device=dev) for s in ep.face_shapes]
        ms, fs, bs = _time_rollout(torch, dev, ep, u0, T, 1)
        res[solver] = dict(value=args.n ** 3 * T / (ms / 1e3), unit=UNIT, rollout_steps=T,
                           substeps=int(fs["steps"]), ms_per_rollout=ms,
                           fwd_iters=fs["iters"], bwd_iters=bs["iters"])
        ep.close()
        ctx.close()
    res["mixed_same_frames_as_cg"] = mixed_short
    res["speedup_vs_fp64_mgpcg"] = ours_value / res["mgpcg"]["value"]
    res["speedup_vs_fp64_cg"] = mixed_short["value"] / res["cg"]["value"]
    res["note"] = ("fp64 mgpcg: the metric's full rollout (same frames and substeps as value); "
                   f"fp64 cg: the first {Tp} frames, against MIXED on the same {Tp} frames")
    return res


def _cpu_sample(n):
    """One forward + adjoint step of the chamber scene on n^3 by the oracle."""
    from oracle import Grid
    from oracle import step as S
    cfg = chamber(n, 1, seed=0)
    g = Grid(cfg["grid"])
    t0 = time.perf_counter()
    U, tape = S.step(g, cfg["scene"], cfg["u0"], 0, 1e-6)
    J, gU = S.outflow(g, U)
    S.rollout_backward(g, cfg["scene"], [tape], gU, 1e-6)
    return time.perf_counter() - t0


def cpu_model():
    """The host CPU's model name (from /proc/cpuinfo), or None."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


def cpu_baseline(args):
    """The FP64 oracle on a bounded sample: one forward + adjoint step of the
    same chamber scene on a coarser grid, scaled to cell-steps/s. It runs in
    a child interpreter with BLAS and OpenMP held to one thread, so `cores`
    is what ran."""
    n = args.cpu_n
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    res = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-sample",
                          "--cpu-n", str(n)], env=env, capture_output=True, text=True,
                         timeout=1800)
    if res.returncode != 0:
        raise RuntimeError(f"CPU oracle sample failed: {res.stderr[-2000:]}")
    dt = float(res.stdout.strip().splitlines()[-1])
    return dict(value=n ** 3 / dt, unit=UNIT, cores=1, host_cpus=os.cpu_count(),
                cpu_model=cpu_model(), kind="oracle",
                sample=f"1 step (forward + adjoint) of the same chamber scene on {n}^3 "
                       f"(FP64 NumPy, unpreconditioned CG to 1e-6, one thread), scaled per "
                       f"cell-step; a coarser grid needs fewer CG iterations, so this "
                       f"flatters the oracle",
                seconds=dt)


def cpu_baseline_all_cores(args, procs=None):
    """The same oracle sample run by ``procs`` one-thread interpreters at once
    (default: one per host CPU): independent episodes, as the replicas of the
    GPU run. value = procs x cells / the slowest sample's time."""
    n = args.cpu_n
    P = procs or max(1, os.cpu_count() or 1)
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1",
               MKL_NUM_THREADS="1", NUMEXPR_NUM_THREADS="1")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-sample", "--cpu-n", str(n)]
    t0 = time.perf_counter()
    ps = [subprocess.Popen(cmd, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                           text=True) for _ in range(P)]
    outs = [p.communicate(timeout=1800) for p in ps]
    wall = time.perf_counter() - t0
    for p, (_, err) in zip(ps, outs):
        if p.returncode != 0:
            raise RuntimeError(f"CPU oracle sample failed: {err[-2000:]}")
    dts = [float(o.strip().splitlines()[-1]) for o, _ in outs]
    return dict(value=P * n ** 3 / max(dts), unit=UNIT, cores=P, host_cpus=os.cpu_count(),
                cpu_model=cpu_model(), kind="oracle", seconds=max(dts), wall_seconds=wall,
                sample=f"{P} concurrent one-thread copies of the {n}^3 sample")


# -------------------------------------------------------------- serving ----

def _serve_episode(kind, n, seed):
    """Grid, scene and loss of one episode of the mix (sphere, chamber or plate)."""
    rng = np.random.default_rng(seed)
    if kind == "sphere":
        cfg = I.config_sphere(n)
        v = (0.1 + 0.05 * rng.uniform(-1, 1), 0.05 * rng.uniform(-1, 1), 0.05 * rng.uniform(-1, 1))
        cfg["scene"] = I.sphere_scene(v=v)
        return cfg["grid"], cfg["scene"], "kinetic_energy"
    if kind == "chamber":
        cfg = chamber(n, 100, seed % (1 << 16))
        return cfg["grid"], cfg["scene"], "outflow"
    cfg = I.config_plate(n, seed=seed % (1 << 16))
    return cfg["grid"], cfg["scene"], "kinetic_energy"


def _serve_run(P, plan, slots, budget, batch=8):
    srv = P.Server(slots=slots, hbm_budget=budget, precision="mixed", tol=1e-6,
                   max_iters=1000, cfl_max=8.0, checkpoint_every=10, batch=batch)
    tickets = []
    t0 = time.perf_counter()
    for ep in plan:
        wait = ep["arrival_ms"] / 1e3 - (time.perf_counter() - t0)
        if wait > 0:
            time.sleep(wait)
        ts = [srv.open(ep["key"], ep["grid"], ep["scene"])]
        ts += [srv.step(ep["key"], frames=1, adjoint=a, loss=ep["loss"]) for a in ep["adjoint"]]
        ts.append(srv.close(ep["key"]))
        tickets.append((ep, ts))
    srv.drain()
    wall = time.perf_counter() - t0
    stats = srv.stats()
    lat = {"step": [], "step_adjoint": []}
    cell_frames, failed = 0, 0
    for ep, ts in tickets:
        res = [srv.poll(t) for t in ts]
        failed += sum(1 for r in res if r["status"] not in (0, 3))
        for r, a in zip(res[1:-1], ep["adjoint"]):
            lat["step_adjoint" if a else "step"].append(r["end_ms"] - r["submit_ms"])
            cell_frames += ep["cells"]
    srv.close_server()
    every = lat["step"] + lat["step_adjoint"]
    batches = (int(stats["batches"]), int(stats["batched_requests"]))
    pct = lambda v, q: float(np.percentile(v, q)) if v else None  # noqa: E731
    return dict(value=cell_frames / wall, unit="cell-frames/s", wall_s=wall,
                requests=len(every), failed=failed,
                p50_ms=pct(every, 50), p99_ms=pct(every, 99),
                step_p50_ms=pct(lat["step"], 50), step_p99_ms=pct(lat["step"], 99),
                adjoint_p50_ms=pct(lat["step_adjoint"], 50),
                adjoint_p99_ms=pct(lat["step_adjoint"], 99),
                slots=slots, batch=batch, batches=batches[0], batched_requests=batches[1],
                bytes_peak=int(stats["bytes_peak"]))


def _serve_plan(count, rate, seed=0, requests=2, sizes=(32, 64, 96, 128, 192)):
    mix = I.serving_mix(seed=seed, count=count, rate_per_ms=rate, sizes=sizes)
    rng = np.random.default_rng(12345)
    plan = []
    for key, m in enumerate(mix):
        grid, scene, loss = _serve_episode(m["scene_kind"], m["n"], m["seed"])
        plan.append(dict(key=key, arrival_ms=m["arrival_ms"], grid=grid, scene=scene, loss=loss,
                         cells=m["n"] ** 3,
                         adjoint=[bool(x) for x in rng.uniform(size=requests) < 0.3]))
    return plan


def serving_summary(args):
    """A compact serving run for the default bench line: episodes of the mix
    (grids 32..192^3, three scene kinds, 30 % of one-frame requests with the
    adjoint) arriving faster than the device serves them (saturating), served
    four ways on the same schedule: 8 slots (the default: no cross-episode
    batching), 8 slots with batched steps, one slot with batched steps, one
    episode at a time; for the full size mix and for its small grids (32 and
    64^3) alone."""
    import paper_2405_14903_b300 as P
    budget = int(args.serve_budget_gb * 1e9)
    keys = ("value", "unit", "p50_ms", "p99_ms", "wall_s", "requests", "failed", "batches",
            "batched_requests")
    out = {}
    for mix, sizes in (("mix", (32, 64, 96, 128, 192)), ("small", (32, 64))):
        plan = _serve_plan(args.serve_summary_count, rate=5.0, sizes=sizes)
        res = {}
        for name, slots, batch in (("slots", 8, 1), ("batched", 8, 8), ("batched_one_slot", 1, 8),
                                   ("one_at_a_time", 1, 1)):
            r = _serve_run(P, plan, slots, budget, batch=batch)
            res[name] = {k: r[k] for k in keys}
        res["workload"] = (f"{args.serve_summary_count} episodes arriving at 5/ms (saturating), "
                           f"grids {'/'.join(str(n) for n in sizes)}^3, sphere/chamber/plate, "
                           "2 one-frame requests each, 30 % with adjoint, MIXED MGPCG 1e-6")
        out[mix] = res
    return out


def run_serving(args):
    """Serving mix: Poisson arrivals of episodes (grid sizes 32..192, sphere,
    chamber and plate scenes), each issuing one-frame step requests of which a seeded 30 %
    carry the adjoint, then closing; the same schedule served with `slots`
    concurrent slots and one episode at a time."""
    import torch
    import paper_2405_14903_b300 as P
    torch.cuda.set_device(0)
    plan = _serve_plan(args.serve_count, args.serve_rate, requests=args.serve_requests)
    budget = int(args.serve_budget_gb * 1e9)
    ours = _serve_run(P, plan, args.serve_slots, budget, batch=args.serve_batch)
    unbatched = _serve_run(P, plan, args.serve_slots, budget, batch=1)
    one = _serve_run(P, plan, 1, budget, batch=1)
    return dict(metric="served cell-frames/s, serving mix (p50/p99 request latency)",
                value=ours["value"], unit="cell-frames/s", n_gpus=1, steps=1, warmup=0,
                ms_per_step=1e3 * ours["wall_s"], higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=f"{args.serve_count} episodes, Poisson arrivals at "
                                     f"{args.serve_rate}/ms, grids 32-192^3, sphere/chamber/"
                                     f"plate scenes, {args.serve_requests} one-frame requests "
                                     "per episode, 30 % with adjoint, MIXED MGPCG 1e-6",
                            slots=args.serve_slots, budget_gb=args.serve_budget_gb),
                p50_ms=ours["p50_ms"], p99_ms=ours["p99_ms"], served=ours,
                slots_without_batching=unbatched, one_episode_at_a_time=one)


# ------------------------------------------------------------ precision ----

# kernel classes of the pressure solve (everything but geometry, advection,
# right-hand side, update, labelling and gauge)
SOLVER_CLASSES = ("residual64", "axpy64", "cg_init", "apply_dot", "cg_xr", "cg_rz", "cg_d",
                  "mg_coarsen", "mg_smooth", "mg_residual", "mg_restrict", "mg_prolong",
                  "mg_chain", "mg_smooth0", "mg_mid")


def run_precision(args):
    """Precision sweep: one projection of a divergent N(0, 1) velocity around 64 static
    spheres at 256^3, to relative residual 1e-8, by FP64 MGPCG, FP32 MGPCG and
    MIXED (FP32 CG, BF16-coarse V-cycle, FP64 refinement). The velocity error
    is measured against FP64 MGPCG to 1e-12 (the oracle's unpreconditioned CG
    does not finish at this size; FP64 MGPCG is pinned to it at small sizes)."""
    import torch
    import paper_2405_14903_b300 as P
    torch.cuda.set_device(0)
    n = args.n if args.n != 128 else 256
    cfg = I.config_spheres(n, tol=1e-8)
    u0 = [torch.tensor(x, device="cuda", dtype=torch.float64) for x in cfg["u0"]]

    def project(precision, tol):
        ctx = P.Context(precision, "mgpcg", tol=tol, max_iters=5000)
        ep = ctx.episode(cfg["grid"], cfg["scene"])
        ep.set_velocity(u0, project=False)         # warm the solver (graphs, pools)
        ep.set_velocity(u0, project=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s = torch.cuda.current_stream()
        ctx.profile("all")
        e0.record(s)
        st = ep.set_velocity(u0, project=True)
        e1.record(s)
        torch.cuda.synchronize()
        solve_ms = sum(ctx.profile_read(k)[1] for k in SOLVER_CLASSES)
        ctx.profile(None)
        u = [x.double() for x in ep.velocity(dtype=torch.float64)]
        ep.close()
        ctx.close()
        return dict(st, solve_ms=solve_ms), e0.elapsed_time(e1), u

    st_ref, _, u_ref = project("fp64", 1e-12)
    ref_norm = float(torch.sqrt(sum((x * x).sum() for x in u_ref)))
    ncell = n ** 3
    variants = {}
    for name, prec in (("fp64_mgpcg", "fp64"), ("fp32_mgpcg", "fp32"), ("mixed", "mixed")):
        st, ms, u = project(prec, 1e-8)
        err = float(torch.sqrt(sum(((a - b) ** 2).sum() for a, b in zip(u, u_ref)))) / ref_norm
        vb = 8 if prec == "fp64" else 4
        # algorithmic bytes of one PCG iteration: apply (d, 3 fractions, q),
        # CG updates (x, r, d, q, z) and one V-cycle (4 fine sweeps of 18,
        # residual 20, restrict 4.5, prolong 8, coarse levels x 8/7)
        it_bytes = ncell * (vb * 5 + vb * 2 * 5 + (4 * 18 + 20 + 4.5 + 8) * vb / 4 * 8 / 7)
        variants[name] = dict(iterations=st["iters"], outer=st["outer"],
                              velocity_norm=float(torch.sqrt(sum((x * x).sum() for x in u))),
                              rel_residual=st["rel_residual"], projection_ms=ms,
                              solve_kernel_ms=st["solve_ms"],
                              achieved_gbs=it_bytes * st["iters"] / (st["solve_ms"] / 1e3) / 1e9,
                              velocity_rel_err=err,
                              converged=st["rel_residual"] <= 1e-8)
    return dict(metric="single projection at 256^3 to rel res 1e-8 (64 static spheres)",
                value=variants["mixed"]["solve_kernel_ms"], unit="ms", n_gpus=1, steps=1,
                warmup=1, ms_per_step=variants["mixed"]["projection_ms"], higher_is_better=False,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                config=dict(workload=f"{n}^3, 64 static spheres r in [0.02, 0.08], "
                                     "N(0,1) divergent face velocity, one cut-cell projection",
                            reference="FP64 MGPCG to 1e-12",
                            reference_norm=ref_norm, reference_stats=st_ref),
                variants=variants)


def run_reference(args, rank):
    if rank != 0:
        return None
    K, W = args.steps, args.warmup
    for _ in range(W):
        cpu_baseline(args)
    vals = [cpu_baseline(args) for _ in range(K)]
    v = float(np.mean([x["value"] for x in vals]))
    secs = float(np.mean([x["seconds"] for x in vals]))
    base = vals[-1]
    return dict(metric=METRIC, value=v, unit=UNIT, n_gpus=1, steps=K, warmup=W,
                ms_per_step=1e3 * secs, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic", impl="reference",
                config=dict(workload=f"pulsing chamber, bounded sample: {base['sample']}",
                            grid=args.cpu_n),
                cpu_baseline=dict(value=v, unit=UNIT, cores=base["cores"], kind="oracle",
                                  sample=base["sample"]),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))


def main():
    args = parse()
    if args.cpu_sample:
        print(_cpu_sample(args.cpu_n))
        return
    world, rank, local_rank = ranks_from_env()
    if args.impl == "reference":
        out = run_reference(args, rank)
    elif args.workload == "serving":
        out = run_serving(args) if rank == 0 else None
    elif args.workload == "precision":
        out = run_precision(args) if rank == 0 else None
    else:
        if world > 1:
            import torch
            import torch.distributed as dist
            torch.cuda.set_device(local_rank)
            dist.init_process_group("nccl")
        out = run_ours(args, rank, world, local_rank)
    if out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
