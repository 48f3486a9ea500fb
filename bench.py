#!/usr/bin/env python
"""Benchmark: Gauss-Newton time-to-residual of BL PDE-LDDMM (deformation-state variant,
SL-RK) on a paper-scale synthetic pair, plus SL voxel-steps/s, on one B300 per rank.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

One step = one full registration from a cold start (v~ = 0) of a 192 x 224 x 192 pair:
velocity synthesis, characteristics, state / adjoint / incremental sweeps, projections,
PCG, line search and the stopping test -- every row of the hot path. Inputs are resident
in device memory before timing starts; the e2e figure repeats the step through the public
API with host buffers (host->device images, device->host velocity) inside the timing.

Under torchrun (N > 1) each rank registers its own pair (independent replicas: a pair
does not shard); the value divides the slowest rank's time by all pairs processed.

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same workload
(one band-limited SL-RK step of the deformation state, extrapolated to a registration by
the step count the GPU path performs on this workload).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPE = (192, 224, 192)        # nz, ny, nx
K = 32
NT = 10
MAX_GN, MAX_PCG, GTOL = 10, 20, 1e-3
SIGMA2, ALPHA, S_EXP = 0.01, 0.0025, 2
METRIC = "GN time-to-residual 1e-3 (s/pair) + SL voxel-steps/s, plain FP32 vs chosen form"
WORKLOAD = ("192x224x192 brain-like ellipsoid phantom pair (moving = phantom warped by a "
            "random 32^3-mode stationary velocity, 8 vox max; N(0,0.01) noise), "
            "deformation-state BL PDE-LDDMM, K=32, nt=10, trilinear SL-RK, "
            "alpha=0.0025, s=2, sigma^2=0.01, <=10 GN x <=20 PCG, gtol=1e-3")
# BL steps the GPU path performs in one registration of this workload (solves x nt), as
# reported by lddmm_register on a B300 (74 solves x 10 steps); used only to extrapolate the
# oracle's sample in the reference arm.
REF_STEPS_PER_PAIR = 740

# Kernels bound by FP32 arithmetic: the Y/Z contractions of pi and iota (SIMT complex
# multiply-adds with L2-resident operands) and the network's convolutions. Every other kernel
# streams fields through HBM: the SL sweeps, the element-wise and reduction kernels, and the x
# stages of pi / iota, whose tensor-core contractions move far more bytes than their flops need.
ALU_KERNELS = ("pi_y", "pi_z", "iota_y", "iota_z")


def is_hbm_kernel(name):
    return not (name in ALU_KERNELS or name.startswith("cnn_"))


# Bytes per voxel of the SL kernels as the hot-path table of the survey counts them (state a3
# 20 B; adjoint and BL vector steps 36 B; incremental deformation state a7 84 B), beside the
# library's own algorithmic count (KTRACE): the Heun step of the incremental deformation state
# also gathers the previous right-hand side F_j at the departure point and writes F_{j+1}
# (+12 B each), which the survey's 84 B omit, so the library counts 108 B there.
SURVEY_BYTES_PER_VOXEL = {"sl_gather": 20.0, "sl_gather3_scale": 36.0, "sl_gather3_add": 36.0,
                          "sl_inc_defstate": 84.0}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture of
# the kernel, scaled by voxels to the 192x224x192 launch where the capture ran a smaller grid
# (profiles/k_inc_defstate_128x160x128.md: 263.7 MB at 128x160x128 -> 830.6 MB); kernels
# without a capture of their current code are absent (reported as null).
NCU_TRAFFIC_PER_LAUNCH = {"sl_inc_defstate": 830.6e6}


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))), "measured"
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "sm_max_mhz": 2032.0}, "fallback"


def _fp32_simt_peak_tflops(sm_mhz):
    # 148 SMs x 128 FP32 lanes x 2 flop (FMA) per clock
    return 148 * 128 * 2 * sm_mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def make_inputs(L, torch, dev):
    """Phantom pair on the device (float32 [nz, ny, nx] each) and pinned host copies."""
    import numpy as np
    from paper_2006_06823_b300 import synth
    nz, ny, nx = SHAPE
    fixed = synth.ellipsoid_phantom(SHAPE)
    vt = synth.random_velocity_coeffs(K, K, seed=1)
    vt_d = torch.as_tensor(vt.astype(np.complex64), device=dev)
    v = L.bl_include(vt_d, SHAPE)
    to_vox = torch.tensor([nx, ny, nz], dtype=torch.float32, device=dev).view(3, 1, 1, 1) / (2 * np.pi)
    V = v * to_vox
    V *= 8.0 / V.pow(2).sum(0).sqrt().max()
    fixed_d = torch.as_tensor(fixed, dtype=torch.float32, device=dev)
    moving_d = L.sl_transport(V, fixed_d, NT, L.FORWARD, L.INTERP_LINEAR)
    moving = moving_d.cpu().numpy().astype(np.float64)
    I0 = synth.add_noise(moving, seed=2).astype(np.float32)
    I1 = synth.add_noise(fixed, seed=3).astype(np.float32)
    I0h = torch.from_numpy(I0).pin_memory()
    I1h = torch.from_numpy(I1).pin_memory()
    return I0h.to(dev), I1h.to(dev), I0h, I1h, V, fixed_d


def dist_setup():
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """The largest x over the ranks (the slowest rank's time); a host-only reduction for the
    timing, never on the data path."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_b300(args):
    import torch
    import paper_2006_06823_b300 as L
    world, rank, local = dist_setup()
    dev = torch.device("cuda", local if world > 1 else 0)
    peaks, peak_src = _peaks()
    nz, ny, nx = SHAPE
    I0d, I1d, I0h, I1h, V, fixed_d = make_inputs(L, torch, dev)
    ctx = L.Context(nx, ny, nz, K, nt=NT, variant=L.V_DEFSTATE, interp=L.INTERP_LINEAR,
                    alpha=ALPHA, s=S_EXP, sigma2=SIGMA2, max_gn=MAX_GN, max_pcg=MAX_PCG,
                    gtol=GTOL)
    ctx.set_images(I0d, I1d)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    reports = []
    for _ in range(args.warmup):
        _, rep = ctx.register()
        reports.append(rep)
    torch.cuda.synchronize()

    # ---- timed region: K registrations from a cold start, inputs resident on the device
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    launches0 = L.launch_count()
    step_ms = []
    histories = []
    barrier(world)
    torch.cuda.synchronize()
    for _ in range(args.steps):
        flush.fill_(1.0)                       # evict L2 between steps (outside the timing)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.nvtx.range_push("timed_registration")   # lets a profiler select the step
        e0.record(stream)
        _, rep = ctx.register()
        e1.record(stream)
        e1.synchronize()
        torch.cuda.nvtx.range_pop()
        step_ms.append(e0.elapsed_time(e1))
        reports.append(rep)
        histories.append(ctx.history())       # host-only read of the per-iterate record
    torch.cuda.synchronize()
    barrier(world)
    launches = L.launch_count() - launches0
    clocks = sampler.stop() if sampler else None
    total_s = max_over_ranks(sum(step_ms) / 1e3, world)

    # ---- per-kernel breakdown: one more registration with the library's kernel trace (CUDA
    # events around every launch on its stream), outside the timed region so that the event
    # records do not slow the timed steps
    flush.fill_(1.0)
    torch.cuda.synchronize()
    L.trace_reset()
    L.trace_enable(True)
    v_sol, _ = ctx.register()
    trace = L.trace_read()
    L.trace_enable(False)

    # ---- SL voxel-steps/s: nt-step scalar transport of the phantom (Table 1 row 1). Device
    # rate: REPS transports back to back between two events (the host enqueues ahead; the
    # working set, ~300 MB, exceeds L2); single call: one flushed call, host latency included
    ntot = nx * ny * nz
    sl_out = torch.empty_like(fixed_d)

    def sl_rate(fn, reps=10):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return reps * NT * ntot / (e0.elapsed_time(e1) / 1e3)

    sl_vps = sl_rate(lambda: L.sl_transport(V, fixed_d, NT, L.FORWARD, L.INTERP_LINEAR, out=sl_out))
    sl_ms = []
    for i in range(args.warmup + args.steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        L.sl_transport(V, fixed_d, NT, L.FORWARD, L.INTERP_LINEAR, out=sl_out)
        e1.record(stream)
        e1.synchronize()
        if i >= args.warmup:
            sl_ms.append(e0.elapsed_time(e1))
    sl_vps_call = NT * ntot / (statistics.mean(sl_ms) / 1e3)
    # the BF16-storage forms (separately reported mixed-precision variant of the same sweep)
    sl_bf16 = {"fields_bf16": sl_rate(lambda: L.sl_transport_bf16(V, fixed_d, NT, L.FORWARD, False,
                                                                  out=sl_out)),
               "fields_and_offsets_bf16": sl_rate(lambda: L.sl_transport_bf16(V, fixed_d, NT, L.FORWARD,
                                                                              True, out=sl_out))}

    # ---- e2e: the public API with host buffers, copies inside the timing
    # diagnostics of the solution (Sec. 5.1.1): range of det D phi(1)
    jac_range, _ = ctx.jacobian_det(v_sol)
    max_disp = ctx.max_displacement(v_sol)

    e2e_s = []
    v_host = torch.empty((3, K, K, K), dtype=torch.complex64).pin_memory()
    for _ in range(args.steps):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.set_images(I0h, I1h)
        v, _ = ctx.register()
        v_host.copy_(v, non_blocking=True)
        torch.cuda.synchronize()
        e2e_s.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(sum(e2e_s), world)
    ctx.close()
    # ---- the same pair with the Gauss-Newton cap raised to LONG_GN: where the residual
    # plateaus and when (if ever) it reaches 1e-3 (outside the timed region)
    long_run = measure_long_run(L, torch, I0d, I1d, flush) if args.forms and rank == 0 else None
    forms = measure_forms(L, torch, I0d, I1d, stream, flush) if args.forms and rank == 0 else None
    warm = measure_warm_start(L, torch) if args.forms and rank == 0 else None
    chosen = measure_chosen_form(L, torch) if args.forms and rank == 0 else None
    batched = measure_batched_form(args) if args.forms and rank == 0 else None

    if rank != 0:
        return None
    last = reports[-1]
    per_pair = total_s / (args.steps * world)
    hbm_peak = peaks["hbm_gbs"]
    # dominant kernel by total device time in the timed region
    name, kt = max(trace.items(), key=lambda kv: kv[1]["ms"])
    avg_ms = kt["ms"] / kt["launches"]
    hbm = peaks["hbm_gbs"]
    if is_hbm_kernel(name):
        achieved = kt["bytes"] / kt["launches"] / (avg_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm}
    else:
        achieved = kt["flops"] / kt["launches"] / (avg_ms * 1e-3) / 1e12
        pk = _fp32_simt_peak_tflops(peaks.get("sm_max_mhz", 2032.0))
        roof = {"bound": "alu", "achieved": achieved, "peak": pk, "unit": "TFLOP/s",
                "frac": achieved / pk}
    traffic = NCU_TRAFFIC_PER_LAUNCH.get(name)
    if roof["bound"] == "hbm":
        avg_s = avg_ms * 1e-3
        if name in SURVEY_BYTES_PER_VOXEL:
            ach_s = SURVEY_BYTES_PER_VOXEL[name] * nx * ny * nz / avg_s / 1e9
            roof["frac_survey"] = ach_s / hbm
            roof["bytes_per_voxel"] = {"library": kt["bytes"] / kt["launches"] / (nx * ny * nz),
                                       "survey": SURVEY_BYTES_PER_VOXEL[name]}
        if traffic:
            roof["dram_frac"] = traffic / avg_s / 1e9 / hbm
    roof.update({"kernel": name, "traffic": traffic, "peak_source": peak_src,
                 "avg_launch_us": avg_ms * 1e3, "launches": kt["launches"],
                 "share": kt["ms"] / sum(v["ms"] for v in trace.values())})
    out = {
        "metric": METRIC, "value": per_pair, "unit": "s/pair", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "impl": "b300",
        "config": {"workload": WORKLOAD if SHAPE == (192, 224, 192) else
                   f"profiling case: {WORKLOAD} on a {SHAPE[2]}x{SHAPE[1]}x{SHAPE[0]} grid",
                   "pairs_per_step": world,
                   "l2": "flushed (256 MB write) between timed steps; working set ~6 GB"},
        "residual_reached": last["grad_rel_l2"] <= GTOL,
        "value_is": (f"time to the relative residual {GTOL:g}" if last["grad_rel_l2"] <= GTOL else
                     f"time to the {MAX_GN}-GN cap of the workload (relative residual "
                     f"{last['grad_rel_l2']:.3g} there; {GTOL:g} not reached)"),
        "time_to_residual_s": time_to_residual(histories),
        "residual_trajectory": [[round(h["t"], 5), h["residual"], int(h["pcg"])]
                                for h in histories[-1]],
        "report": dict({k: last[k] for k in ("gn_iters", "pcg_iters_total", "stop_reason", "solves",
                                             "E0", "E", "grad_rel_l2", "grad_rel_inf", "mse_rel")},
                       jacobian_det_min=jac_range[0], jacobian_det_max=jac_range[1],
                       max_displacement_vox=max_disp),
        "sl_voxel_steps_per_s": sl_vps,
        "sl_voxel_steps_per_s_single_call": sl_vps_call,
        "sl_roofline": {"bytes_per_voxel_step": 20, "achieved_GB_s": sl_vps * 20 / 1e9,
                        "frac": sl_vps * 20 / 1e9 / hbm_peak},
        "sl_voxel_steps_per_s_bf16_storage": sl_bf16,
        "e2e": {"value": e2e_total / (args.steps * world), "unit": "s/pair",
                "h2d_bytes_per_step": 2 * ntot * 4, "d2h_bytes_per_step": 3 * K ** 3 * 8},
        "gpu_launches": launches,
        "launches_before_timed": launches0,
        "clocks": clocks,
        "roofline": roof,
        "kernels": {k: {"launches": v["launches"], "ms": round(v["ms"], 3)} for k, v in
                    sorted(trace.items(), key=lambda kv: -kv[1]["ms"])[:12]},
    }
    if forms is not None:
        out["forms"] = forms
    if long_run is not None:
        out["long_run"] = long_run
    if chosen is not None:
        out["chosen_form"] = chosen
    if warm is not None:
        out["warm_start_blobs"] = warm
    if batched is not None:
        out["batched_form"] = batched
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(steps_per_pair=last["solves"] * NT, samples=1)
    return out


RESIDUAL_LEVELS = (1e-1, 1e-2, 1e-3)
LONG_GN = 40
BATCH_PAIRS_IN_LINE = 16


def measure_batched_form(args):
    """The batched form on the first BATCH_PAIRS_IN_LINE pairs of the batched workload (the
    `--config batch` run with fewer pairs), reported beside the headline: pairs/s through
    lddmm_register_batch against the sequential loop, and the persistent batched transport.
    Outside the timed region; a failure is reported in place of the numbers."""
    sub = argparse.Namespace(**vars(args))
    sub.pairs = min(args.pairs, BATCH_PAIRS_IN_LINE)
    try:
        r = run_batch(sub)
    except Exception as e:   # noqa: BLE001 - reported, the headline stands
        return {"error": f"{type(e).__name__}: {e}"}
    keep = ("value", "unit", "config", "sequential_pairs_per_s", "speedup_vs_sequential",
            "per_pair_time_to_residual_s", "residual_reached", "identical_to_sequential",
            "gpu_launches", "transport")
    return {k: r[k] for k in keep if k in r}


def first_time_at(hist, level):
    """Seconds from the start of the registration to the first Gauss-Newton iterate whose
    relative residual ||g||/||g_ref|| is at or below `level` (None if none is)."""
    for h in hist:
        if h["residual"] <= level:
            return h["t"]
    return None


def time_to_residual(histories):
    """Mean over the timed registrations of the time to each residual level (None where a
    registration never reached it), with the smallest residual reached."""
    out = {}
    for lv in RESIDUAL_LEVELS:
        ts = [first_time_at(h, lv) for h in histories]
        out[f"{lv:g}"] = statistics.mean(ts) if all(t is not None for t in ts) else None
    out["min_residual"] = min(min(x["residual"] for x in h) for h in histories)
    return out


def measure_long_run(L, torch, I0d, I1d, flush):
    """The bench pair registered once more with the Gauss-Newton cap raised to LONG_GN (all
    else as the workload): the residual trajectory shows whether and when 1e-3 is reached."""
    nz, ny, nx = SHAPE
    ctx = L.Context(nx, ny, nz, K, nt=NT, variant=L.V_DEFSTATE, interp=L.INTERP_LINEAR,
                    alpha=ALPHA, s=S_EXP, sigma2=SIGMA2, max_gn=LONG_GN, max_pcg=MAX_PCG,
                    gtol=GTOL)
    ctx.set_images(I0d, I1d)
    flush.fill_(1.0)
    torch.cuda.synchronize()
    _, rep = ctx.register()
    hist = ctx.history()
    ctx.close()
    return {"max_gn": LONG_GN, "gn_iters": rep["gn_iters"], "pcg_iters": rep["pcg_iters_total"],
            "stop_reason": rep["stop_reason"], "E": rep["E"], "seconds": rep["seconds"],
            "time_to_residual_s": time_to_residual([hist]),
            "trajectory": [[round(h["t"], 5), h["residual"], int(h["pcg"]), h["E"]]
                           for h in hist]}


# name, variant, interpolation, precision, non-stationary, spatial domain
FORMS = [("defstate/linear/bf16x3_jbf16", "V_DEFSTATE", "INTERP_LINEAR", "PREC_BF16X3_JBF16", False, False, 0),
         ("image/linear/fp32", "V_IMAGE", "INTERP_LINEAR", "PREC_FP32", False, False, 0),
         ("defstate/cubic/fp32", "V_DEFSTATE", "INTERP_CUBIC", "PREC_FP32", False, False, 0),
         ("image/cubic/fp32", "V_IMAGE", "INTERP_CUBIC", "PREC_FP32", False, False, 0),
         ("defstate/linear/fp32/nonstationary", "V_DEFSTATE", "INTERP_LINEAR", "PREC_FP32", True, False, 0),
         ("state/linear/fp32", "V_STATE", "INTERP_LINEAR", "PREC_FP32", False, False, 0),
         ("image/linear/fp32/nonstationary", "V_IMAGE", "INTERP_LINEAR", "PREC_FP32", True, False, 0),
         ("state/linear/fp32/nonstationary", "V_STATE", "INTERP_LINEAR", "PREC_FP32", True, False, 0),
         ("defstate/linear/fp32/spatial", "V_DEFSTATE", "INTERP_LINEAR", "PREC_FP32", False, True, 0),
         ("image/linear/fp32/spatial", "V_IMAGE", "INTERP_LINEAR", "PREC_FP32", False, True, 0),
         # two-level preconditioner, at most 5 coarse PCG iterations per application
         ("defstate/linear/fp32/two_level", "V_DEFSTATE", "INTERP_LINEAR", "PREC_FP32", False, False, 5)]


def measure_forms(L, torch, I0d, I1d, stream, flush):
    """The bench pair in the other forms of the workload (variant x interpolation, the
    mixed-precision form, the non-stationary velocity, the spatial domain, the two-level
    preconditioner): one untimed and one event-timed registration each."""
    nz, ny, nx = SHAPE
    res = {}
    for name, var, interp, prec, nonst, spatial, two_level in FORMS:
        ctx = L.Context(nx, ny, nz, K, nt=NT, variant=getattr(L, var), interp=getattr(L, interp),
                        alpha=ALPHA, s=S_EXP, sigma2=SIGMA2, max_gn=MAX_GN, max_pcg=MAX_PCG,
                        gtol=GTOL, precision=getattr(L, prec), nonstationary=nonst, spatial=spatial)
        if two_level:
            ctx.set_option(L.OPT_TWO_LEVEL, two_level)
        ctx.set_images(I0d, I1d)
        ctx.register()
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _, rep = ctx.register()
        e1.record(stream)
        e1.synchronize()
        hist = ctx.history()
        ctx.close()
        res[name] = {"s_per_pair": e0.elapsed_time(e1) / 1e3, "gn_iters": rep["gn_iters"],
                     "time_to_residual_s": time_to_residual([hist]),
                     "pcg_iters": rep["pcg_iters_total"], "E": rep["E"],
                     "coarse_pcg_iters": rep["pcg_inner_total"],
                     "grad_rel_l2": rep["grad_rel_l2"],
                     "residual_reached": rep["grad_rel_l2"] <= GTOL}
    return res


# the paper-scale pairs of the chosen-form comparison: velocity seeds (noise seeds s + 1, s + 2);
# seed 1 is the benchmark's own pair
CHOSEN_SEEDS = (1, 4, 7, 10)


def measure_chosen_form(L, torch):
    """The spec comparison on the paper-scale pairs themselves: the plain FP32 method
    (cold start, one pair after another, the workload's 10-GN cap) against batched forms that
    stop once they reach the relative residual the plain method ended at on the same pair:
    FP32 cold batched, mixed-precision (BF16X3_JBF16) cold batched, and the chosen form
    (network warm start trained on this recipe + BF16X3_JBF16 + lddmm_register_batch; the
    cold-start reference norm computed by the library, as for any warm start). Wall-clock
    times with device sync; the chosen arm's clock includes the network's inference."""
    import os as _os
    from paper_2006_06823_b300 import warmstart as WS
    nz, ny, nx = SHAPE
    pairs = [WS.make_phantom_pair(s, (s + 1, s + 2), host_noise=True) for s in CHOSEN_SEEDS]
    base = dict(nt=NT, variant=L.V_DEFSTATE, interp=L.INTERP_LINEAR, alpha=ALPHA, s=S_EXP,
                sigma2=SIGMA2, max_pcg=MAX_PCG)
    ctx = L.Context(nx, ny, nz, K, **dict(base, max_gn=MAX_GN, gtol=GTOL))
    ctx.set_images(*pairs[0])
    ctx.register()                                   # warm-up
    plain = []
    for I0, I1 in pairs:
        ctx.set_images(I0, I1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = ctx.register()
        torch.cuda.synchronize()
        rep["wall_s"] = time.perf_counter() - t0
        plain.append(rep)
    ctx.close()
    t_plain = sum(r["wall_s"] for r in plain)
    res = {"workload": (f"{len(pairs)} paper-scale pairs (192x224x192 noisy ellipsoid phantom, "
                        f"velocity seeds {list(CHOSEN_SEEDS)}; seed 1 is the benchmark pair), "
                        "deformation state, K=32, nt=10, trilinear, <=20 PCG"),
           "plain": {"form": "FP32, cold start, one pair after another, <=10 GN",
                     "s_per_pair": t_plain / len(pairs),
                     "gn_iters": [r["gn_iters"] for r in plain],
                     "final_residual": [r["grad_rel_l2"] for r in plain]}}
    net = None
    if _os.path.exists(WS.WEIGHTS_PHANTOM):
        net = L.Net(WS.NET_D, WS.NET_C, batch_max=1, seed=0)
        WS.load_params(net, WS.WEIGHTS_PHANTOM)
    arms = [("batched_fp32", L.PREC_FP32, False), ("batched_mixed", L.PREC_BF16X3_JBF16, False),
            ("chosen", L.PREC_BF16X3_JBF16, True)]
    for name, prec, warm in arms:
        if warm and net is None:
            res[name] = {"unavailable": "no warm-start weights trained on the paper-scale recipe"}
            continue
        streams = [torch.cuda.Stream() for _ in pairs]
        ctxs = []
        for st, r in zip(streams, plain):
            with torch.cuda.stream(st):
                ctxs.append(L.Context(nx, ny, nz, K, **dict(base, max_gn=2 * MAX_GN,
                                                            gtol=r["grad_rel_l2"], precision=prec)))
        for c, (I0, I1) in zip(ctxs, pairs):
            c.set_images(I0, I1)
        torch.cuda.synchronize()
        start = (lambda I0, I1: net.warm_start(I0, I1, K)) if warm else (lambda I0, I1: None)
        v0 = start(*pairs[0])
        L.register_batch(ctxs[:1], [v0 if v0 is not None else ctxs[0].zeros_cube()])  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        vs = [start(I0, I1) for I0, I1 in pairs]
        vs = [v if v is not None else c.zeros_cube() for v, c in zip(vs, ctxs)]
        reps = L.register_batch(ctxs, vs)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        for c in ctxs:
            c.close()
        res[name] = {"form": (("network warm start + " if warm else "cold start + ") +
                              ("LDDMM_PREC_BF16X3_JBF16" if prec == L.PREC_BF16X3_JBF16 else "FP32") +
                              " + lddmm_register_batch, stop at the plain run's final residual"),
                     "s_per_pair": t / len(pairs), "speedup": t_plain / t,
                     "gn_iters": [r["gn_iters"] for r in reps],
                     "reached": sum(b["grad_rel_l2"] <= a["grad_rel_l2"] * (1 + 1e-12)
                                    for a, b in zip(plain, reps)),
                     "energy_gap_rel_max": max(abs(b["E"] - a["E"]) / abs(a["E"])
                                               for a, b in zip(plain, reps))}
    if net is not None:
        net.close()
    res["speedup"] = res["chosen"].get("speedup")
    return res


WARM_PAIRS = 4


def measure_warm_start(L, torch):
    """Time to the relative residual 1e-3 on held-out warm-start workload pairs
    (192x224x192 Gaussian-blob pairs, 8-voxel deformations): the plain FP32 method (cold start,
    one pair after another) against the chosen form (network warm start + BF16X3 spectral
    stages with BF16 Hessian Jacobians + all pairs batched), both capped at 30 GN."""
    import os as _os
    from paper_2006_06823_b300 import warmstart as WS
    if not _os.path.exists(WS.WEIGHTS):
        return {"unavailable": "no trained warm-start weights in the package"}
    nz, ny, nx = WS.SHAPE
    solver = dict(WS.SOLVER, max_gn=WS.EVAL_MAX_GN)
    seeds = [WS.EVAL_SEED0 + 2 * i for i in range(WARM_PAIRS)]
    pairs = [WS.make_pair(sd) for sd in seeds]
    net = L.Net(WS.NET_D, WS.NET_C, batch_max=1, seed=0)
    WS.load_params(net, WS.WEIGHTS)
    torch.cuda.synchronize()
    # plain FP32, cold, sequential
    ctx = L.Context(nx, ny, nz, WS.K, **solver)
    ctx.set_images(*pairs[0])
    ctx.register()                       # warm-up
    plain = []
    for I0, I1 in pairs:
        ctx.set_images(I0, I1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, rep = ctx.register()
        torch.cuda.synchronize()
        rep["wall_s"] = time.perf_counter() - t0
        plain.append(rep)
    ctx.close()
    # chosen form: warm start + BF16X3_JBF16 + batched
    streams = [torch.cuda.Stream() for _ in pairs]
    ctxs = []
    for st in streams:
        with torch.cuda.stream(st):
            ctxs.append(L.Context(nx, ny, nz, WS.K, **dict(solver, precision=L.PREC_BF16X3_JBF16)))
    for c, (I0, I1) in zip(ctxs, pairs):
        c.set_images(I0, I1)
    torch.cuda.synchronize()
    L.register_batch(ctxs[:1], [net.warm_start(*pairs[0], WS.K)])   # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vs = [net.warm_start(I0, I1, WS.K) for I0, I1 in pairs]
    torch.cuda.synchronize()
    reps = L.register_batch(ctxs, vs)
    torch.cuda.synchronize()
    t_chosen = time.perf_counter() - t0
    for c in ctxs:
        c.close()
    net.close()
    t_plain = sum(r["wall_s"] for r in plain)
    gap = max(abs(b["E"] - a["E"]) / abs(a["E"]) for a, b in zip(plain, reps))
    return {"workload": (f"{WARM_PAIRS} held-out warm-start pairs (192x224x192 Gaussian blobs, "
                         "8-voxel stationary deformation), deformation state, K=32, nt=10, "
                         "trilinear, gtol 1e-3, <=30 GN x <=20 PCG"),
            "plain_fp32_s_per_pair": t_plain / WARM_PAIRS,
            "chosen_s_per_pair": t_chosen / WARM_PAIRS,
            "speedup": t_plain / t_chosen,
            "plain_reached": sum(r["grad_rel_l2"] <= GTOL for r in plain),
            "chosen_reached": sum(r["grad_rel_l2"] <= GTOL for r in reps),
            "plain_gn_iters": [r["gn_iters"] for r in plain],
            "chosen_gn_iters": [r["gn_iters"] for r in reps],
            "energy_gap_rel_max": gap,
            "chosen": "network warm start + LDDMM_PREC_BF16X3_JBF16 + lddmm_register_batch"}


ORACLE_GB_PER_REPLICA = 3.0     # peak host memory of one oracle step at 192x224x192 (~1.9 GB)


def _oracle_step_inputs():
    """Seeded inputs of the oracle's one-step sample (a BL SL-RK step of the deformation
    state at the workload's grid)."""
    from paper_2006_06823_b300 import synth
    r = synth.rng(7)
    u = synth.random_velocity_coeffs(K, K, seed=8) * 0.05
    D = synth.random_displacement(SHAPE, seed=9, max_vox=4.0, smooth=2.0)
    W = r.standard_normal((3,) + SHAPE) * 1e-3
    return u, D, W


def _oracle_step(inputs):
    """One BL SL-RK step by the FP64 oracle: iota of 3 components, trilinear Heun gather, pi."""
    from oracle import sl as SL
    u, D, W = inputs
    SL.bl_heun_source_step(u, D, W, W, 0.1, 1, SHAPE, K)


def _oracle_replica(shape, n_warm, n_timed, barriers, queue):
    """One replica of the sample in a spawned process: inputs built, n_warm untimed steps,
    then (all replicas together) n_timed timed steps; reports (start, end) of the timed ones
    in wall-clock time."""
    global SHAPE
    SHAPE = tuple(shape)
    inputs = _oracle_step_inputs()
    barriers[0].wait()
    for _ in range(n_warm):
        _oracle_step(inputs)
    barriers[1].wait()
    t0 = time.time()
    for _ in range(n_timed):
        _oracle_step(inputs)
    queue.put((t0, time.time()))


def _oracle_parallel(nproc, warm=0, timed=None):
    """Wall time of `timed` oracle steps (default: one per replica) spread over nproc
    concurrent replica processes (started with spawn), after `warm` untimed steps spread
    the same way. Returns (wall seconds, replicas used)."""
    import multiprocessing as mp
    timed = nproc if timed is None else timed
    nproc = max(1, min(nproc, max(timed, 1)))
    share = lambda n, i: n // nproc + (1 if i < n % nproc else 0)
    ctx = mp.get_context("spawn")
    barriers = (ctx.Barrier(nproc), ctx.Barrier(nproc))
    queue = ctx.Queue()
    procs = [ctx.Process(target=_oracle_replica,
                         args=(SHAPE, share(warm, i), share(timed, i), barriers, queue))
             for i in range(nproc)]
    for pr in procs:
        pr.start()
    spans = [queue.get(timeout=3600) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
    return max(t1 for _, t1 in spans) - min(t0 for t0, _ in spans), nproc


def _host_replicas():
    """Replicas the host can run at once: one per core, bounded by the available memory."""
    ncpu = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    try:
        import psutil
        mem_gb = psutil.virtual_memory().available / 1e9
        return max(1, min(ncpu, int(mem_gb * 0.8 / ORACLE_GB_PER_REPLICA))), ncpu
    except Exception:
        return max(1, min(ncpu, 4)), ncpu


def cpu_baseline(steps_per_pair, samples=1, parallel=True):
    """The FP64 oracle timed on one BL SL-RK step of the deformation state at full size
    (iota of 3 components, trilinear gather, pi), extrapolated to a registration: on one
    core, and as P concurrent replicas on the host's cores (independent pairs, one per core,
    the way a CPU machine would serve many registrations; P bounded by the memory)."""
    nz, ny, nx = SHAPE
    inputs = _oracle_step_inputs()
    ts = []
    for _ in range(samples):
        t0 = time.perf_counter()
        _oracle_step(inputs)
        ts.append(time.perf_counter() - t0)
    step_s = min(ts)
    single = {"value": step_s * steps_per_pair, "unit": "s/pair", "cores": 1,
              "step_s": step_s, "voxel_steps_per_s": nx * ny * nz / step_s}
    P, ncpu = _host_replicas() if parallel else (1, 1)
    if P > 1:
        wall, P = _oracle_parallel(P)
        per_step = wall / P
        value, cores = per_step * steps_per_pair, P
        sample = (f"one BL SL-RK step (iota x3, trilinear gather, pi x3) at {nx}x{ny}x{nz} in "
                  f"FP64 numpy, {P} concurrent replicas on {ncpu} host cores: {wall:.2f} s wall "
                  f"= {per_step:.2f} s per step per pair; single core {step_s:.2f} s; x "
                  f"{steps_per_pair} steps per registration (the GPU path's count)")
    else:
        per_step, value, cores = step_s, single["value"], 1
        sample = (f"one BL SL-RK step (iota x3, trilinear gather, pi x3) at {nx}x{ny}x{nz} "
                  f"in FP64 numpy = {step_s:.2f} s on one core, x {steps_per_pair} steps per "
                  f"registration (the GPU path's count on this workload)")
    return {"value": value, "unit": "s/pair", "cores": cores, "host_cores": ncpu,
            "kind": "oracle", "sample": sample, "voxel_steps_per_s": nx * ny * nz / per_step,
            "single_core": single}


def run_reference(args):
    """The FP64 oracle on the host cores: the one-step sample of the workload (a BL SL-RK step
    of the deformation state at 192x224x192), `warmup` untimed and `steps` timed samples spread
    over concurrent replica processes (one per core, bounded by memory), extrapolated to a
    registration by the GPU path's step count."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    steps_per_pair = REF_STEPS_PER_PAIR
    nz, ny, nx = SHAPE
    P, ncpu = _host_replicas()
    t_start = time.perf_counter()
    wall, used = _oracle_parallel(P, warm=args.warmup, timed=args.steps)
    per_step = wall / args.steps
    value = per_step * steps_per_pair
    cb = {"value": value, "unit": "s/pair", "cores": used, "host_cores": ncpu, "kind": "oracle",
          "sample": (f"{args.steps} timed (+{args.warmup} untimed) one-step samples (BL SL-RK step "
                     f"of the deformation state: iota x3, trilinear gather, pi x3, FP64 numpy, "
                     f"{nx}x{ny}x{nz}) over {used} concurrent replica processes on {ncpu} host "
                     f"cores: {wall:.2f} s wall = {per_step:.2f} s per pair-step, x "
                     f"{steps_per_pair} steps per registration"),
          "voxel_steps_per_s": nx * ny * nz / per_step}
    return {"metric": METRIC, "value": value, "unit": "s/pair", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": wall * 1e3 / args.steps,
            "wall_s": time.perf_counter() - t_start,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference", "config": {"workload": WORKLOAD},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "s/pair", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


BATCH_SHAPES = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (160, 160, 160), (96, 128, 96)]
def batch_workload(npairs):
    return (f"{npairs} seeded ellipsoid-phantom pairs (seeds 100-{99 + npairs}), grids drawn "
            "from {64^3, 96^3, 128^3, 160^3, 96x128x96}, K drawn from even 16..32, "
            "deformation-state, nt=10, trilinear, <=10 GN x <=20 PCG, gtol=1e-3")


def measure_batch_transport(L, torch, warps, reps=5):
    """The state sweep (nt-step scalar SL transport, trilinear) of every pair: one persistent
    cooperative launch for all pairs (lddmm_sl_transport_batch) against one lddmm_sl_transport
    call per pair, event-timed on the current stream; voxel-steps/s of each and whether the
    results agree bit for bit."""
    stream = torch.cuda.current_stream()
    vels = [v for v, _ in warps]
    fields = [f for _, f in warps]
    voxels = sum(f.numel() for f in fields)

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            out = fn()
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) / 1e3)
        return min(ts), out

    outs_b = [torch.empty_like(f) for f in fields]
    outs_s = [torch.empty_like(f) for f in fields]
    t_b, _ = timed(lambda: L.sl_transport_batch(vels, fields, NT, L.FORWARD, outs=outs_b))
    t_s, _ = timed(lambda: [L.sl_transport(v, f, NT, L.FORWARD, L.INTERP_LINEAR, out=o)
                            for v, f, o in zip(vels, fields, outs_s)])
    same = all(torch.equal(a, b) for a, b in zip(outs_b, outs_s))
    return {"pairs": len(warps), "nt": NT, "voxels": voxels,
            "persistent_batch_voxel_steps_per_s": NT * voxels / t_b,
            "per_pair_calls_voxel_steps_per_s": NT * voxels / t_s,
            "speedup": t_s / t_b, "bit_identical": same,
            "persistent_ms": t_b * 1e3, "per_pair_ms": t_s * 1e3}


def run_batch(args):
    """Batched form: all pairs through lddmm_register_batch (stream per pair, graph-captured
    Hessian products, autotuned SL block shapes) against a sequential loop of plain solves."""
    import numpy as np
    import torch
    import paper_2006_06823_b300 as L
    from paper_2006_06823_b300 import synth
    torch.cuda.set_device(0)
    npairs = args.pairs
    pairs = []
    warps = []            # (velocity in voxels, fixed image) of each pair, for the transport
    for i in range(npairs):
        g = synth.rng(100 + i)
        shape = BATCH_SHAPES[int(g.integers(0, len(BATCH_SHAPES)))]
        K = int(g.choice(np.arange(16, 33, 2)))
        nz, ny, nx = shape
        fixed = synth.ellipsoid_phantom(shape)
        vt = synth.random_velocity_coeffs(K, K, seed=1000 + i)
        v = L.bl_include(torch.as_tensor(vt.astype(np.complex64), device="cuda"), shape)
        to_vox = torch.tensor([nx, ny, nz], dtype=torch.float32, device="cuda").view(3, 1, 1, 1) / (2 * np.pi)
        V = v * to_vox
        V *= (8.0 * nx / 192) / V.pow(2).sum(0).sqrt().max()
        fixed_d = torch.as_tensor(fixed, dtype=torch.float32, device="cuda")
        moving = L.sl_transport(V, fixed_d, NT)
        I0 = synth.add_noise(moving.cpu().numpy().astype(np.float64), seed=2000 + i)
        I1 = synth.add_noise(fixed, seed=3000 + i)
        pairs.append((shape, K, torch.as_tensor(I0, dtype=torch.float32, device="cuda"),
                      torch.as_tensor(I1, dtype=torch.float32, device="cuda")))
        warps.append((V, fixed_d))
    torch.cuda.synchronize()
    transport = measure_batch_transport(L, torch, warps)
    streams = [torch.cuda.Stream() for _ in pairs]
    ctxs = []
    # the autotuner's cache of block shapes per grid (a scratch file outside the repository)
    tune = os.path.join(tempfile.gettempdir(), "lddmm_autotune.json")
    for (shape, K, I0, I1), st in zip(pairs, streams):
        nz, ny, nx = shape
        with torch.cuda.stream(st):
            c = L.Context(nx, ny, nz, K, nt=NT, variant=L.V_DEFSTATE, interp=L.INTERP_LINEAR,
                          alpha=ALPHA, s=S_EXP, sigma2=SIGMA2, max_gn=MAX_GN, max_pcg=MAX_PCG,
                          gtol=GTOL)
            c.set_images(I0, I1)
            c.autotune(tune)
        ctxs.append(c)
    torch.cuda.synchronize()
    # warm-up: one small pass of each path
    for c in ctxs[: min(4, npairs)]:
        c.register()
    L.register_batch(ctxs[: min(4, npairs)], [c.zeros_cube() for c in ctxs[: min(4, npairs)]])
    torch.cuda.synchronize()
    # sequential loop of plain solves
    t0 = time.perf_counter()
    seq = [c.register()[1] for c in ctxs]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    # batched
    vs = [c.zeros_cube() for c in ctxs]
    torch.cuda.synchronize()
    launches0 = L.launch_count()
    t0 = time.perf_counter()
    reps = L.register_batch(ctxs, vs, max_threads=args.batch_threads)
    torch.cuda.synchronize()
    t_bat = time.perf_counter() - t0
    launches = L.launch_count() - launches0
    for c in ctxs:
        c.close()
    same = sum(1 for a, b in zip(seq, reps) if a["gn_iters"] == b["gn_iters"] and
               abs(a["E"] - b["E"]) <= 1e-9 * abs(a["E"]))
    return {"metric": "batched registration throughput (pairs/s)", "value": npairs / t_bat,
            "unit": "pairs/s", "n_gpus": 1, "steps": 1, "warmup": 1,
            "ms_per_step": t_bat * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "b300",
            "config": {"workload": batch_workload(npairs), "pairs": npairs,
                       "threads": args.batch_threads},
            "sequential_pairs_per_s": npairs / t_seq,
            "speedup_vs_sequential": t_seq / t_bat,
            "per_pair_time_to_residual_s": {
                "batched_mean": float(np.mean([r["seconds"] for r in reps])),
                "sequential_mean": float(np.mean([r["seconds"] for r in seq]))},
            "residual_reached": int(sum(r["grad_rel_l2"] <= GTOL for r in reps)),
            "identical_to_sequential": same, "gpu_launches": launches,
            "transport": transport}


def run_spectral(args):
    """Operator throughput of the band-limited projection and inclusion (three components at
    the paper-scale grid, K = 32) in the FP32 and BF16X3 forms, per kernel from the library's
    trace; not a bench line of the headline metric."""
    import torch
    import paper_2006_06823_b300 as L
    torch.cuda.set_device(0)
    nz, ny, nx = SHAPE
    f = torch.rand((3, nz, ny, nx), device="cuda")
    c = L.bl_project(f, K)
    out = torch.empty_like(f)
    res = {}
    for name, prec in (("fp32", L.PREC_FP32), ("bf16x3", L.PREC_BF16X3)):
        for _ in range(args.warmup):
            L.bl_project(f, K, precision=prec, out=c)
            L.bl_include(c, SHAPE, precision=prec, out=out)
        torch.cuda.synchronize()
        L.trace_reset()
        L.trace_enable(True)
        for _ in range(args.steps):
            L.bl_project(f, K, precision=prec, out=c)
            L.bl_include(c, SHAPE, precision=prec, out=out)
        tr = L.trace_read()
        L.trace_enable(False)
        res[name] = {k: {"us_per_launch": v["ms"] / v["launches"] * 1e3,
                         "GB_s": v["bytes"] / (v["ms"] * 1e-3) / 1e9,
                         "TFLOP_s": v["flops"] / (v["ms"] * 1e-3) / 1e12}
                     for k, v in tr.items() if k != "twiddle"}
    return {"metric": "band-limited projection + inclusion, 3 components (per-kernel us)",
            "unit": "us", "impl": "b300", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": f"pi and iota of 3 random fields, {nx}x{ny}x{nz}, K={K}"},
            "kernels": res}


NET_FORMS = (("bf16_tensor_cores", "NET_BF16"), ("bf16_simt", "NET_BF16_SIMT"),
             ("fp32_simt", "NET_FP32"), ("fp32_tensor_cores", "NET_FP32_TC"))


def run_net(args):
    """The warm-start network (64^3 input, 16 base channels, batch 8) in each storage form:
    forward pass and training step (forward, backward, Adam), event-timed, and the per-kernel
    throughput of its convolutions from the library's trace; not a bench line of the headline
    metric."""
    import torch
    import paper_2006_06823_b300 as L
    from paper_2006_06823_b300 import synth
    torch.cuda.set_device(0)
    D, c, B = 64, 16, 8
    x = torch.as_tensor(synth.random_field((D, D, D), 5, ncomp=2 * B, smooth=1.5),
                        dtype=torch.float32, device="cuda").reshape(B, 2, D, D, D).contiguous()
    t = torch.as_tensor(synth.rng(6).standard_normal((B, 3, D // 2, D // 2, D // 2)),
                        dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / args.steps

    res = {}
    for name, form in NET_FORMS:
        net = L.Net(D, c, batch_max=B, seed=0, storage=getattr(L, form))
        fwd = timed(lambda: net.forward(x))
        step = timed(lambda: net.train_step(x, t, 1e-4, want_loss=False))
        L.trace_reset()
        L.trace_enable(True)
        net.train_step(x, t, 1e-4, want_loss=False)
        tr = L.trace_read()
        L.trace_enable(False)
        net.close()
        res[name] = {"forward_ms": fwd, "train_step_ms": step,
                     "conv_TFLOP_s": {k: v["flops"] / (v["ms"] * 1e-3) / 1e12 for k, v in tr.items()
                                      if k in ("cnn_conv", "cnn_dgrad", "cnn_wgrad")}}
    return {"metric": "warm-start network forward / training step (ms)", "unit": "ms",
            "impl": "b300", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": f"encoder-decoder, {D}^3 input, {c} base channels, batch {B}"},
            "forms": res,
            "speedup_train_step_bf16": res["bf16_simt"]["train_step_ms"] / res["bf16_tensor_cores"]["train_step_ms"]}


TRANSPORT_SHAPES = [(64, 64, 64), (96, 96, 96), (128, 128, 128), (160, 160, 160), (96, 128, 96),
                    (64, 64, 64), (128, 128, 128), (96, 96, 96)]


def run_transport(args):
    """The SL state sweep alone (nt = 10 steps, trilinear): the scalar transport at the paper
    grid in FP32 and the BF16-storage forms, and a batch of eight pairs of the batched
    workload's grids in one persistent launch against one call per pair; device rates with the
    transports issued back to back (the working sets exceed L2)."""
    import torch
    import paper_2006_06823_b300 as L
    from paper_2006_06823_b300 import synth
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()

    def rate(fn, voxels):
        for _ in range(args.warmup):
            fn()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            fn()
        e1.record(stream)
        e1.synchronize()
        return args.steps * NT * voxels / (e0.elapsed_time(e1) / 1e3)

    nz, ny, nx = SHAPE
    V = torch.as_tensor(synth.random_displacement(SHAPE, seed=1, max_vox=8.0, smooth=6.0),
                        dtype=torch.float32, device="cuda")
    f = torch.as_tensor(synth.ellipsoid_phantom(SHAPE), dtype=torch.float32, device="cuda")
    o = torch.empty_like(f)
    n = f.numel()
    single = {"fp32": rate(lambda: L.sl_transport(V, f, NT, L.FORWARD, L.INTERP_LINEAR, out=o), n),
              "fields_bf16": rate(lambda: L.sl_transport_bf16(V, f, NT, L.FORWARD, False, out=o), n),
              "fields_and_offsets_bf16": rate(lambda: L.sl_transport_bf16(V, f, NT, L.FORWARD, True, out=o), n)}
    vels, fields = [], []
    for i, sh in enumerate(TRANSPORT_SHAPES):
        vels.append(torch.as_tensor(synth.random_displacement(sh, seed=10 + i, max_vox=8.0 * sh[2] / 192,
                                                              smooth=4.0), dtype=torch.float32, device="cuda"))
        fields.append(torch.as_tensor(synth.ellipsoid_phantom(sh), dtype=torch.float32, device="cuda"))
    outs_b = [torch.empty_like(x) for x in fields]
    outs_s = [torch.empty_like(x) for x in fields]
    nb = sum(x.numel() for x in fields)
    batch = {"persistent": rate(lambda: L.sl_transport_batch(vels, fields, NT, outs=outs_b), nb),
             "per_pair_calls": rate(lambda: [L.sl_transport(v, x, NT, L.FORWARD, L.INTERP_LINEAR, out=y)
                                             for v, x, y in zip(vels, fields, outs_s)], nb)}
    batch["bit_identical"] = all(torch.equal(a, b) for a, b in zip(outs_b, outs_s))
    return {"metric": "SL voxel-steps/s (state sweep, nt = 10, trilinear)", "unit": "voxel-steps/s",
            "impl": "b300", "steps": args.steps, "warmup": args.warmup,
            "config": {"workload": f"scalar transport of the phantom at {nx}x{ny}x{nz}; batch of "
                                   f"{len(TRANSPORT_SHAPES)} pairs of the batched workload's grids"},
            "single_pair": single, "batch": batch}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", dest="forms", action="store_false",
                    help="skip the other forms of the workload and the warm-start comparison")
    ap.add_argument("--config", default="paper", choices=["paper", "batch", "spectral", "net", "transport"])
    ap.add_argument("--pairs", type=int, default=64)
    ap.add_argument("--batch-threads", type=int, default=16)
    ap.add_argument("--grid", type=int, nargs=3, metavar=("NZ", "NY", "NX"), default=None,
                    help="smaller phantom grid for profiling captures (not a bench line)")
    args = ap.parse_args()
    if args.grid:
        global SHAPE
        SHAPE = tuple(args.grid)
    if args.config == "batch" and args.impl == "b300":
        out = run_batch(args)
    elif args.config == "spectral" and args.impl == "b300":
        out = run_spectral(args)
    elif args.config == "net" and args.impl == "b300":
        out = run_net(args)
    elif args.config == "transport" and args.impl == "b300":
        out = run_transport(args)
    else:
        out = run_reference(args) if args.impl == "reference" else run_b300(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
