"""Benchmark: Mcell-updates/s per RK stage of the ASE-DF residual (2D Euler, FP64) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one SSP-RK3 step (three residual evaluations: x-face sweep, y-face sweep,
flux difference + stage combination, plus the CFL wave-speed reduction) of the
isentropic vortex on a 1024 x 1024 periodic grid with ASE-DF(9,7,5,3) (the 7th-order
scheme is timed too and reported beside it).  Inputs are synthetic (closed-form initial
data).  value = cells x 3 stages x K / (max over ranks of the device time of K steps).

Under torchrun (N > 1) every rank runs an independent replica of the workload on its own
GPU (the solver has no data-path exchange on one grid per GPU): weak scaling.

--impl reference runs the CPU oracle (the plain serial FP64 reference the library is
checked against) on the host cores, on a bounded sample of the same workload per step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2410_05489_gb300 import problems as P  # noqa: E402

METRIC = "Mcell-updates/s per RK stage (2D Euler, ASE-DF 7th/9th, FP64) + % HBM roofline"
UNIT = "Mcell-updates/s"
N_GRID = 1024
ORDER = 9
ORDER_ALSO = 7
HBM_BYTES_PER_CELL_STAGE_2D = 128.0  # read W^(s), W^n, write W^(s+1), sigma in/out, both directions
# Sources of the face-sweep kernel: the ncu summaries under profiles/ record a hash of these
# files beside their counters, and the counters are reported only while the hash matches.
SWEEP_SOURCES = ("ase_df_sweep.cu", "ase_df_sweep_body.cuh", "ase_df_device.cuh", "ase_df_internal.cuh",
                 "ase_df_tileplan.h")
SWEEP_PROFILE = {9: "sweep_kernel_r9_2d_vortex1024_ncu.md", 7: "sweep_kernel_r7_2d_vortex1024_ncu.md"}


def sweep_sources_hash() -> str:
    """First 16 hex digits of the SHA-256 of the sweep kernel's source files, in order."""
    import hashlib

    h = hashlib.sha256()
    for name in SWEEP_SOURCES:
        with open(os.path.join(ROOT, "paper_2410_05489_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_hbm_gbs():
    """The measured HBM copy bandwidth of this GPU pool (MEASURED_PEAKS.json), or None."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f).get("hbm_gbs")
    except (OSError, ValueError):
        return None


def profiled_counters(order: int):
    """(DRAM bytes per sweep launch, FP64 pipe active of active cycles, note) from the ncu
    summary of the order's 1024^2 sweep; (None, None, why) when there is none or when the
    kernel sources changed after it was taken."""
    path = os.path.join(ROOT, "profiles", SWEEP_PROFILE.get(order, ""))
    try:
        with open(path) as f:
            text = f.read()
    except OSError:
        return None, None, "no ncu summary for this order"
    vals = {}
    for line in text.splitlines():
        for key in ("kernel-sources-sha256", "dram-bytes-per-launch", "fp64-pipe-active"):
            if line.strip().startswith(key + ":"):
                vals[key] = line.split(":", 1)[1].strip()
    if vals.get("kernel-sources-sha256") != sweep_sources_hash():
        return None, None, "the kernel sources changed after the ncu capture"
    try:
        return float(vals["dram-bytes-per-launch"]), float(vals["fp64-pipe-active"]), "ncu, same kernel sources"
    except (KeyError, ValueError):
        return None, None, "ncu summary without counters"


# FP64 operations of one Gauss point: both sides' primitives, the Lax-Friedrichs flux
# 1/2 (F_L + F_R - lambda (q_R - q_L)) and sigma (Sec. 2.3, Sec. 3.1).  This is the oracle's
# operation count for one point less one multiplication per component: the oracle scales
# both halves of the flux by 1/2 (74 and 59 operations in 2D and 1D; tests/test_flop_model.py).
GAUSS_POINT_FLOPS = {2: 70, 1: 56}


def algorithmic_flops_per_face(ndim: int, r: int) -> float:
    """FP64 operations (add, sub, mul, div, sqrt: 1 each) of one face of one sweep on the
    all-smooth branch: the normal reconstruction of the face's cell evaluated at both of
    its faces (2 C (2r-1)), the tangential reconstruction at the G Gauss points of both
    states (2 C G (2r-1)), and per Gauss point the Lax-Friedrichs flux with primitives
    and sigma (GAUSS_POINT_FLOPS) plus the Gauss sum (2 C + 1); + 1 for the face sigma."""
    C = 4 if ndim == 2 else 3
    G = ((r - 1) // 2 if r > 3 else 1) if ndim == 2 else 1
    phi = GAUSS_POINT_FLOPS[ndim]
    normal = 2 * C * (2 * r - 1)
    tang = 2 * C * G * (2 * r - 1) if ndim == 2 else 0
    return normal + tang + G * (phi + 2 * C + 1) + 1


# The gas-kinetic Gauss point (Sec. 2.2, Appendix A): FP64 operations of one closed-form
# evaluation of F and F_t (three Maxwellians and their moments, half-line moments of two,
# seven slope solves, the compatibility condition, the time integrals), exp and erfc counted
# as one operation each; and sigma of one Gauss point (Sec. 3.1).  tests/test_flop_model.py
# counts both from an evaluation that reproduces the oracle's values.
GKS_POINT_FLOPS = {2: 1365, 1: 598}
SIGMA_POINT_FLOPS = {2: 43, 1: 32}


def gks_flops_per_face(ndim: int, r: int) -> float:
    """FP64 operations of one face of one gas-kinetic sweep on the all-smooth branch: the
    normal reconstruction of the face's cell, value and derivative at both of its faces
    (4 C (2r-1), + 2 C to scale the derivatives by 1/h); in 2D per side, component and Gauss
    point the tangential value, tangential derivative and the tangential reconstruction of
    the normal derivative (3 (2r-1), + 1 to scale the tangential derivative); per Gauss point
    the gas-kinetic flux, sigma and the Gauss sums of F, F_t and sigma (4 C + 1); + 1 for the
    face sigma."""
    C = 4 if ndim == 2 else 3
    G = ((r - 1) // 2 if r > 3 else 1) if ndim == 2 else 1
    normal = 4 * C * (2 * r - 1) + 2 * C
    tang = 2 * C * G * (3 * (2 * r - 1) + 1) if ndim == 2 else 0
    return normal + tang + G * (GKS_POINT_FLOPS[ndim] + SIGMA_POINT_FLOPS[ndim] + 4 * C + 1) + 1


def gks_sweep_roofline(A, torch, s, pb, steps: int, peak_tflops: float, clk_mhz: float) -> dict:
    """Roofline of the gas-kinetic face sweep from its launch times: `steps` more S2O4 steps
    of solver s with a CUDA event pair around every launch (x and y sweeps in series)."""
    A.ase_df_profile_enable(s.ctx, True)
    for _ in range(steps):
        s.gks_step()
    torch.cuda.synchronize()
    ms, n = A.ase_df_profile_read(s.ctx)
    A.ase_df_profile_enable(s.ctx, False)
    sweep_ms, sweep_n = ms[0] + ms[1], n[0] + n[1]
    faces = 0.5 * ((pb.nx + 1) * pb.ny + (pb.ny + 1) * pb.nx) if pb.ndim == 2 else pb.nx + 1
    flops = gks_flops_per_face(pb.ndim, pb.order) * faces
    achieved = flops / (sweep_ms / sweep_n * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "gks_sweep_kernel<%d>, x and y launches" % pb.order,
            "achieved": round(achieved, 4), "peak": round(peak_tflops, 4), "unit": "TFLOP/s",
            "frac": round(achieved / peak_tflops, 4), "flops_per_launch": flops,
            "flops_per_face": gks_flops_per_face(pb.ndim, pb.order),
            "launch_ms": round(sweep_ms / sweep_n, 4),
            "launch_ms_source": "CUDA event pair around every launch, %d further steps" % steps,
            "peak_source": "2 FP64 FMA/cycle/SM x SMs x %.0f MHz x 2 flops" % clk_mhz}


# Edges per operation of the oracle's reverse-mode graph of one 2D residual (smooth data,
# 32^2 periodic; tests/test_flop_model.py): the reverse sweep does one multiply-add per edge
# (the cost model of reverse mode), so the residual adjoint's algorithmic flops are taken as
# those of the forward residual times 1 + 2 e.
VJP_EDGES_PER_OP = {5: 1.4197, 7: 1.4451, 9: 1.4552}


def residual_flops(ndim: int, r: int, nx: int, ny: int) -> float:
    """Algorithmic flops of one residual: every face of both sweeps and the flux difference
    (two differences, two products and an add per component and cell)."""
    C = 4 if ndim == 2 else 3
    faces = (nx + 1) * ny + ((ny + 1) * nx if ndim == 2 else 0)
    return algorithmic_flops_per_face(ndim, r) * faces + 5 * C * nx * ny


def residual_adjoint_flops(ndim: int, r: int, nx: int, ny: int) -> float:
    """Algorithmic flops of one residual VJP: the forward recomputed, and one multiply-add
    per edge of its graph in the reverse sweep (VJP_EDGES_PER_OP edges per operation)."""
    return residual_flops(ndim, r, nx, ny) * (1.0 + 2.0 * VJP_EDGES_PER_OP[r])


def fp64_peak_tflops(torch, clk_mhz: float = 2070.0) -> float:
    """2 FP64 FMA per cycle per SM x SMs x SM clock x 2 flops (default: the maximum clock)."""
    n_sm = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return 2.0 * 2.0 * n_sm * clk_mhz * 1e6 / 1e12


def algorithmic_flops_per_cell_stage(ndim: int, r: int) -> float:
    """Both sweeps plus the flux difference and RK combination (9 flops per component)."""
    C = 4 if ndim == 2 else 3
    return ndim * algorithmic_flops_per_face(ndim, r) + 9 * C


# ----------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        return summarise_clocks(self.lines)


def summarise_clocks(lines):
    """Median SM clock, highest maximum SM clock, the throttle reasons seen active in any
    sample, the sample count and the peak power, from nvidia-smi CSV lines in the order of
    ClockSampler.FIELDS (no header, no units); lines that do not parse are skipped."""
    sm, smax, reasons, power = [], [], set(), []
    names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
    for ln in lines:
        parts = [p.strip() for p in ln.split(",")]
        if len(parts) < 8:
            continue
        try:
            clk, clk_max = float(parts[0]), float(parts[1])
        except ValueError:
            continue
        sm.append(clk)
        smax.append(clk_max)
        try:
            power.append(float(parts[2]))
        except ValueError:  # "[N/A]" on parts without a power sensor
            pass
        for nm, v in zip(names, parts[4:8]):
            if v.lower() == "active":
                reasons.add(nm)
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons), "samples": len(sm), "power_w_max": max(power) if power else None}


# ----------------------------------------------------------------------------------
# distributed helpers (replicas)
# ----------------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        import torch

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------
def time_steps(A, torch, pb, W0, steps, warmup, flush_buf, profile=False):
    """Device time (ms) of `steps` SSP-RK3 CFL steps, L2 flushed between steps."""
    s = A.Solver(pb, W0)
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        s.step()
    torch.cuda.synchronize()
    if profile:
        A.ase_df_profile_enable(s.ctx, True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush_buf.fill_(float(k))  # writes 256 MiB: evicts the 129 MB L2 between timed steps
        ev[k][0].record(stream)
        s.step()
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    prof = None
    if profile:
        prof = A.ase_df_profile_read(s.ctx)
        A.ase_df_profile_enable(s.ctx, False)
    flags, last_dt, t = s.status()
    s.close()
    return sum(ms), prof, flags


def time_e2e(A, torch, pb, W0, steps, warmup):
    """Same metric through the public API with host buffers: every step copies its input W^n
    from pinned host memory to the device and its result W^{n+1} back, inside the timed region.
    Two device state buffers let the copies of one step overlap the compute of its neighbours,
    as a caller streaming states through the solver would run it: a copy stream, and events
    that order each buffer's host-to-device copy, step and device-to-host copy."""
    s = A.Solver(pb, W0)
    host_in = torch.from_numpy(np.ascontiguousarray(W0)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    comp = torch.cuda.current_stream()
    cp = torch.cuda.Stream()
    bufs = [s.W, torch.empty_like(s.W)]
    ev = lambda: torch.cuda.Event()  # noqa: E731
    ready, done = [ev(), ev()], [ev(), ev()]
    sy = s.sy if pb.ndim == 2 else None

    def pipeline(n, start):
        cp.wait_event(start)
        for k in range(min(2, n)):
            with torch.cuda.stream(cp):
                bufs[k].copy_(host_in, non_blocking=True)
                ready[k].record(cp)
        for k in range(n):
            b = k % 2
            comp.wait_event(ready[b])
            A.ase_df_step(s.ctx, bufs[b], s.sx, sy, 0.0, comp)
            done[b].record(comp)
            cp.wait_event(done[b])
            with torch.cuda.stream(cp):
                host_out.copy_(bufs[b], non_blocking=True)
                if k + 2 < n:
                    bufs[b].copy_(host_in, non_blocking=True)
                    ready[b].record(cp)
        comp.wait_stream(cp)  # the last read-back is inside the timed region

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(comp)
    pipeline(warmup, e0)
    torch.cuda.synchronize()
    e0.record(comp)
    pipeline(steps, e0)
    e1.record(comp)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    s.close()
    nbytes = host_in.numel() * 8
    return ms, nbytes, nbytes


def cpu_baseline_sample(order: int):
    """The oracle as it stands, one residual evaluation (= one RK stage) of the full
    1024 x 1024 vortex workload: on one host core, and with its face loops on all host
    cores (oracle.threads; the results are the serial ones bit for bit)."""
    from oracle import oracle as O

    O.build()
    pb, W = P.isentropic_vortex(N_GRID, order)
    sx, sy = P.zero_sigma(pb)  # the vortex is smooth: zero and primed sigma take the same branch
    t0 = time.perf_counter()
    O.residual(pb, W, sx, sy)
    dt = time.perf_counter() - t0
    cores = _cores()
    with O.threads(cores):
        t0 = time.perf_counter()
        O.residual(pb, W, sx, sy)
        dt_all = time.perf_counter() - t0
    return {"value": pb.ncells / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "one residual evaluation (one RK stage) of the %dx%d r=%d vortex, serial C++ oracle, "
                      "%.1f s" % (N_GRID, N_GRID, order, dt),
            "all_cores": {"value": round(pb.ncells / dt_all / 1e6, 4), "unit": UNIT, "cores": cores,
                          "sample": "the same residual with the oracle's face loops on %d host threads, %.2f s"
                                    % (cores, dt_all)}}


def run_ours(args, world, rank, local):
    import torch

    from paper_2410_05489_gb300 import ase_df as A
    from paper_2410_05489_gb300 import build

    build.build()
    torch.cuda.set_device(local)
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device="cuda")
    fma_rate = A.ase_df_fp64_fma_rate()

    pb, W0 = P.isentropic_vortex(args.n, args.order)
    pb7, W7 = P.isentropic_vortex(args.n, ORDER_ALSO)

    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    ms, _, flags = time_steps(A, torch, pb, W0, args.steps, args.warmup, flush)
    torch.cuda.synchronize()
    barrier(world)
    ms_max = max_over_ranks(ms, world)
    # Launch durations of the kernels: the same K steps once more with an event pair around
    # every launch.  The pairs add a few microseconds at each launch boundary (~2 % of a
    # 1024^2 step), so the headline above is timed without them.
    ms_prof, prof, _ = time_steps(A, torch, pb, W0, args.steps, args.warmup, flush, profile=True)
    clocks = sampler.stop()
    ms7, _, _ = time_steps(A, torch, pb7, W7, args.steps, args.warmup, flush)
    ms7_max = max_over_ranks(ms7, world)
    _, prof7, _ = time_steps(A, torch, pb7, W7, args.steps, args.warmup, flush, profile=True)
    e2e_ms, bi, bo = time_e2e(A, torch, pb, W0, args.steps, args.warmup)
    e2e_ms = max_over_ranks(e2e_ms, world)

    cells = pb.ncells
    value = world * cells * 3 * args.steps / (ms_max * 1e-3) / 1e6
    value7 = world * cells * 3 * args.steps / (ms7_max * 1e-3) / 1e6
    e2e_value = world * cells * 3 * args.steps / (e2e_ms * 1e-3) / 1e6

    # roofline of the dominant kernel: the face sweep (x and y launches of one kernel)
    # FP64 peak from the unit count and the clock: 2 FP64 FMA per cycle per SM (the
    # issue rate ncu reports as the DFMA peak_sustained on this part) x SMs x the median
    # SM clock sampled during the timed region x 2 flops per FMA
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    clk_mhz = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    peak_tflops = 2.0 * 2.0 * n_sm * clk_mhz * 1e6 / 1e12
    total_prof_ms = sum(prof[0])
    hbm_gbs = measured_hbm_gbs()
    hbm_achieved = value * 1e6 * HBM_BYTES_PER_CELL_STAGE_2D / 1e9
    step_flops = algorithmic_flops_per_cell_stage(2, args.order) * cells * 3
    step_flops7 = algorithmic_flops_per_cell_stage(2, ORDER_ALSO) * cells * 3

    def sweep_roofline(order, pr, ms_steps, ms_with_pairs):
        """Roofline of the face sweep (x and y launches) of one order from its launch times."""
        sweep_ms = pr[0][0] + pr[0][1]
        sweep_n = pr[1][0] + pr[1][1]
        faces_per_launch = 0.5 * ((pb.nx + 1) * pb.ny + (pb.ny + 1) * pb.nx)
        flops_per_launch = algorithmic_flops_per_face(2, order) * faces_per_launch
        achieved = flops_per_launch / (sweep_ms / sweep_n * 1e-3) / 1e12
        traffic, pipe, note = profiled_counters(order) if args.n == N_GRID else (None, None, "not 1024^2")
        r = {
            "bound": "alu",
            "kernel": "sweep_kernel<%d> (fused DF / ASE reconstruction / Gauss-point Lax-Friedrichs flux / sigma), "
                      "x and y launches" % order,
            "achieved": round(achieved, 4),
            "peak": round(peak_tflops, 4),
            "unit": "TFLOP/s",
            "frac": round(achieved / peak_tflops, 4),
            "traffic": traffic,
            "traffic_unit": "bytes per sweep launch (ncu dram__bytes_read.sum + dram__bytes_write.sum)",
            "ncu_fp64_pipe_active": pipe,
            "ncu_note": note,
            "peak_source": "2 FP64 FMA/cycle/SM (ncu DFMA peak_sustained) x %d SMs x %.0f MHz (median sampled "
                           "SM clock in the timed region) x 2 flops" % (n_sm, clk_mhz),
            "peak_microbench": round(2.0 * fma_rate / 1e12, 4),
            "frac_of_microbench": round(achieved / (2.0 * fma_rate / 1e12), 4),
            "flops_per_launch": flops_per_launch,
            "launch_ms": round(sweep_ms / sweep_n, 4),
            "launch_ms_source": "CUDA event pair around every launch, in a second timed pass of the same K steps "
                                "(%.4f ms/step with the pairs)" % (ms_with_pairs / args.steps),
            "share_of_step_time": round(sweep_ms / sum(pr[0]), 4) if sum(pr[0]) > 0 else None,
        }
        return r

    roof = sweep_roofline(args.order, prof, ms_max, ms_prof)
    roof["step_frac_of_fp64_peak"] = round(step_flops * args.steps / (ms_max * 1e-3) / 1e12 / peak_tflops, 4)
    roof["hbm"] = {"achieved_gbs": round(hbm_achieved, 2), "peak_gbs": hbm_gbs,
                   "frac": round(hbm_achieved / hbm_gbs, 5) if hbm_gbs else None,
                   "bytes_per_cell_stage": HBM_BYTES_PER_CELL_STAGE_2D}
    roof7 = sweep_roofline(ORDER_ALSO, prof7, ms7_max, ms7_max)
    roof7["step_frac_of_fp64_peak"] = round(step_flops7 * args.steps / (ms7_max * 1e-3) / 1e12 / peak_tflops, 4)
    roof7.pop("launch_ms_source")
    out = {
        "metric": METRIC,
        "value": round(value, 3),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": dict(workload_config(args, world), value_order7=round(value7, 3),
                       ms_per_step_order7=round(ms7_max / args.steps, 4)),
        "roofline": roof,
        "roofline_order7": roof7,
        "e2e": {"value": round(e2e_value, 3), "unit": UNIT, "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                "method": "every step copies its input from pinned host memory and its result back; two device "
                          "state buffers and a copy stream overlap the copies with the neighbouring steps; no L2 "
                          "flush (the copied input passes through L2, unlike the device-timed steps)"},
        "gpu_launches": int(sum(prof[1])),  # counted in the profiled pass: the same K steps, the same launches
        "clocks": clocks,
        "status_flags": flags,
    }
    if not args.no_batched:
        out["batched"] = batched_bench(A, torch, args)
    if not args.no_adjoint:
        out["adjoint"] = adjoint_bench(A, torch, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_sample(args.order)
    if rank == 0:
        print(json.dumps(out), flush=True)


def batched_bench(A, torch, args):
    """The batched workload (512 problems, 1D N in [128, 16384] and 2D N^2 with N in
    [64, 512], random Riemann data, orders 3/5/7/9): CUDA-graph replays of batch steps
    with the autotuned schedule, against one ase_df_step call per problem per step."""
    from paper_2410_05489_gb300 import batch as Bt

    probs = P.batched_problems()
    order = getattr(args, "batch_order", 0)
    cut = getattr(args, "batch_cut", 0)
    if order:  # the 2D problems of one order (the first `cut` of them if cut is given)
        probs = [p for p in probs if p[0].ndim == 2 and p[0].order == order]
        if cut:
            probs = probs[:cut]
    elif cut:  # the first cut/2 1D and the first cut/2 2D problems (the set lists the 256 1D ones first)
        probs = probs[:cut // 2] + probs[256:256 + cut - cut // 2]
    bt = Bt.Batch([p for p, _ in probs], [w for _, w in probs])
    tune = Bt.autotune(bt, steps=1)
    bt.run(args.warmup)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ksteps = max(2, min(10, args.steps // 4))
    e0.record()
    bt.run(ksteps)
    e1.record()
    e1.synchronize()
    ms_b = e0.elapsed_time(e1) / ksteps
    flags, _, _ = bt.status()
    cells = bt.ncells
    # smooth-branch algorithmic flops of one step (3 stages); the fallback branch at the
    # Riemann data's discontinuities costs more and is not counted
    step_flops = 3 * sum(p.ncells * algorithmic_flops_per_cell_stage(p.ndim, p.order) for p, _ in probs)
    bt.close()
    # one problem per launch: a context per problem, ase_df_step on each in turn
    solvers = [A.Solver(p, w) for p, w in probs]
    for s_ in solvers:
        s_.step()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(ksteps):
        for s_ in solvers:
            s_.step()
    e1.record()
    e1.synchronize()
    ms_1 = e0.elapsed_time(e1) / ksteps
    for s_ in solvers:
        s_.close()
    workload = ("512 problems (256 1D, N log-uniform 128..16384; 256 2D N^2, N log-uniform 64..512), "
                "random Riemann data, orders 3/5/7/9, outflow, CFL 0.5, seed 20241008")
    if order or cut:
        workload = "%d problems of the batched set (%s) -- " % (
            len(probs), ("2D, order %d" % order) if order else "first 1D and 2D ones") + workload
    return {
        "workload": workload,
        "cells": cells, "steps": ksteps,
        "value": round(cells * 3 / (ms_b * 1e-3) / 1e6, 3), "unit": UNIT,
        "ms_per_step": round(ms_b, 4),
        "one_problem_per_launch": {"value": round(cells * 3 / (ms_1 * 1e-3) / 1e6, 3), "ms_per_step": round(ms_1, 4)},
        "speedup": round(ms_1 / ms_b, 3),
        "step_tflops": round(step_flops / (ms_b * 1e-3) / 1e12, 4),
        "step_frac_of_fp64_peak": round(step_flops / (ms_b * 1e-3) / 1e12 / fp64_peak_tflops(torch), 4),
        "schedule": tune.get("schedule"),
        "tiles_2d_lines_by_order": tune.get("tiles"),
        "nonphysical_problems": int(((flags & 1) != 0).sum()),
    }


def adjoint_roofline(torch, pb, order, adj_ms):
    flops = residual_adjoint_flops(pb.ndim, order, pb.nx, pb.ny)
    peak = fp64_peak_tflops(torch)
    achieved = flops / (adj_ms * 1e-3) / 1e12
    return {"bound": "alu", "kernel": "residual adjoint: face, normal and gather kernels of both directions",
            "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
            "frac": round(achieved / peak, 4), "flops": flops,
            "model": "the forward residual's algorithmic flops x (1 + 2 x %.4f): one multiply-add per edge of "
                     "the reverse-mode graph, the oracle tape's %.4f edges per operation at order %d"
                     % (VJP_EDGES_PER_OP[order], VJP_EDGES_PER_OP[order], order),
            "peak_source": "2 FP64 FMA/cycle/SM x SMs x 2070 MHz x 2 flops"}


def adjoint_bench(A, torch, args):
    """The adjoint workload: vortex 256^2 with a seeded 1% density perturbation, order 7,
    50 SSP-RK3 steps at the t = 0 CFL dt, checkpoints every 10 steps, J = sum rho_final^2.
    Times the taped forward (with checkpoint copies), the checkpointed backward, the plain
    forward (ase_df_run), and one residual adjoint against one residual."""
    import numpy as np

    from paper_2410_05489_gb300.adjoint import rollout

    n, order, nsteps, every = 256, 7, 50, 10
    pb, W0 = P.isentropic_vortex(n, order)
    rng = np.random.default_rng(1)
    W0 = W0.copy()
    W0[0] = W0[0] * (1.0 + 0.01 * rng.uniform(-1.0, 1.0, W0[0].shape))
    s = A.Solver(pb, W0)
    # the t = 0 CFL dt, from the library's own CFL step
    probe = A.Solver(pb, W0)
    probe.step(0.0)
    dt = probe.status()[1]
    probe.close()
    W0d = torch.as_tensor(W0, dtype=torch.float64, device="cuda")
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def one():
        W = W0d.clone().requires_grad_(True)
        e0, e1, e2 = ev(), ev(), ev()
        e0.record()
        Wf = rollout(s, W, nsteps, dt, every=every)
        J = (Wf[0] ** 2).sum()
        e1.record()
        (G,) = torch.autograd.grad(J, [W])
        e2.record()
        e2.synchronize()
        return e0.elapsed_time(e1), e1.elapsed_time(e2), G

    for _ in range(2):
        one()
    fw, bw = [], []
    for _ in range(3):
        f_, b_, G = one()
        fw.append(f_)
        bw.append(b_)
    fwd_ms, bwd_ms = min(fw), min(bw)
    # plain forward: the same steps as graph replays, no checkpoints
    s.set_state(W0)
    s.run(nsteps, dt)
    torch.cuda.synchronize()
    plain = []
    for _ in range(3):
        s.set_state(W0)
        e0, e1 = ev(), ev()
        e0.record()
        s.run(nsteps, dt)
        e1.record()
        e1.synchronize()
        plain.append(e0.elapsed_time(e1))
    plain_ms = min(plain)
    # one residual adjoint vs one residual (same inputs)
    s.set_state(W0)
    L, sxo, syo = s.residual()
    Lbar = torch.ones_like(L)
    Wb, sxb, syb = s.residual_adjoint(s.W, s.sx, s.sy, Lbar)
    reps = 20
    torch.cuda.synchronize()
    e0, e1, e2 = ev(), ev(), ev()
    e0.record()
    for _ in range(reps):
        A.ase_df_residual(s.ctx, s.W, s.sx, s.sy, L, sxo, syo)
    e1.record()
    for _ in range(reps):
        A.ase_df_residual_adjoint(s.ctx, s.W, s.sx, s.sy, Lbar, None, None, Wb, sxb, syb)
    e2.record()
    e2.synchronize()
    res_ms, adj_ms = e0.elapsed_time(e1) / reps, e1.elapsed_time(e2) / reps
    _, marked, _ = A.ase_df_get_repair_stats(s.ctx)
    s.close()
    return {
        "workload": "isentropic vortex 256^2 periodic, rho x (1 + 0.01 U[-1,1]) per cell (seed 1), order 7, "
                    "50 SSP-RK3 steps at the t=0 CFL dt, checkpoints every 10 steps, J = sum rho_final^2",
        "dt": dt,
        "forward_ms": round(fwd_ms, 3),
        "backward_ms": round(bwd_ms, 3),
        "plain_forward_ms": round(plain_ms, 3),
        "backward_over_forward": round(bwd_ms / fwd_ms, 3),
        "gradient_over_plain_forward": round((fwd_ms + bwd_ms) / plain_ms, 3),
        "residual_ms": round(res_ms, 4),
        "residual_adjoint_ms": round(adj_ms, 4),
        "residual_adjoint_over_residual": round(adj_ms / res_ms, 3),
        "residual_adjoint_roofline": adjoint_roofline(torch, pb, order, adj_ms),
        "grad_norm": float(torch.linalg.vector_norm(G)),
        "repaired_cells": marked,
    }


# ----------------------------------------------------------------------------------
# reference arm: the CPU oracle
# ----------------------------------------------------------------------------------
def workload_config(args, world):
    """The workload both arms of the benchmark are quoted on."""
    return {
        "workload": "isentropic vortex (strength 5, free stream (1,1,1,1), gamma 1.4) on periodic "
                    "[0,10]^2, %dx%d cells, ASE-DF order %d, SSP-RK3 with CFL 0.5 dt, sigma_thres 2.0"
                    % (args.n, args.n, args.order),
        "nx": args.n, "ny": args.n, "order": args.order, "stages_per_step": 3,
        "l2": "256 MiB device buffer written between timed steps (outside the step events)",
        "parallelism": "replicas" if world > 1 else "single GPU",
    }


def run_reference(args, world, rank):
    if rank != 0:
        return
    from oracle import oracle as O

    O.build()
    ns = args.ref_n
    pb, W = P.isentropic_vortex(ns, args.order)
    sx, sy = O.prime_sigma(pb, W)
    for _ in range(args.warmup):
        O.step(pb, W, sx, sy)
    t0 = time.perf_counter()
    Wk, sxk, syk = W, sx, sy
    for _ in range(args.steps):
        Wk, sxk, syk, _ = O.step(pb, Wk, sxk, syk)
    dt = time.perf_counter() - t0
    value = pb.ncells * 3 * args.steps / dt / 1e6
    sample = ("per step: one SSP-RK3 step of the same vortex workload on a %dx%d grid instead of %dx%d "
              "(same order %d, same per-cell arithmetic; the metric is per cell update) by the serial C++ "
              "oracle" % (ns, ns, args.n, args.n, args.order))
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(value, 5),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": workload_config(args, world),
        "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------------------------
# --suite: every configuration of the workload list, GPU and CPU oracle side by side
# ----------------------------------------------------------------------------------
def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _oracle_all_cores(O, pb, W, sx, sy, threads):
    """One residual evaluation by the oracle with its face loops on `threads` host threads
    (oracle.threads: the serial results bit for bit)."""
    with O.threads(threads):
        O.residual(pb, W, sx, sy)


def _cpu_rates(O, pb, W, sx, sy, cores):
    t0 = time.perf_counter()
    O.residual(pb, W, sx, sy)
    t1 = time.perf_counter()
    _oracle_all_cores(O, pb, W, sx, sy, cores)
    t2 = time.perf_counter()
    return ({"value": round(pb.ncells / (t1 - t0) / 1e6, 4), "cores": 1},
            {"value": round(pb.ncells / (t2 - t1) / 1e6, 4), "cores": cores})


def suite_bench(args):
    """GPU throughput, roofline fraction and the CPU oracle (one core and all cores) for
    the Sod tube, the vortex at orders 5/7/9, the jet, the batched set and the adjoint."""
    import torch

    from oracle import oracle as O
    from paper_2410_05489_gb300 import ase_df as A
    from paper_2410_05489_gb300 import build

    build.build()
    O.build()
    flush = torch.empty(256 * 1024 * 1024 // 8, dtype=torch.float64, device="cuda")
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    cores = _cores()
    hbm_gbs = measured_hbm_gbs()
    rows = []
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    # Sod: 200 cells, r = 5, to t = 0.2 (the whole run, CFL steps)
    pb, W0 = P.sod(200, 5)
    t0 = time.perf_counter()
    _, _, _, t_end, nsteps = O.run(pb, W0, t_end=0.2)
    cpu_s = time.perf_counter() - t0
    s = A.Solver(pb, W0, t_end=0.2)
    s.run(nsteps)
    torch.cuda.synchronize()
    s.set_state(W0)
    e0, e1 = ev(), ev()
    e0.record()
    s.run(nsteps)
    e1.record()
    e1.synchronize()
    gms = e0.elapsed_time(e1)
    flags, _, t_gpu = s.status()
    s.close()
    rows.append({"config": "Sod 1D, 200 cells, r=5, to t=0.2 (%d CFL steps)" % nsteps,
                 "gpu": {"value": round(pb.ncells * 3 * nsteps / (gms * 1e-3) / 1e6, 3), "ms_run": round(gms, 3),
                         "t_end": t_gpu, "flags": flags,
                         "note": "launch-bound: 200 cells per stage; the whole run is one graph per step"},
                 "cpu_1core": {"value": round(pb.ncells * 3 * nsteps / cpu_s / 1e6, 4), "cores": 1},
                 "cpu_all_cores": {"value": None, "cores": cores, "note": "one row: nothing to split"}})

    # vortex 1024^2 at r = 5, 7, 9 (GPU), oracle on 256^2
    for r in (5, 7, 9):
        pb, W0 = P.isentropic_vortex(1024, r)
        ms, _, flags = time_steps(A, torch, pb, W0, args.steps, args.warmup, flush)
        value = pb.ncells * 3 * args.steps / (ms * 1e-3) / 1e6
        _, prof, _ = time_steps(A, torch, pb, W0, args.steps, args.warmup, flush, profile=True)  # launch times
        sweep_ms, sweep_n = prof[0][0] + prof[0][1], prof[1][0] + prof[1][1]
        faces = 0.5 * ((pb.nx + 1) * pb.ny + (pb.ny + 1) * pb.nx)
        achieved = algorithmic_flops_per_face(2, r) * faces / (sweep_ms / sweep_n * 1e-3) / 1e12
        peak = 2.0 * 2.0 * n_sm * 2070.0e6 / 1e12
        pbc, Wc = P.isentropic_vortex(256, r)
        c1, ca = _cpu_rates(O, pbc, Wc, *P.zero_sigma(pbc), cores)
        rows.append({"config": "vortex 2D 1024^2, r=%d (oracle: one stage at 256^2)" % r,
                     "gpu": {"value": round(value, 3), "ms_per_step": round(ms / args.steps, 4), "flags": flags},
                     "roofline_frac": round(achieved / peak, 4), "hbm_frac":
                         (round(value * 1e6 * HBM_BYTES_PER_CELL_STAGE_2D / 1e9 / hbm_gbs, 5) if hbm_gbs else None),
                     "cpu_1core": c1, "cpu_all_cores": ca})

    # jet 1600 x 800, r = 9: 20 CFL steps from t = 0
    pb, W0 = P.high_mach_jet(1600, 800, 9)
    ms, _, flags = time_steps(A, torch, pb, W0, args.steps, args.warmup, flush)
    value = pb.ncells * 3 * args.steps / (ms * 1e-3) / 1e6
    sx, sy = P.zero_sigma(pb)
    lo, hi = 368, 431
    t0 = time.perf_counter()
    O.residual_rows(pb, W0, sx, sy, lo, hi)
    band = time.perf_counter() - t0
    t0 = time.perf_counter()
    _oracle_all_cores(O, pb, W0, sx, sy, cores)
    full = time.perf_counter() - t0
    rows.append({"config": "jet 2D 1600x800, r=9, %d CFL steps after %d warm-up steps from t=0" % (args.steps, args.warmup),
                 "gpu": {"value": round(value, 3), "ms_per_step": round(ms / args.steps, 4), "flags": flags},
                 "cpu_1core": {"value": round(pb.nx * (hi - lo + 1) / band / 1e6, 4), "cores": 1,
                               "sample": "one stage of rows %d..%d of the initial state, sigma = 0" % (lo, hi)},
                 "cpu_all_cores": {"value": round(pb.ncells / full / 1e6, 4), "cores": cores,
                                   "sample": "one stage of the whole initial state, sigma = 0"}})

    # batched set (GPU) and a seeded subset of it (oracle, one CFL step per problem)
    b = batched_bench(A, torch, args)
    probs = P.batched_problems()[:16]
    t0 = time.perf_counter()
    for pb, W in probs:
        O.step(pb, W, *O.prime_sigma(pb, W))
    one = time.perf_counter() - t0
    from concurrent.futures import ThreadPoolExecutor

    t0 = time.perf_counter()
    with ThreadPoolExecutor(min(cores, len(probs))) as ex:
        list(ex.map(lambda pw: O.step(pw[0], pw[1], *O.prime_sigma(pw[0], pw[1])), probs))
    allc = time.perf_counter() - t0
    sub_cells = sum(pb.ncells for pb, _ in probs)
    rows.append({"config": "batched: 512 problems, 18.0 M cells (oracle: the first 16 problems, priming + one step)",
                 "gpu": {"value": b["value"], "ms_per_step": b["ms_per_step"],
                         "one_problem_per_launch": b["one_problem_per_launch"], "speedup": b["speedup"]},
                 "cpu_1core": {"value": round(sub_cells * 4 / one / 1e6, 4), "cores": 1},
                 "cpu_all_cores": {"value": round(sub_cells * 4 / allc / 1e6, 4), "cores": min(cores, len(probs))}})

    # adjoint: GPU ratios, and the oracle tape's reverse/forward ratio on a 32^2 sample
    a = adjoint_bench(A, torch, args)
    pb, W0 = P.isentropic_vortex(32, 7)
    W0 = W0.copy()
    W0[0] *= 1.0 + 0.01 * np.random.default_rng(1).uniform(-1.0, 1.0, W0[0].shape)
    dt = O.cfl_dt(pb, W0)
    t0 = time.perf_counter()
    Wf = O.run(pb, W0, nsteps=2, dt=dt)[0]
    fwd = time.perf_counter() - t0
    Wbf = np.zeros_like(Wf)
    Wbf[0] = 2.0 * Wf[0]
    t0 = time.perf_counter()
    O.run_vjp(pb, W0, 2, dt, Wbf)
    rev = time.perf_counter() - t0
    rows.append({"config": "adjoint: vortex 256^2 + 1% density noise, r=7, 50 steps, checkpoints every 10",
                 "gpu": {k: a[k] for k in ("forward_ms", "backward_ms", "plain_forward_ms", "backward_over_forward",
                                           "gradient_over_plain_forward", "residual_adjoint_over_residual")},
                 "cpu_1core": {"tape_over_forward": round(rev / fwd, 2), "cores": 1,
                               "sample": "oracle tape (reverse mode incl. taping) vs plain oracle, 32^2, 2 steps"}})
    # gas-kinetic path: Configuration 3, 20 S2O4 steps at 100^2 .. 400^2 (the workload of
    # the paper's Table 4, whose single-core EPYC times are quoted as context)
    table4 = {5: [5.974, 23.116, 51.349, 90.954], 7: [9.053, 32.852, 72.788, 128.006],
              9: [10.803, 42.554, 94.64, 165.221]}
    for r in (5, 7, 9):
        per_n = []
        for k, nn in enumerate((100, 200, 300, 400)):
            pb, W0 = P.configuration3(nn, r)
            s = A.Solver(pb, W0)
            for _ in range(2):
                s.gks_step()
            s.set_state(W0)
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record()
            for _ in range(20):
                s.gks_step()
            e1.record()
            e1.synchronize()
            gms = e0.elapsed_time(e1)
            flags = s.status()[0]
            roof = gks_sweep_roofline(A, torch, s, pb, 20, fp64_peak_tflops(torch), 2070.0)
            s.close()
            per_n.append({"n": nn, "ms_20_steps": round(gms, 3), "sweep_frac": roof["frac"],
                          "value": round(pb.ncells * 2 * 20 / (gms * 1e-3) / 1e6, 3), "flags": flags,
                          "paper_cpu_s_20_steps": table4[r][k],
                          "paper_cpu_over_gpu": round(table4[r][k] / (gms * 1e-3), 1)})
        pbc, Wc = P.configuration3(100, r)
        sxc, syc = O.prime_sigma(pbc, Wc)
        t0 = time.perf_counter()
        O.gks_residual(pbc, Wc, sxc, syc, 0.5 * O.cfl_dt(pbc, Wc))
        one = time.perf_counter() - t0
        rows.append({"config": "GKS + S2O4, Configuration 3, r=%d, 20 CFL steps (Table 4 workload)" % r,
                     "gpu": per_n, "unit": "Mcell-updates/s per stage (2 stages per S2O4 step)",
                     "cpu_1core": {"value": round(pbc.ncells / one / 1e6, 4), "cores": 1,
                                   "sample": "one GKS stage of Configuration 3 at 100^2, oracle"}})
    # double Mach reflection at the paper's 960 x 240 (Sec. 4.3 Example 4), order 9, both
    # flux solvers: 20 CFL steps from t = 0 after 2 warm-up steps; oracle one stage at 240 x 60
    for gks in (False, True):
        pb, W0 = P.double_mach_reflection(960, 9)
        s = A.Solver(pb, W0)
        for _ in range(2):
            s.gks_step() if gks else s.step()
        s.set_state(W0)
        torch.cuda.synchronize()
        e0, e1 = ev(), ev()
        e0.record()
        for _ in range(20):
            s.gks_step() if gks else s.step()
        e1.record()
        e1.synchronize()
        gms = e0.elapsed_time(e1)
        flags, _, t_gpu = s.status()
        s.close()
        stages = 2 if gks else 3
        pbc, Wc = P.double_mach_reflection(240, 9)
        sxc, syc = O.prime_sigma(pbc, Wc)
        t0 = time.perf_counter()
        if gks:
            O.gks_residual(pbc, Wc, sxc, syc, 0.5 * O.cfl_dt(pbc, Wc))
        else:
            O.residual(pbc, Wc, sxc, syc)
        one = time.perf_counter() - t0
        rows.append({"config": "double Mach reflection 960x240, r=9, %s, 20 CFL steps from t=0" %
                               ("GKS + S2O4" if gks else "L-F + SSP-RK3"),
                     "gpu": {"value": round(pb.ncells * stages * 20 / (gms * 1e-3) / 1e6, 3),
                             "ms_per_step": round(gms / 20, 4), "t": t_gpu, "flags": flags},
                     "cpu_1core": {"value": round(pbc.ncells / one / 1e6, 4), "cores": 1,
                                   "sample": "one stage at 240x60, oracle"}})
    print(json.dumps({"suite": rows, "cores": cores}), flush=True)


def gks_bench(args):
    """The gas-kinetic path alone: Configuration 3 at n^2 and order r, 20 CFL S2O4 steps after
    2 warm-up steps; one JSON line (Mcell-updates/s per stage, 2 stages per step)."""
    import torch

    from paper_2410_05489_gb300 import ase_df as A
    from paper_2410_05489_gb300 import build

    build.build()
    pb, W0 = P.configuration3(args.n, args.order)
    s = A.Solver(pb, W0)
    for _ in range(max(2, args.warmup)):
        s.gks_step()
    s.set_state(W0)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        s.gks_step()
    e1.record()
    e1.synchronize()
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    flags = s.status()[0]
    clk = clocks.get("sm_mhz") or clocks.get("sm_max_mhz") or 2070.0
    roof = gks_sweep_roofline(A, torch, s, pb, args.steps, fp64_peak_tflops(torch, clk), clk)
    s.close()
    print(json.dumps({"workload": "GKS + S2O4, Configuration 3, %d^2, order %d" % (args.n, args.order),
                      "steps": args.steps, "ms_per_step": round(ms / args.steps, 4),
                      "value": round(pb.ncells * 2 * args.steps / (ms * 1e-3) / 1e6, 3),
                      "unit": "Mcell-updates/s per stage", "flags": flags, "roofline": roof,
                      "clocks": clocks}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--n", type=int, default=N_GRID)
    ap.add_argument("--order", type=int, default=ORDER)
    ap.add_argument("--ref-n", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--gks", action="store_true",
                    help="time only the gas-kinetic path on Configuration 3 (--n, --order, --steps)")
    ap.add_argument("--suite", action="store_true",
                    help="measure every workload configuration (GPU and CPU oracle) instead of the headline line")
    ap.add_argument("--only", choices=("batched", "adjoint"),
                    help="time only the batched or only the adjoint workload (one JSON line; for profiling)")
    ap.add_argument("--batch-order", type=int, default=0, choices=(0, 3, 5, 7, 9),
                    help="with --only batched: only the 2D problems of this order")
    ap.add_argument("--batch-cut", type=int, default=0,
                    help="with --only batched: the first N/2 1D and the first N/2 2D problems of the batched set")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.only:
        if rank == 0:
            import torch

            from paper_2410_05489_gb300 import ase_df as A
            from paper_2410_05489_gb300 import build

            build.build()
            out = batched_bench(A, torch, args) if args.only == "batched" else adjoint_bench(A, torch, args)
            print(json.dumps(out), flush=True)
    elif args.gks:
        if rank == 0:
            gks_bench(args)
    elif args.suite:
        if rank == 0:
            suite_bench(args)
    elif args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
