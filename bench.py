#!/usr/bin/env python
"""Throughput of the transport-velocity WCSPH kick-drift-kick step on GB300.

Workload: 3-D Taylor-Green vortex, periodic [0, 2 pi]^3, 128^3 = 2,097,152
particles on a jittered lattice, h = 1.3 dp, Re = 1600, c0 = 10 (synthetic,
seeded).  One step = kick + drift + cell sort + density + fused pair pass
(Riemann pressure, viscous, limited transport-velocity correction) + closing
kick + FP64 reductions + dt, all in libsphtv's CUDA kernels.

    python bench.py [--gpus N --steps K --warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  value = particle-steps/s of the FP32 form
over all ranks (each rank steps its own replica; the method is not sharded,
so N > 1 runs independent replicas, weak scaling).  The FP64 form is timed
too and reported beside it.  --impl reference times the FP64 CPU oracle on
the host cores instead (same metric, a bounded sample of the workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-steps/s (3D TGV 2.1M, FP32 vs FP64 on GB300); adjoint/forward time"
UNIT = "particle-steps/s"
WORKLOAD = "3-D Taylor-Green vortex 128^3 = 2,097,152 particles, periodic [0,2pi]^3, Re=1600, h=1.3dp, c0=10"

# Algorithmic cost of the fused pair kernel (k_forces, FP32 form), per ordered
# interacting pair (i, j), counted from the formulas it evaluates (an FMA is
# 2 flops; sqrt, reciprocal and division count 1 each):
#   pair vector and r^2 11, sqrt 1, h_ij and 1/h_ij 3, W'(r) 11,
#   rho_j and p_j 2, 1/r 1, e_ij and U_l, U_r 15, dU and beta 5, rho_bar 2,
#   P* 7, 1/(rho_i rho_j) 2, c_p 3, c_v 4, V_j 1, W'/r 1,
#   per axis: grad W 1, pressure+viscous increment 4, residual increment 1
#   (x3 = 18), Kahan compensation 4 per accumulator (x6 = 24)          -> 111
FLOPS_PER_PAIR_FP32 = 111
# Algorithmic cost of the density pass (k_density32, FP32 form) per
# interacting pair, self included: pair vector and r^2 11, sqrt 1,
# W = a_D h^-D t^4 (2q + 1) with q = r/h, t = 1 - q/2: 9, Kahan 4     -> 25.
# The candidate tests of the cell scan (about 146 per particle in 3-D, for
# 81 pairs) are implementation overhead and are not counted.
FLOPS_PER_PAIR_DENSITY32 = 25
# For context only (not algorithmic): the clipped 5^3-cell walk of the density
# pass, its rows cut at quarter-cell sub-cells, tests about 146 candidates per
# particle on this lattice (81 accepted, self included; 184 with the rows cut
# at whole cells), 8 flops each (pair vector and r^2 against the support).
CANDIDATES_PER_PARTICLE = {1: 184, 2: 161, 4: 146}     # by sph_params.x_subcells
FLOPS_PER_CANDIDATE = 8
# Algorithmic bytes of k_density32 per particle: read the float4 position,
# v (12 B), kind (1 B), sigma0 (8 B), cell index (4 B); write the float4
# {v, rho - rho0} and the neighbour count (4 B).  The neighbour list it
# writes (about 80 x 4 B) is an implementation artefact, not counted.
BYTES_PER_PARTICLE_DENSITY = 61
# Algorithmic bytes of k_forces per particle (FP32 form, 3-D): read the
# particle's float4 position + h and float4 {v, rho - rho0} (32 B), mass and
# kind (9 B), cell index (4 B); write a, dr, v, R (48 B), chi (4 B).  Each
# neighbour's data is counted once (it is some other particle's own data).
BYTES_PER_PARTICLE_FORCES = 97
# Measured-peak fallbacks (used only when MEASURED_PEAKS.json is absent).
FALLBACK_HBM_GBS = 6800.0
SMS, FP32_LANES_PER_SM, FP64_LANES_PER_SM = 152, 128, 2
SM_MAX_MHZ = 2070.0


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


# Dual-criteria acoustic substep, per interacting pair: the pressure pass 65
# flops (pair vector 11, r and 1/r 2, W'/r 7, neighbour density and pressure
# 3, U_l - U_r 9, limiter 4, rho_bar 2, P* 7, coefficient 5, three compensated
# accumulations 15) and the continuity pass 49 (pair vector 11, r 2, W'/r 7,
# neighbour state 3, (v_i - v_j).r 8, rho_bar and its reciprocal 3,
# U* - U_l 7, the compensated term 8).
FLOPS_PER_PAIR_ACOUSTIC = 65 + 49
# The FP64 form evaluates the same formulas with plain (uncompensated) sums.
FLOPS_PER_PAIR_FP64 = FLOPS_PER_PAIR_FP32 - 24


def fp32_peak_tflops(sm_mhz: float) -> float:
    """FP32 FMA peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flops x clock."""
    return SMS * FP32_LANES_PER_SM * 2 * sm_mhz * 1e6 / 1e12


def measured_fma_peak(torch, sph, precision: int, target_ms: float = 20.0, reps: int = 3) -> float:
    """FMA throughput (TFLOP/s) of this GPU from the library's sph_fma_peak
    launch: 8 blocks of 256 threads per SM, iterations sized to about
    target_ms, best of reps launches, CUDA events on the launching stream."""
    dev = torch.cuda.current_device()
    blocks = 8 * torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(blocks * 256, dtype=torch.float32 if precision == 32 else torch.float64, device="cuda")
    stream = torch.cuda.current_stream()

    def run(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        flops = sph.sph_fma_peak(precision, blocks, iters, sink, stream)
        e1.record(stream)
        e1.synchronize()
        return flops / (e0.elapsed_time(e1) * 1e-3) / 1e12

    iters = 256
    rate = run(iters)
    iters = max(256, int(rate * 1e12 * target_ms * 1e-3 / (16.0 * blocks * 256)))
    return max(run(iters) for _ in range(reps))


# ------------------------------------------------------------ clocks sampler

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap,timestamp")

    def __init__(self, gpu_index: int):
        self.gpu_index = gpu_index
        self.proc = None
        self.path = None
        self.window = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu_index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "20", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)          # let the sampler run before the timed region opens

    def mark(self, begin: bool):
        """Host time at the start / end of the timed region (the rows kept are those inside it)."""
        import datetime
        now = datetime.datetime.now()
        self.window = (now, None) if begin else (self.window[0] if self.window else now, now)

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.path)
        inside = rows
        if self.window and self.window[1] is not None:
            import datetime

            def stamp(r):
                try:
                    return datetime.datetime.strptime(r[9], "%Y/%m/%d %H:%M:%S.%f")
                except (ValueError, IndexError):
                    return None
            t0, t1 = self.window
            inside = [r for r in rows if stamp(r) is not None and t0 <= stamp(r) <= t1]
            if not inside:       # a region shorter than one sampling interval: the nearest rows
                inside = rows
        rows = inside
        sm = [float(r[1]) for r in rows if _isnum(r[1])]
        smax = [float(r[2]) for r in rows if _isnum(r[2])]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if _isnum(r[3])), default=None)}


def _isnum(s):
    try:
        float(s)
        return True
    except ValueError:
        return False


def _gpu_index(torch, dev):
    """nvidia-smi index of torch device ``dev`` (matched by PCI bus id)."""
    try:
        props = torch.cuda.get_device_properties(dev)
        bus = "%02x:%02x" % (props.pci_bus_id, props.pci_device_id)
        out = subprocess.run(["nvidia-smi", "--query-gpu=index,pci.bus_id", "--format=csv,noheader"],
                             capture_output=True, text=True, timeout=20).stdout
        for line in out.strip().splitlines():
            idx, pci = [t.strip() for t in line.split(",")]
            if pci.lower().endswith(bus + ".0"):
                return int(idx)
    except Exception:  # noqa: BLE001 - best effort
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    if vis and vis.split(",")[0].strip().isdigit():
        return int(vis.split(",")[0])
    return dev


# ------------------------------------------------------------- distributed

def _dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def max_over_ranks(value: float, torch=None, dist=None) -> float:
    """Maximum of a float over all ranks (identity without a process group)."""
    if dist is None or not dist.is_initialized():
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, torch=None, dist=None) -> float:
    if dist is None or not dist.is_initialized():
        return value
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------- CPU oracle

def oracle_rate(n_side: int, steps: int, warmup: int, threads: int):
    """FP64 CPU oracle on a 3-D Taylor-Green of n_side^3 particles (same h/dp,
    same neighbour count per particle as the workload): particle-steps/s over
    ``steps`` timed steps after ``warmup`` untimed ones."""
    import oracle
    from paper_2411_13992_gb300 import cases
    oracle.build()
    oracle.set_threads(threads)
    c = cases.tgv3d(n_side)
    P = oracle.make_params(3, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                           u_ref=c["u_ref"])
    s0 = oracle.sigma0_for(c, 3)
    fp = oracle.force_pass(P, c, c["x"], c["v"], s0)
    st = {"x": c["x"], "v": c["v"], "a": fp["a"], "dr": fp["dr"]}
    dt = oracle.time_step(P, c["v"], c["kind"])
    for _ in range(warmup):
        st = oracle.step(P, c, st, s0, dt)
    t0 = time.perf_counter()
    for _ in range(steps):
        st = oracle.step(P, c, st, s0, dt)
    el = time.perf_counter() - t0
    return c["n"] * steps / el, el, c["n"]


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    threads = os.cpu_count() or 1
    n_side = args.ref_n
    rate, el, n = oracle_rate(n_side, args.steps, args.warmup, threads)
    sample = ("FP64 oracle, cell-list neighbours, OpenMP over particles; 3-D Taylor-Green %d^3 = %d particles "
              "(same h/dp and neighbours per particle as the 128^3 workload), %d timed steps after %d warm-up"
              % (n_side, n, args.steps, args.warmup))
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": "%d^3" % n_side, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- native (GPU)

def _timed_steps(torch, sim, steps, profile=True):
    """Time ``steps`` steps with CUDA events on the library's stream; with
    per-kernel events inside the same region."""
    import paper_2411_13992_gb300 as sph
    stream = sim.stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if profile:
        sph.sph_profile_begin(sim.ctx, steps)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    prof = sph.sph_profile_end(sim.ctx) if profile else None
    sim.sync()
    return e0.elapsed_time(e1), prof


def _rooflines(case, prof, peak_tflops, hbm_gbs, peak_note, kernel_names):
    """Rooflines of the two FP32 pair kernels from a profiled pass (live CUDA
    events on the library stream); the first one returned is the kernel with
    the larger share of the step."""
    n = case["n"]
    pairs = _pairs_per_launch(case)
    roof_d = _alu_roofline("density", kernel_names["density"], prof, pairs + n, FLOPS_PER_PAIR_DENSITY32,
                           BYTES_PER_PARTICLE_DENSITY, n, peak_tflops, hbm_gbs)
    roof_f = _alu_roofline("forces", kernel_names["forces"], prof, pairs, FLOPS_PER_PAIR_FP32,
                           BYTES_PER_PARTICLE_FORCES, n, peak_tflops, hbm_gbs)
    for r in (roof_d, roof_f):
        r["peak_source"] = peak_note
    d_s = roof_d["avg_launch_ms"] * 1e-3
    roof_d["with_candidate_tests"] = {
        "tflops": (pairs + n) * FLOPS_PER_PAIR_DENSITY32 / d_s / 1e12
        + n * CANDIDATES_PER_PARTICLE[_RUN["x_subcells"]] * FLOPS_PER_CANDIDATE / d_s / 1e12,
        "candidates_per_particle": CANDIDATES_PER_PARTICLE[_RUN["x_subcells"]],
        "flops_per_candidate": FLOPS_PER_CANDIDATE,
        "note": "implementation rate: the neighbour search's candidate tests added to the algorithmic flops; "
                "not the roofline figure"}
    # what binds each kernel, from the ncu counters of the committed summary
    # (null once the kernel sources have changed since they were taken)
    roof_d["binding"] = _profiled_counters("density", "binding")
    roof_f["binding"] = _profiled_counters("forces", "binding")
    dominant = prof["density"][0] >= prof["forces"][0]
    return (roof_d, roof_f) if dominant else (roof_f, roof_d)


def _kernel_shares(prof):
    tot = max(sum(t[0] for t in prof.values()), 1e-9)
    return {k: {"ms_per_step": v[0] / max(v[1], 1), "share": v[0] / tot} for k, v in prof.items() if v[1]}


def _density_kernel_name(sim):
    return {0: "k_density32<3,KSum,uniform>", 1: "k_density32_tile<3,KSum>",
            2: "k_density32_coop<3,KSum>", 3: "k_density32_flat<3,KSum>"}[int(sim.params.pair_tiles)]


def run_native(args):
    import numpy as np
    import torch
    import paper_2411_13992_gb300 as sph
    from paper_2411_13992_gb300 import cases

    rank, world, local = _dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.cuda.current_device()

    case = cases.tgv3d(args.n)
    n = case["n"]

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    peaks, src = _peaks()
    hbm_gbs = peaks.get("hbm_gbs", FALLBACK_HBM_GBS)
    gpu_index = _gpu_index(torch, dev)

    # ---- FP32 form: the headline number.  The timed region holds the K steps
    # only: no per-kernel events inside it (the breakdown is a separate pass).
    _RUN["x_subcells"] = args.x_subcells
    sim = sph.Simulation(case, precision=32, pair_tiles=args.pair_tiles, x_subcells=args.x_subcells)
    sim.set_state()
    sim.build_cells()
    sim.step(args.warmup)
    sim.sync()
    launches0 = sim.launches()
    sampler = ClockSampler(gpu_index)
    sampler.start()
    barrier()
    sampler.mark(True)
    ms, _ = _timed_steps(torch, sim, args.steps, profile=False)
    sampler.mark(False)
    barrier()
    clocks = sampler.stop()
    launches = sim.launches() - launches0
    ms_max = max_over_ranks(ms, torch, dist)
    total = sum_over_ranks(float(n * args.steps), torch, dist)
    value = total / (ms_max * 1e-3)
    diag = sim.diag()
    step0 = args.warmup + 1
    # per-kernel breakdown right after the headline steps (not headlined)
    kp = max(1, args.prof_steps)
    ms_p, prof = _timed_steps(torch, sim, kp, profile=True)
    names = {"density": _density_kernel_name(sim), "forces": "k_forces32<3,KSum,uniform>"}

    # ---- steady state: the lattice disorders as the flow develops and the
    # row runs of a warp's lanes grow unequal; step on untimed to step
    # args.steady_from, then time args.steady_steps steps (and a profiled pass)
    steady = None
    if args.steady_steps > 0:
        done = args.warmup + args.steps + kp
        if args.steady_from > done:
            sim.step(args.steady_from - done)
            sim.sync()
        sampler2 = ClockSampler(gpu_index)
        sampler2.start()
        barrier()
        sampler2.mark(True)
        ms_s, _ = _timed_steps(torch, sim, args.steady_steps, profile=False)
        sampler2.mark(False)
        barrier()
        clocks_s = sampler2.stop()
        ms_s = max_over_ranks(ms_s, torch, dist)
        _, prof_s = _timed_steps(torch, sim, kp, profile=True)
        first = max(args.steady_from, done) + 1
        steady = {"value": sum_over_ranks(float(n * args.steady_steps), torch, dist) / (ms_s * 1e-3),
                  "unit": UNIT, "ms_per_step": ms_s / args.steady_steps, "steps": args.steady_steps,
                  "first_step": first, "last_step": first + args.steady_steps - 1, "clocks": clocks_s,
                  "kernels": _kernel_shares(prof_s), "prof": prof_s}
    sim.close()

    # ---- FP64 form, same workload
    sim64 = sph.Simulation(case, precision=64)
    sim64.set_state()
    sim64.build_cells()
    sim64.step(1)
    sim64.sync()
    k64 = max(1, min(args.steps, args.fp64_steps))
    barrier()
    ms64, _ = _timed_steps(torch, sim64, k64, profile=False)
    barrier()
    ms64 = max_over_ranks(ms64, torch, dist)
    value64 = sum_over_ranks(float(n * k64), torch, dist) / (ms64 * 1e-3)
    _, prof64 = _timed_steps(torch, sim64, 1, profile=True)
    sim64.close()

    # ---- dual-criteria integrator (Sec. 2.4), FP32, same workload: one step
    # is one advection step with its acoustic substeps
    dual = None
    if not args.no_dual:
        simd = sph.Simulation(case, precision=32, integrator=sph.INT_DUAL)
        simd.set_state()
        simd.build_cells()
        simd.step(args.warmup)
        simd.sync()
        kd = max(1, min(args.steps, args.dual_steps))
        barrier()
        msd, _ = _timed_steps(torch, simd, kd, profile=False)
        barrier()
        _, profd = _timed_steps(torch, simd, 2, profile=True)
        dd = simd.diag()
        simd.close()
        msd = max_over_ranks(msd, torch, dist)
        ac_ms = profd["acoustic"][0] / max(profd["acoustic"][1], 1) / max(dd["substeps"], 1)
        ac_tflops = _pairs_per_launch(case) * FLOPS_PER_PAIR_ACOUSTIC / (ac_ms * 1e-3) / 1e12
        dual = {"value": sum_over_ranks(float(n * kd), torch, dist) / (msd * 1e-3),
                "acoustic_substep": {"ms": ac_ms, "flops_per_pair": FLOPS_PER_PAIR_ACOUSTIC,
                                     "achieved_tflops": ac_tflops,
                                     "note": "pressure + continuity pair passes per substep over the whole "
                                             "substep's time (its half drifts and reductions included)"},
                "unit": "particle-advection-steps/s", "ms_per_step": msd / kd, "steps": kd,
                "substeps_per_step": dd["substeps"], "Dt_ad": dd["dt"],
                "simulated_time_per_s": dd["dt"] * kd / (msd * 1e-3),
                "kernels_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in profd.items() if v[1]}}

    # ---- end to end through the C ABI with host buffers
    e2e = _e2e(torch, sph, case, args, dist)

    # ---- adjoint / forward time on the adjoint workload
    adjoint = _adjoint_ratio(torch, sph, cases) if not args.no_adjoint else None

    # ---- the other generated workloads (rank 0 of a single-GPU run only)
    others = _other_configs(torch, sph, cases, args) if (world == 1 and not args.no_configs) else None

    # ---- rooflines of the two pair kernels (live event timing of the
    # profiled pass); the line's "roofline" is the one with the larger share
    peak_tflops = measured_fma_peak(torch, sph, 32)
    dfma_tflops = measured_fma_peak(torch, sph, 64)
    units_tflops = fp32_peak_tflops(peaks.get("sm_max_mhz", SM_MAX_MHZ))
    peak_note = ("measured: FP32 FMA microbenchmark (sph_fma_peak) on this GPU; unit counts x max SM clock give "
                 "%.1f TFLOP/s; HBM peak %s" % (units_tflops, src))
    roof, roof_other = _rooflines(case, prof, peak_tflops, hbm_gbs, peak_note, names)
    pairs = _pairs_per_launch(case)
    f64_ms, f64_cnt = prof64["forces"]
    f64_tflops = pairs * FLOPS_PER_PAIR_FP64 / (f64_ms / max(f64_cnt, 1) * 1e-3) / 1e12
    fp64_forces = {"achieved": f64_tflops, "peak": dfma_tflops, "frac": f64_tflops / dfma_tflops,
                   "flops_per_pair": FLOPS_PER_PAIR_FP64,
                   "peak_source": "measured: FP64 FMA microbenchmark (sph_fma_peak)",
                   "binding": _profiled_counters("forces_f64", "binding")}
    if steady is not None:
        prof_s = steady.pop("prof")
        steady["roofline"], steady["roofline_other_pair_kernel"] = _rooflines(case, prof_s, peak_tflops, hbm_gbs,
                                                                              peak_note, names)

    # ---- the larger lattice of the same workload family, 256^3 (rank 0 of a
    # single-GPU run only)
    big = None
    if world == 1 and args.big_n > 0:
        big = _big_lattice(torch, sph, cases, args, peak_tflops, hbm_gbs, peak_note)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, el, nn = oracle_rate(args.cpu_n, 1, 0, threads)
        cpu = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "one FP64 oracle step (cell-list neighbours, OpenMP) of the 3-D Taylor-Green at %d^3 = %d "
                         "particles, %.1f s" % (args.cpu_n, nn, el),
               "parity_sample": _parity_sample(torch, sph, cases)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles_per_gpu": n, "precision": "FP32 pair sums (Kahan), FP64 "
                       "positions and reductions", "parallelism": "replicas" if world > 1 else "single GPU",
                       "timed_steps": "steps %d-%d of the run" % (step0, step0 + args.steps - 1),
                       "density_pass": names["density"], "x_subcells": int(sim.params.x_subcells),
                       "l2": "inputs larger than L2 (%.0f MB state per GPU)" % (sph.sph_query_workspace(
                           sph.params_from_case(case, 32), n) / 1e6)},
            "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64 / k64, "steps": k64,
                     "kernels_ms_per_step": {k: v[0] / max(v[1], 1) for k, v in prof64.items() if v[1]},
                     "forces_roofline": fp64_forces},
            "fp32_over_fp64": value / value64,
            "simulated_time_per_s": diag["dt"] * args.steps / (ms_max * 1e-3),
            "steady_state": steady,
            "tgv3d_256": big,
            "dual_criteria": dual,
            "roofline": roof,
            "roofline_other_pair_kernel": roof_other,
            "kernels": _kernel_shares(prof),
            "kernels_pass": "a profiled pass of %d steps right after the timed steps (CUDA events per kernel "
                            "class on the library stream), not part of the timed region" % kp,
            "e2e": e2e,
            "adjoint": adjoint,
            "other_configs": others,
            "gpu_launches": launches,
            "clocks": clocks,
            "cpu_baseline": cpu,
            "diag_after": {"ke": diag["ke"], "vmax": diag["vmax"], "n_chi": diag["n_chi"]},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def _big_lattice(torch, sph, cases, args, peak_tflops, hbm_gbs, peak_note):
    """The 3-D Taylor-Green at args.big_n^3 (256^3 = 16,777,216 particles),
    FP32: args.big_steps timed steps after 3 warm-up steps, then a profiled
    pass for the kernel breakdown and the rooflines."""
    c = cases.tgv3d(args.big_n)
    sim = sph.Simulation(c, precision=32)
    sim.set_state()
    sim.build_cells()
    sim.step(3)
    sim.sync()
    k = max(1, args.big_steps)
    ms, _ = _timed_steps(torch, sim, k, profile=False)
    _, prof = _timed_steps(torch, sim, 5, profile=True)
    names = {"density": _density_kernel_name(sim), "forces": "k_forces32<3,KSum,uniform>"}
    sim.close()
    roof, roof_other = _rooflines(c, prof, peak_tflops, hbm_gbs, peak_note, names)
    return {"workload": "3-D Taylor-Green vortex %d^3 = %d particles" % (args.big_n, c["n"]),
            "value": c["n"] * k / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / k, "steps": k,
            "timed_steps": "steps 4-%d" % (3 + k), "kernels": _kernel_shares(prof), "roofline": roof,
            "roofline_other_pair_kernel": roof_other}


def _parity_sample(torch, sph, cases):
    """Measured per-field errors of the FP32 and FP64 GPU steps against the
    FP64 oracle, one step from the same state (3-D Taylor-Green 24^3 =
    13,824 particles, same h/dp as the workload): normwise relative,
    max_i |q_i - q_i^ref| / max_i |q_i^ref| per field, with the bound each
    field is tested to."""
    import numpy as np
    import oracle
    c = cases.tgv3d(24)
    P = oracle.make_params(3, c["lo"], c["L"], c["periodic"], c["rho0"], c["c"], c["eta"], c["h_min"],
                           u_ref=c["u_ref"])
    s0 = oracle.sigma0_for(c, 3)
    fp = oracle.force_pass(P, c, c["x"], c["v"], s0)
    dt = oracle.time_step(P, c["v"], c["kind"])
    ref = oracle.step(P, c, {"x": c["x"], "v": c["v"], "a": fp["a"], "dr": fp["dr"]}, s0, dt)
    L = np.asarray(c["L"])

    def disp(x):
        d = x - c["x"]
        return d - L * np.round(d / L)

    def nw(a, b):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        if a.ndim == 2:
            num, den = np.linalg.norm(a - b, axis=1).max(), np.linalg.norm(b, axis=1).max()
        else:
            num, den = np.abs(a - b).max(), np.abs(b).max()
        return float(num / den) if den > 0 else float(num)

    out = {"workload": "3-D Taylor-Green 24^3 = 13,824 particles, one step from the oracle's initial force pass",
           "metric": "normwise relative max_i|q_i - q_i^oracle| / max_i|q_i^oracle|; dr absolute (it is 0 on "
                     "this lattice: chi = 0)"}
    for prec in (32, 64):
        sim = sph.Simulation(c, precision=prec, fixed_dt=dt)
        sim.set_state(a=fp["a"], dr=fp["dr"])
        sim.build_cells()
        sim.step(1)
        sim.sync()
        got = sim.get_state()
        d = sim.diag()
        sim.close()
        ke_ref = 0.5 * float((c["m"][:, None] * ref["v"] ** 2).sum())
        out["fp%d" % prec] = {"x_displacement": nw(disp(got["x"]), disp(ref["x"])), "v": nw(got["v"], ref["v"]),
                              "rho": nw(got["rho"], ref["rho"]), "a": nw(got["a"], ref["a"]),
                              "dr_abs": float(np.abs(got["dr"] - ref["dr"]).max()),
                              "ke": abs(d["ke"] - ke_ref) / ke_ref}
    out["bounds"] = {"fp64": "1e-12 every field", "fp32": "1e-5 for x, v, rho, KE (the stated per-step bound); "
                     "1e-3 for a and dr: p = c^2 (rho - rho0) of Eq. 2 divides the ~1e-7 relative error of FP32 "
                     "positions by (rho - rho0)/rho ~ 1e-3..1e-4 on these flows"}
    return out


def _pairs_per_launch(case) -> int:
    """Ordered interacting pairs (r < 2h, j != i) of the workload: every
    particle of the jittered lattice at h = 1.3 dp has the 80 lattice
    neighbours with |k|^2 <= 6 (|k| < 2.6); jitter of 1e-3 dp cannot move a
    pair across 2h (next shell |k|^2 = 8)."""
    return case["n"] * 80


COUNTERS = os.path.join(ROOT, "profiles", "pair_counters.json")


# settings of this run that the committed ncu counters depend on
_RUN = {"x_subcells": 4}


def _profiled_counters(kernel: str, what: str):
    """ncu counters of a pair kernel ("density", "forces" or "forces_f64")
    from the committed summary: what = "binding" (issue activity, lanes per
    warp instruction, pipe and DRAM utilisation) or "dram_bytes_per_particle".
    None when the summary is absent, the kernel sources have changed since
    the counters were taken (it records a SHA-1 of the sources) or this run
    sorts with other sub-cells than the captured one."""
    import hashlib
    try:
        with open(COUNTERS) as f:
            d = json.load(f)
        h = hashlib.sha1()
        for rel in d["sources"]:
            with open(os.path.join(ROOT, rel), "rb") as f:
                h.update(f.read())
        if h.hexdigest() != d["source_sha1"] or d.get("x_subcells") != _RUN["x_subcells"]:
            return None
        return d["kernels"][kernel][what]
    except (OSError, ValueError, KeyError):
        return None


def _profiled_traffic(kernel: str, n: int):
    """DRAM bytes per launch of a pair kernel for n particles: the captured
    bytes per particle (ncu on a smaller lattice of the same workload) times
    n, since the traffic grows in proportion to the particles (the same
    neighbours per particle); None when the counters are stale."""
    b = _profiled_counters(kernel, "dram_bytes_per_particle")
    return None if b is None else b * n


def _alu_roofline(name, kernel, prof, pairs, flops_per_pair, bytes_per_particle, n, peak_tflops, hbm_gbs):
    ms, cnt = prof[name]
    avg_s = ms / max(cnt, 1) * 1e-3
    achieved = pairs * flops_per_pair / avg_s / 1e12
    hbm = n * bytes_per_particle / avg_s / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": peak_tflops, "unit": "TFLOP/s",
            "frac": achieved / peak_tflops, "traffic": _profiled_traffic(name, n), "kernel": kernel,
            "pairs_per_launch": pairs, "flops_per_pair": flops_per_pair, "avg_launch_ms": avg_s * 1e3,
            "hbm_algorithmic_gbs": hbm, "hbm_peak_gbs": hbm_gbs, "hbm_frac": hbm / hbm_gbs}


def _e2e(torch, sph, case, args, dist):
    """Same metric through the C ABI with host buffers: each step uploads the
    state from pinned host memory, sorts it, steps once and reads the state
    back to pinned host memory."""
    import numpy as np
    n = case["n"]
    sim = sph.Simulation(case, precision=32)
    sim.set_state()
    sim.build_cells()
    sim.step(1)
    pin = {k: torch.empty((n, 3), dtype=torch.float64).pin_memory() for k in ("x", "v", "a", "dr")}
    h = torch.from_numpy(case["h"]).pin_memory()
    m = torch.from_numpy(case["m"]).pin_memory()
    sph.sph_get_state(sim.ctx, pin["x"], pin["v"], pin["a"], pin["dr"], None)
    k = max(1, min(args.steps, args.e2e_steps))

    def one():
        sph.sph_set_state(sim.ctx, pin["x"], pin["v"], pin["a"], pin["dr"], h, m, None, None, None)
        sph.sph_build_cells(sim.ctx)
        sph.sph_step(sim.ctx, 1)
        sph.sph_get_state(sim.ctx, pin["x"], pin["v"], pin["a"], pin["dr"], None)

    one()
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(k):
        one()
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    el = max_over_ranks(el, torch, dist)
    sim.sync()
    sim.close()
    value = sum_over_ranks(float(n * k), torch, dist) / el
    return {"value": value, "unit": UNIT, "h2d_bytes_per_step": 4 * n * 24 + 2 * n * 8,
            "d2h_bytes_per_step": 4 * n * 24, "steps": k,
            "path": "sph_set_state (pinned host) + sph_build_cells + sph_step(1) + sph_get_state (pinned host)"}


def _other_configs(torch, sph, cases, args):
    """Throughput of the other generated workloads (device-resident, CUDA
    events on the library stream, after 3 warm-up steps): the 2-D
    Taylor-Green 50^2 (FP64), the lid-driven cavity 256^2 with its walls
    (FP32 and FP64) and the variable-resolution cylinder (per-particle h,
    FP32 and FP64).  Context for the headline workload, not bench lines."""
    plan = [("2-D Taylor-Green 50^2 = 2,500 particles", cases.tgv2d(50), ((64, 200),)),
            ("lid-driven cavity 256^2 fluid + 3 wall layers, U = 1", cases.cavity2d(256, U=1.0), ((32, 50), (64, 10))),
            ("variable-resolution cylinder (h ratio 2, per-particle h, walls)", cases.cylinder2d(), ((32, 20), (64, 3)))]
    out = []
    for name, c, runs in plan:
        for prec, k in runs:
            sim = sph.Simulation(c, precision=prec)
            sim.set_state()
            sim.build_cells()
            sim.step(3)
            sim.sync()
            ms, _ = _timed_steps(torch, sim, k, profile=False)
            sim.close()
            out.append({"workload": name, "particles": int(c["n"]), "precision": "FP%d" % prec, "steps": k,
                        "ms_per_step": ms / k, "value": c["n"] * k / (ms * 1e-3), "unit": UNIT})
    return out


def _adjoint_ratio(torch, sph, cases):
    """Backward / forward time of a checkpointed rollout: 2-D Taylor-Green
    256^2 = 65,536 particles, 50 steps, checkpoints every 10 steps, loss =
    final kinetic energy, FP32 forward and adjoint.  Forward = the rollout
    with its checkpoint copies; backward = segment replays + reverse steps +
    the adjoint of the initial force pass (gradients w.r.t. v0 and nu)."""
    c = cases.tgv2d(256)
    nsteps, every = 50, 10
    sim = sph.Simulation(c, precision=32, fixed_dt=2.77e-4, adjoint_steps=every)
    dev = sim.device
    x0 = torch.tensor(c["x"], dtype=torch.float64, device=dev)
    m = torch.tensor(c["m"], dtype=torch.float64, device=dev)

    def once():
        v0 = torch.tensor(c["v"], dtype=torch.float64, device=dev, requires_grad=True)
        nu = torch.tensor(c["nu"], dtype=torch.float64, requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xT, vT = sph.Rollout.apply(x0, v0, nu, sim, nsteps, every)
        ke = 0.5 * (m[:, None] * vT ** 2).sum()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        ke.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        return t1 - t0, t2 - t1

    once()
    runs = [once() for _ in range(3)]
    fwd = min(r[0] for r in runs)
    bwd = min(r[1] for r in runs)
    sim.close()
    return {"workload": "2-D Taylor-Green 256^2 = 65,536 particles, 50 steps, checkpoints every 10, FP32",
            "forward_ms": fwd * 1e3, "backward_ms": bwd * 1e3, "adjoint_over_forward": bwd / fwd,
            "timing": "host wall clock around synchronised calls, best of 3 after 1 warm-up"}


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--n", type=int, default=128, help="particles per side of the 3-D Taylor-Green lattice")
    ap.add_argument("--fp64-steps", type=int, default=5)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-n", type=int, default=128, help="lattice side of the CPU-baseline sample")
    ap.add_argument("--ref-n", type=int, default=64, help="lattice side of the reference arm's per-step sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the throughput of the other generated workloads")
    ap.add_argument("--no-dual", action="store_true", help="skip the dual-criteria integrator timing")
    ap.add_argument("--dual-steps", type=int, default=10)
    ap.add_argument("--prof-steps", type=int, default=20,
                    help="steps of the profiled pass (per-kernel events) after the timed steps")
    ap.add_argument("--steady-from", type=int, default=400, help="first step of the steady-state leg")
    ap.add_argument("--steady-steps", type=int, default=100, help="timed steps of the steady-state leg (0: skip)")
    ap.add_argument("--big-n", type=int, default=256, help="lattice side of the larger-lattice leg (0: skip)")
    ap.add_argument("--big-steps", type=int, default=20)
    ap.add_argument("--pair-tiles", type=int, default=0, choices=(0, 1, 2, 3),
                    help="density pass of the headline: 0 row walk (default), 1 tile walk, 2 cooperative tile "
                         "walk, 3 flattened tile walk")
    ap.add_argument("--x-subcells", type=int, default=4, choices=(1, 2, 4),
                    help="sub-cells per cell along x of the sort, where the row walk cuts its runs (default 4)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "native":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
