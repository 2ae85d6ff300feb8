"""Benchmark of the WCSPH wall-boundary step (arXiv 2110.02621) on GB300.

Workload: the 3-D single-phase dam break (tank 1.6 x 0.67 x 0.6 m, water
column 0.4 x 0.67 x 0.3 m, dp = 0.01 m: 80,400 fluid and 120,234 wall
particles, Tait EOS, penalty on, density reinitialisation every 20 steps),
FP32, synthetic lattice input.  One benchmark step = one time step (re-bin
and sort, continuity, wall pressure, momentum, integration) enqueued with
sph_step_async, timed with CUDA events on the library's stream around it, with
a 256 MB write between steps so that every step starts with a cold L2; the
status of the timed steps is checked with sph_sync afterwards.

Metric: M particle-steps/s, particles = fluid + wall particles with fluid
support in that step.  One JSON line on stdout (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

With N > 1 (torchrun) every rank runs an independent replica (the step has no
data-parallel split without a halo exchange, so replicas only); value sums the
ranks' particle-steps over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "M particle-steps/s FP32 vs FP64 GPU at stated error; adjoint/forward time"
UNIT = "M particle-steps/s"
WORKLOAD = "dam_break_80k"

# Algorithmic floating-point operations per in-support pair (add, sub, mul,
# div, sqrt = 1; fma = 2), counted from the pair formulas as the kernels
# evaluate them.  The 27-cell candidate tests of the neighbour search are not
# algorithmic work (a different search visits fewer candidates) and are not
# counted.
FLOPS_PAIR = {
    "momentum_ff": 50,      # Riemann p*, limiter, pressure force, sigma
    "momentum_fw": 40,      # Eq. (RSatWall) pressure force, sigma (penalty rarely active)
    "continuity_ff": 36,    # Riemann continuity term
    "continuity_fw": 33,
    "wall_pressure": 24,    # extrapolation sums
}
# Algorithmic bytes of one launch (the unique data it must read and write
# once): per fluid particle for the streaming kernels, per cell for the scan,
# and for the neighbour build its state (position, cell, row mask, counts: 50
# bytes per particle) plus 4 bytes per list entry and per tagged wall
BYTES_PER_PARTICLE = {"predict": 100, "scatter": 28, "gather": 212}
NB_BYTES_PER_PARTICLE = 50
NB_BYTES_PER_ENTRY = 4
BYTES_PER_CELL_SCAN = 8
BYTES_PER_ACTIVE_WALL = 48
# the whole step's algorithmic bytes per fluid particle: state read and
# written by the three sweeps plus the sort and reorder (no neighbour lists,
# which are this design's own working data)
STEP_BYTES_PER_PARTICLE = 300
# the same step with this design's lists and per-kernel state traffic, for
# the design-inclusive figure kept beside it
DESIGN_BYTES_PER_PARTICLE = {"predict": 100, "scatter": 28, "gather": 212, "neighbors": 400,
                             "continuity": 500, "momentum": 500}
CANDIDATE_TEST_FLOPS = 11   # r (6) and |r|^2 (5) per 27-cell candidate
FP32_LANES_PER_SM = 128
ISSUE_PER_SM_PER_CLOCK = 4  # one warp instruction per scheduler per cycle


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the FP64-form, accuracy and adjoint measurements")
    ap.add_argument("--adjoint-only", action="store_true",
                    help="run only the forward+backward measurement (for profiling the adjoint)")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def replica_throughput(dist, t_ms: float, particle_steps: float, device: str):
    """Whole-job throughput of independent replicas: the particle-steps of all
    ranks over the slowest rank's time (max over ranks), in M/s.  dist is
    torch.distributed (any backend) or None for one process."""
    if dist is None:
        return particle_steps / (t_ms / 1e3) / 1e6, t_ms
    import torch
    t = torch.tensor([t_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    w = torch.tensor([particle_steps], device=device, dtype=torch.float64)
    dist.all_reduce(w, op=dist.ReduceOp.SUM)
    t_max = float(t.item())
    return float(w.item()) / (t_max / 1e3) / 1e6, t_max


def scene():
    from paper_2110_02621_gb300 import scenes
    return scenes.dam_break()


def pair_counts(x_f: np.ndarray, x_w: np.ndarray, h: float):
    """Exact numbers of (ordered) fluid-fluid, fluid-wall pairs within 2h and
    of wall particles with fluid support (cKDTree, host)."""
    from scipy.spatial import cKDTree
    tf = cKDTree(x_f)
    ff = tf.count_neighbors(tf, 2 * h * (1 - 1e-12)) - len(x_f)
    if len(x_w):
        tw = cKDTree(x_w)
        fw = tf.count_neighbors(tw, 2 * h * (1 - 1e-12))
        near = tw.query_ball_tree(tf, 2 * h * (1 - 1e-12))
        active = sum(1 for v in near if v)
    else:
        fw, active = 0, 0
    return int(ff), int(fw), int(active)


def candidate_tests(sim) -> int:
    """Distance tests of the 27-cell neighbour search: for every fluid
    particle, the fluid and wall particles of its cell and the 26 around."""
    c = sim.cells()
    nx, ny, nz = (int(v) for v in c["dims"])
    occ = np.diff(c["start_f"].astype(np.int64)).reshape(nz, ny, nx)
    occw = np.diff(c["start_w"].astype(np.int64)).reshape(nz, ny, nx)
    tot = np.pad(occ + occw, 1)
    box = np.zeros_like(occ)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                box += tot[dz:dz + nz, dy:dy + ny, dx:dx + nx]
    return int((box * occ).sum())


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# sources of the step's kernels (device functions, step kernels, pair sweeps,
# scan); the recorded ncu traffic is void once any of them changes
KERNEL_SOURCES = ("sph_device.cuh", "sph_kernels.cuh", "sph_sweeps.cuh", "sph_sort.cu")


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2110_02621_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, field: str = "dram_bytes_per_launch"):
    """A per-launch figure of a kernel (DRAM bytes, warp instructions) from the
    committed ncu summary, if it was taken on the current kernel sources."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    entry = rec.get(kernel)
    if not entry or entry.get("source_hash") != kernel_source_hash():
        return None
    return entry.get(field)


def streaming_roofline(kernel_us: dict, n_fluid: int, n_cells: int, hbm_gbs: float) -> dict:
    """Achieved HBM bandwidth of the streaming kernels (binning, sort,
    reorder): algorithmic bytes / live time per step, against the measured
    copy bandwidth."""
    out = {}
    for kind in ("predict", "scan", "scatter", "gather"):
        us = kernel_us.get(kind, 0.0)
        if not us:
            continue
        b = n_cells * BYTES_PER_CELL_SCAN if kind == "scan" else n_fluid * BYTES_PER_PARTICLE[kind]
        gbs = b / (us * 1e-6) / 1e9
        out[kind] = {"bytes": b, "us": us, "GB/s": round(gbs, 1), "frac": round(gbs / hbm_gbs, 4)}
    return out


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def device_peaks():
    """Roofline denominators: HBM from MEASURED_PEAKS.json (the driver's copy
    measurement; else the fallback figure), FP32 FMA and instruction issue
    from the device's SM count and the maximum SM clock."""
    import torch
    sm = int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    p = measured_peaks()
    sm_max = float(p.get("sm_max_mhz", 2070.0))
    return {"sm_count": sm, "sm_max_mhz": sm_max,
            "fp32_tflops": sm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12,
            "issue_twips": sm * ISSUE_PER_SM_PER_CLOCK * sm_max * 1e6 / 1e12,
            "hbm_gbs": float(p.get("hbm_gbs", 6800.0)),
            "hbm_source": "measured copy (MEASURED_PEAKS.json)" if "hbm_gbs" in p else "fallback 6.8 TB/s"}


def kernel_work(kind: str, n_fluid: int, ff: float, fw: float, active: float, n_cells: int):
    """Algorithmic work of one launch of a step kernel: ("alu", flops) for the
    pair sweeps, ("hbm", bytes) for the neighbour build and the streaming
    kernels."""
    if kind == "momentum":
        return "alu", ff * FLOPS_PAIR["momentum_ff"] + fw * FLOPS_PAIR["momentum_fw"]
    if kind == "continuity":
        return "alu", ff * FLOPS_PAIR["continuity_ff"] + fw * FLOPS_PAIR["continuity_fw"]
    if kind == "wall_pressure":
        return "alu", fw * FLOPS_PAIR["wall_pressure"]
    if kind == "neighbors":
        return "hbm", n_fluid * NB_BYTES_PER_PARTICLE + NB_BYTES_PER_ENTRY * (ff + fw + active)
    if kind == "scan":
        return "hbm", n_cells * BYTES_PER_CELL_SCAN
    return "hbm", n_fluid * BYTES_PER_PARTICLE[kind]


# fluid particles of the workload the committed ncu capture was taken on
# (the 80,400-particle dam break); other workloads scale its per-launch
# counters by their particle count
NCU_CAPTURE_N_FLUID = 80400


def kernel_roofline(kind: str, ms: float, work, peaks: dict, n_fluid: int = NCU_CAPTURE_N_FLUID) -> dict:
    """achieved = algorithmic work per launch / launch time, against the FP32
    FMA peak (pair sweeps) or the measured copy bandwidth (the rest).  The
    DRAM traffic and warp instructions come from the committed ncu capture;
    for a workload of another size they are that capture's figures scaled by
    n_fluid / NCU_CAPTURE_N_FLUID (per-particle work of the same kind)."""
    scale = n_fluid / NCU_CAPTURE_N_FLUID
    bound, amount = work
    if bound == "alu":
        ach = amount / (ms / 1e3) / 1e12
        r = {"bound": "alu", "kernel": f"k_{kind}", "achieved": ach, "peak": peaks["fp32_tflops"],
             "unit": "TFLOP/s", "frac": ach / peaks["fp32_tflops"], "flops_per_launch": amount,
             "peak_source": f"FP32 FMA: {peaks['sm_count']} SMs (device property) x {FP32_LANES_PER_SM} "
                            f"lanes x 2 x {peaks['sm_max_mhz']:.0f} MHz (derived)"}
    else:
        ach = amount / (ms / 1e3) / 1e9
        r = {"bound": "hbm", "kernel": f"k_{kind}", "achieved": ach, "peak": peaks["hbm_gbs"],
             "unit": "GB/s", "frac": ach / peaks["hbm_gbs"], "bytes_per_launch": amount,
             "peak_source": peaks["hbm_source"]}
    traffic = ncu_traffic(f"k_{kind}")
    r["traffic"] = None if traffic is None else traffic * scale
    if traffic is not None and scale != 1.0:
        r["traffic_source"] = (f"ncu capture of the {NCU_CAPTURE_N_FLUID}-particle dam break, scaled by "
                               f"{n_fluid}/{NCU_CAPTURE_N_FLUID} particles")
    r["ms_per_launch"] = ms
    # the same launch against the SMs' instruction issue rate, from ncu's
    # warp-instruction count of the committed capture (current sources only)
    inst = ncu_traffic(f"k_{kind}", "warp_inst_per_launch")
    if inst:
        inst = inst * scale
        issue = inst / (ms / 1e3) / 1e12
        src = "smsp__inst_executed.sum of the committed ncu capture"
        if scale != 1.0:
            src += f", scaled by {n_fluid}/{NCU_CAPTURE_N_FLUID} particles"
        r["issue"] = {"achieved": issue, "peak": peaks["issue_twips"], "unit": "T warp-instructions/s",
                      "frac": issue / peaks["issue_twips"], "warp_inst_per_launch": inst, "source": src}
    return r


def step_roofline(n_fluid: int, ff: float, fw: float, t_step_us: float, peaks: dict) -> dict:
    """The whole step's algorithmic work (the pair formulas of continuity,
    momentum and wall pressure; the state bytes of the sweeps, sort and
    reorder) as a lower bound on its time, max(flops / FP32 peak, bytes / HBM
    peak), over the measured step time."""
    flops = (ff * (FLOPS_PAIR["continuity_ff"] + FLOPS_PAIR["momentum_ff"])
             + fw * (FLOPS_PAIR["continuity_fw"] + FLOPS_PAIR["momentum_fw"] + FLOPS_PAIR["wall_pressure"]))
    nbytes = STEP_BYTES_PER_PARTICLE * n_fluid
    t_f = flops / (peaks["fp32_tflops"] * 1e12) * 1e6
    t_b = nbytes / (peaks["hbm_gbs"] * 1e9) * 1e6
    return {"flops": flops, "bytes": nbytes, "flops_per_particle": flops / n_fluid,
            "us_at_fp32_peak": t_f, "us_at_hbm_peak": t_b, "us_measured": t_step_us,
            "bound": "alu" if t_f >= t_b else "hbm", "frac": max(t_f, t_b) / t_step_us,
            "peaks": f"FP32 {peaks['fp32_tflops']:.1f} TFLOP/s (derived), HBM {peaks['hbm_gbs']:.0f} GB/s "
                     f"({peaks['hbm_source']})"}


def step_roofline_design(n_fluid: int, ff: float, fw: float, active: float, n_cells: int, cand: int,
                         t_step_us: float, peaks: dict) -> dict:
    """The same bound with this design's own work added: the 27-cell
    candidate tests and the neighbour lists' bytes."""
    flops = (cand * CANDIDATE_TEST_FLOPS
             + ff * (FLOPS_PAIR["continuity_ff"] + FLOPS_PAIR["momentum_ff"])
             + fw * (FLOPS_PAIR["continuity_fw"] + FLOPS_PAIR["momentum_fw"] + FLOPS_PAIR["wall_pressure"]))
    nbytes = (n_fluid * sum(DESIGN_BYTES_PER_PARTICLE.values()) + n_cells * BYTES_PER_CELL_SCAN
              + active * BYTES_PER_ACTIVE_WALL)
    t_f = flops / (peaks["fp32_tflops"] * 1e12) * 1e6
    t_b = nbytes / (peaks["hbm_gbs"] * 1e9) * 1e6
    return {"flops": flops, "bytes": nbytes, "candidate_tests": cand, "us_at_fp32_peak": t_f,
            "us_at_hbm_peak": t_b, "us_measured": t_step_us, "frac": max(t_f, t_b) / t_step_us}


# --------------------------------------------------------------- CPU oracle
def cpu_baseline(sc, active_walls: float, seconds: float):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the same workload (whole steps of the full dam break)."""
    import oracle
    oracle.build()
    sim = oracle.OracleSim(sc)
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter() - t0
    n = max(1, min(2000, int(seconds / max(t1, 1e-3)) - 1))
    t0 = time.perf_counter()
    sim.step(n)
    el = time.perf_counter() - t0
    steps = n + 1
    total = el + t1
    parts = sc.n_fluid + active_walls
    cores = oracle.threads()
    # the same oracle on one core, a shorter sample
    oracle.set_threads(1)
    try:
        t0 = time.perf_counter()
        sim.step(1)
        t_one = time.perf_counter() - t0
        n1 = max(1, min(200, int(0.25 * seconds / max(t_one, 1e-3)) - 1))
        t0 = time.perf_counter()
        sim.step(n1)
        total1 = time.perf_counter() - t0 + t_one
    finally:
        oracle.set_threads(cores)
    sim.close()
    return {"value": parts * steps / total / 1e6, "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{steps} full steps of the {sc.n_fluid}-fluid/{sc.n_wall}-wall dam break "
                      f"({total:.1f} s, FP64 C oracle, OpenMP over particles)",
            "single_core": {"value": parts * (n1 + 1) / total1 / 1e6, "unit": UNIT, "cores": 1,
                            "sample": f"{n1 + 1} further steps ({total1:.1f} s)"}}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    sc = scene()
    import oracle
    oracle.build()
    sim = oracle.OracleSim(sc)
    for _ in range(min(args.warmup, 1)):
        sim.step(1)
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter() - t0
    budget = 60.0
    n = max(1, min(args.steps, int(budget / max(t1, 1e-3))))
    t0 = time.perf_counter()
    sim.step(n)
    el = time.perf_counter() - t0
    _, _, active = pair_counts(sim.fluid()["x"], sc.wall_pos, sc.h)
    parts = sc.n_fluid + active
    value = parts * n / el / 1e6
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": n, "warmup": args.warmup, "ms_per_step": el / n * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "n_fluid": sc.n_fluid,
                                            "n_wall": sc.n_wall, "dp": sc.dp},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(),
                             "kind": "oracle",
                             "sample": f"{n} of the requested {args.steps} steps (bounded to "
                                       f"about {budget:.0f} s) of the full workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    from paper_2110_02621_gb300 import build, sph

    world, rank, local = dist_env()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    if rank == 0:
        build.build()
    if pg:
        pg.barrier()
    build.build()
    sph.lib()
    precision = sph.SPH_FP64_PLAIN if args.precision == "fp64" else sph.SPH_FP32
    sc = scene()
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")

    sim = sph.Simulation(sc, precision=precision, stream=stream.cuda_stream)
    # warm-up steps with every kernel timed by CUDA events on the library's
    # stream: the per-kernel breakdown and the dominant kernel
    sim.profile(sph.KERNEL_KINDS)
    for _ in range(args.warmup):
        flush.zero_()
        sim.step(1)
    warm = sim.profile_read()
    step_kinds = [k for k in sph.KERNEL_KINDS if k != "other" and not k.startswith("adj")]
    dominant = max(step_kinds, key=lambda k: warm[k]["ms"])
    warm_total = sum(warm[k]["ms"] for k in step_kinds)
    shares = {k: round(warm[k]["ms"] / warm_total, 4) for k in step_kinds if warm_total > 0}
    kernel_us = {k: round(warm[k]["ms"] * 1e3 / max(args.warmup, 1), 2) for k in step_kinds}

    ff0, fw0 = sim.neighbor_totals()
    steps0, act_steps0 = sim.counters()
    launches0 = sum(v["launches"] for v in sim.profile_read().values())

    # timed region: no per-kernel events, so each step is one graph launch
    sim.profile([])
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local)
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        sim.step_async(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    wall1 = time.perf_counter()
    sim.sync()  # status of the timed steps
    if pg:
        pg.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    t_ms = float(sum(step_ms))
    prof = sim.profile_read()
    steps1, act_steps1 = sim.counters()
    launches1 = sum(v["launches"] for v in prof.values())
    active_mean = (act_steps1 - act_steps0) / max(steps1 - steps0, 1)
    ff1, fw1 = sim.neighbor_totals()
    # fluid particles whose fluid / wall list overflowed at the end of the
    # timed steps (their sweeps scan the cells instead)
    list_overflow = sim.neighbor_overflow()
    cand_tests = candidate_tests(sim)
    # the dominant kernel's launch duration, CUDA events around each launch,
    # on the steps that follow the timed region (same workload, cold L2)
    sim.profile([dominant])
    n_prof = min(args.steps, 200)
    for _ in range(n_prof):
        flush.zero_()
        sim.step_async(1)
    sim.sync()
    prof2 = sim.profile_read()
    dom_ms = prof2[dominant]["ms"] / max(prof2[dominant]["timed"], 1)
    _, n_cells, _ = sim.grid()
    sim.close()

    parts = sc.n_fluid + active_mean
    value, t_ms = replica_throughput(pg, t_ms, parts * args.steps, "cuda")
    value_fluid, _ = replica_throughput(pg, t_ms, float(sc.n_fluid * args.steps), "cuda")

    # roofline of the dominant kernel: the pair sweeps against the FP32 FMA
    # peak (no dense contraction), the neighbour build and the streaming
    # kernels against the measured copy bandwidth
    pairs_ff = 0.5 * (ff0 + ff1)
    pairs_fw = 0.5 * (fw0 + fw1)
    peaks = device_peaks()
    roofline = kernel_roofline(dominant, dom_ms,
                               kernel_work(dominant, sc.n_fluid, pairs_ff, pairs_fw, active_mean, n_cells), peaks,
                               sc.n_fluid)
    t_step = t_ms / args.steps * 1e3
    step_roof = step_roofline(sc.n_fluid, pairs_ff, pairs_fw, t_step, peaks)
    step_roof_design = step_roofline_design(sc.n_fluid, pairs_ff, pairs_fw, active_mean, n_cells, cand_tests,
                                            t_step, peaks)
    streaming = streaming_roofline(kernel_us, sc.n_fluid, n_cells, peaks["hbm_gbs"])

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if precision == sph.SPH_FP32 else "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_fluid": sc.n_fluid, "n_wall": sc.n_wall,
                       "active_wall_mean": round(active_mean, 1), "dp": sc.dp,
                       "value_fluid_only": value_fluid, "l2": "256 MB write before every timed step",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "kernel_share_warmup": shares, "kernel_us_per_step_warmup": kernel_us,
                       "step_launch": "one CUDA graph per step"},
            "roofline": roofline, "step_roofline": step_roof, "step_roofline_design": step_roof_design,
            "streaming_roofline": streaming,
            "pairs_per_fluid_particle": {"fluid": pairs_ff / sc.n_fluid, "wall": pairs_fw / sc.n_fluid},
            "list_overflow_particles": {"fluid": list_overflow[0], "wall": list_overflow[1]},
            "gpu_launches": int(launches1 - launches0), "clocks": clk,
            "host_wall_s": wall1 - wall0}

    if rank == 0 and world == 1 and not args.no_e2e:
        line["e2e"] = e2e(sc, args.steps, precision, stream, active_mean)
    if rank == 0 and world == 1 and not args.no_extras:
        line["fp64_plain"] = fp64_throughput(sc, min(args.steps, 200), stream, flush)
        line["accuracy"] = accuracy(sc)
        line["adjoint"] = adjoint_block(stream)
        line["other_workloads"] = other_workloads(stream, flush)
        try:  # reported, not fatal: the main line stands on its own
            line["sensors"] = sensors_block(stream)
        except Exception as e:
            line["sensors"] = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(sc, active_mean, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if pg:
        pg.destroy_process_group()
    return 0


def start_dt(sc) -> float:
    """The CFL time step of a fluid at rest (Sec. 2.6), used as a fixed dt
    where runs are compared."""
    dt = sc.cfl * sc.h / sc.c0
    gn = float(np.linalg.norm(sc.g))
    return min(dt, sc.cfl * (sc.h / gn) ** 0.5) if gn > 0 else dt


def fp64_throughput(sc, steps, stream, flush):
    """The plain FP64 form of the same step on the same workload."""
    import torch
    from paper_2110_02621_gb300 import sph
    sim = sph.Simulation(sc, precision=sph.SPH_FP64_PLAIN, stream=stream.cuda_stream)
    for _ in range(5):
        flush.zero_()
        sim.step(1)
    s0, a0 = sim.counters()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        sim.step_async(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    s1, a1 = sim.counters()
    sim.close()
    active = (a1 - a0) / max(s1 - s0, 1)
    return {"value": (sc.n_fluid + active) * steps / (t_ms / 1e3) / 1e6, "unit": UNIT,
            "value_fluid_only": sc.n_fluid * steps / (t_ms / 1e3) / 1e6,
            "ms_per_step": t_ms / steps, "steps": steps, "dtype": "f64"}


def accuracy(sc, nsteps: int = 20):
    """Both GPU forms against the FP64 oracle after nsteps steps of fixed dt
    from the same initial state."""
    import oracle
    from paper_2110_02621_gb300 import sph
    oracle.build()
    dt = start_dt(sc)
    ref = oracle.OracleSim(sc)
    ref.step(nsteps, dt)
    o, ow = ref.fluid(), ref.wall()
    ref.close()
    gnorm = float(np.linalg.norm(sc.g))

    def rel(a, b, floor=0.0):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), floor))

    out = {"steps": nsteps, "dt": dt, "against": "FP64 oracle (C, host)",
           "norm": "max over particles of |gpu - oracle| / max |oracle| per field (a: / max(max|a|, |g|))"}
    for name, prec in (("fp32", sph.SPH_FP32), ("fp64_plain", sph.SPH_FP64_PLAIN)):
        s = sph.Simulation(sc, precision=prec)
        s.step(nsteps, dt)
        g = s.state()
        s.close()
        out[name] = {"x_max_err_dp": float(np.abs(g["x"] - o["x"]).max() / sc.dp),
                     "rho_rel_err": rel(g["rho"], o["rho"]), "p_rel_err": rel(g["p"], o["p"]),
                     "pw_rel_err": rel(g["pw"], ow["pw"]),
                     "a_rel_err": rel(g["a"], o["a"], gnorm),
                     "drho_dt_rel_err": rel(g["drho_dt"], o["drho_dt"])}
        if len(sc.phases) > 1:  # per phase: a light phase has its own FP32 floor
            out[name]["a_rel_err_by_phase"] = [
                rel(g["a"][sc.fluid_phase == k], o["a"][sc.fluid_phase == k], gnorm)
                for k in range(len(sc.phases))]
    return out


def adjoint_block(stream, reps: int = 3):
    """Forward + backward against forward alone on the differentiable dam break
    (dp = 0.0075: 188,680 fluid particles, 10 steps of fixed dt, loss = sum of
    squared wall pressures of 64 probe particles behind the water column), and
    the FP32 gradients against the plain FP64 form's."""
    import torch
    from paper_2110_02621_gb300 import scenes, sph
    sc = scenes.standard("dam_break_adjoint_189k")
    dt = start_dt(sc)
    n = sc.steps
    mask = np.zeros(sc.n_wall)
    mask[sc.probes] = 1.0

    def forward_ms():
        sim = sph.Simulation(sc, precision=sph.SPH_FP32, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(n, dt)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        sim.close()
        return el * 1e3

    def grad_run(prec, seed_pw=None):
        sim = sph.Simulation(sc, precision=prec, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.tape(n, dt)
        t1 = time.perf_counter()
        pw = sim.state()["pw"]
        seed = {"pw": 2.0 * pw * mask if seed_pw is None else seed_pw}
        t2 = time.perf_counter()
        g = sim.backward(seed)
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        sim.close()
        return (t1 - t0) * 1e3, (t3 - t2) * 1e3, g, seed["pw"], float((pw * pw * mask).sum())

    # per-kernel time of one taped forward + backward (CUDA events per launch;
    # the recompute then runs kernel by kernel instead of as a graph)
    sim = sph.Simulation(sc, precision=sph.SPH_FP32, stream=stream.cuda_stream)
    sim.profile(sph.KERNEL_KINDS)
    sim.tape(n, dt)
    tape_prof = sim.profile_read()
    sim.profile(sph.KERNEL_KINDS)
    sim.backward({"pw": 2.0 * sim.state()["pw"] * mask})
    bwd_prof = sim.profile_read()
    sim.close()
    kernel_ms = {"tape": {k: round(v["ms"], 4) for k, v in tape_prof.items() if v["timed"]},
                 "backward": {k: round(v["ms"], 4) for k, v in bwd_prof.items() if v["timed"]}}

    fwd = min(forward_ms() for _ in range(reps))
    runs = [grad_run(sph.SPH_FP32) for _ in range(reps)]
    tape_ms = min(r[0] for r in runs)
    bwd_ms = min(r[1] for r in runs)
    g32, loss32 = runs[0][2], runs[0][4]
    _, _, g64, _, loss64 = grad_run(sph.SPH_FP64_PLAIN, seed_pw=runs[0][3])

    def rel(a, b):
        return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))

    return {"workload": "dam_break_adjoint_189k", "n_fluid": sc.n_fluid, "n_wall": sc.n_wall,
            "steps": n, "dt": dt, "loss": "sum of p_w^2 over 64 probe walls behind the column",
            "loss_fp32": loss32, "loss_fp64": loss64,
            "forward_ms": fwd, "tape_ms": tape_ms, "backward_ms": bwd_ms,
            "fwd_bwd_over_fwd": (tape_ms + bwd_ms) / fwd,
            "timing": "host wall clock around the calls (each synchronises), best of 3",
            "covers": "one phase with continuity density (two-phase and summation-density runs return "
                      "SPH_ERR_UNSUPPORTED); the penalty is silent in this run from rest, so dL/dgamma_p is 0",
            "kernel_ms": kernel_ms,
            "fp32_vs_fp64_grad_rel_err": {k: rel(g32[k], g64[k]) for k in ("x", "v", "rho")},
            "fp32_vs_fp64_param_grad": {k: [g32[k], g64[k]] for k in ("c0", "gamma_p", "mu")}}


def timed_steps(sim, steps: int, stream, flush) -> float:
    """Milliseconds of `steps` enqueued steps, CUDA events around each on the
    library's stream, a 256 MB write before each (cold L2)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        sim.step_async(1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    sim.sync()
    return float(sum(a.elapsed_time(b) for a, b in ev))


def other_workloads(stream, flush, steps: int = 50, fp64_steps: int = 20):
    """The two larger configurations, each as a line of its own: the
    two-phase ramp/cylinder tank and the 10.35 M-particle dam break.  FP32
    throughput (same step, same timing method, fewer steps), the per-kernel
    split, the dominant kernel's roofline and the step's; the plain FP64 form's
    throughput on the same workload; both forms' error against the FP64 oracle
    after one step of fixed dt from the created state."""
    from paper_2110_02621_gb300 import scenes, sph
    peaks = device_peaks()
    out = {}
    for name in ("two_phase_ramp_cylinder", "dam_break_10m"):
        try:
            sc = scenes.standard(name)
            sim = sph.Simulation(sc, precision=sph.SPH_FP32, stream=stream.cuda_stream)
            for _ in range(3):
                flush.zero_()
                sim.step(1)
            s0, a0 = sim.counters()
            ff0, fw0 = sim.neighbor_totals()
            t_ms = timed_steps(sim, steps, stream, flush)
            s1, a1 = sim.counters()
            ff1, fw1 = sim.neighbor_totals()
            sim.profile(sph.KERNEL_KINDS)
            for _ in range(3):
                flush.zero_()
                sim.step(1)
            prof = sim.profile_read()
            _, n_cells, _ = sim.grid()
            sim.close()
            active = (a1 - a0) / max(s1 - s0, 1)
            ff, fw = 0.5 * (ff0 + ff1), 0.5 * (fw0 + fw1)
            kus = {k: round(v["ms"] * 1e3 / 3, 1) for k, v in prof.items() if v["timed"]}
            dom = max((k for k in kus if k != "other"), key=lambda k: kus[k])
            t_step = t_ms / steps * 1e3
            sim64 = sph.Simulation(sc, precision=sph.SPH_FP64_PLAIN, stream=stream.cuda_stream)
            for _ in range(2):
                flush.zero_()
                sim64.step(1)
            s64, a64 = sim64.counters()
            t64 = timed_steps(sim64, fp64_steps, stream, flush)
            s64b, a64b = sim64.counters()
            sim64.close()
            act64 = (a64b - a64) / max(s64b - s64, 1)
            out[name] = {"n_fluid": sc.n_fluid, "n_wall": sc.n_wall, "active_wall_mean": round(active, 1),
                         "ms_per_step": t_ms / steps, "steps": steps,
                         "value": (sc.n_fluid + active) * steps / (t_ms / 1e3) / 1e6,
                         "value_fluid_only": sc.n_fluid * steps / (t_ms / 1e3) / 1e6, "unit": UNIT,
                         "dtype": "f32", "kernel_us_per_step": kus,
                         "pairs_per_fluid_particle": {"fluid": ff / sc.n_fluid, "wall": fw / sc.n_fluid},
                         "roofline": kernel_roofline(dom, kus[dom] / 1e3,
                                                     kernel_work(dom, sc.n_fluid, ff, fw, active, n_cells), peaks,
                                                     sc.n_fluid),
                         "step_roofline": step_roofline(sc.n_fluid, ff, fw, t_step, peaks),
                         "streaming_roofline": streaming_roofline(kus, sc.n_fluid, n_cells, peaks["hbm_gbs"]),
                         "fp64_plain": {"ms_per_step": t64 / fp64_steps, "steps": fp64_steps, "dtype": "f64",
                                        "value": (sc.n_fluid + act64) * fp64_steps / (t64 / 1e3) / 1e6,
                                        "value_fluid_only": sc.n_fluid * fp64_steps / (t64 / 1e3) / 1e6,
                                        "fp32_speedup": (t64 / fp64_steps) / (t_ms / steps)}}
            out[name]["accuracy"] = accuracy(sc, 1)
        except Exception as e:  # reported, not fatal: the main line stands on its own
            out.setdefault(name, {})["error"] = f"{type(e).__name__}: {e}"
    return out


def sensors_block(stream, steps: int = 200):
    """Cost of sampling the obstacle dam break's 5 pressure sensors and 4 wave
    gauges after every step (device buffers, enqueued between asynchronous
    steps), against the step alone: CUDA events on the library's stream."""
    import torch
    from paper_2110_02621_gb300 import scenes, sph
    sc = scenes.standard("dam_break_obstacle_123k")
    sim = sph.Simulation(sc, precision=sph.SPH_FP32, stream=stream.cuda_stream)
    dev = torch.device("cuda")
    pts = torch.from_numpy(sc.sensors).to(dev)
    lines = torch.from_numpy(sc.gauges).to(dev)
    p = torch.zeros((steps, len(pts)), dtype=torch.float64, device=dev)
    w = torch.zeros_like(p)
    H = torch.zeros((steps, len(lines)), dtype=torch.float64, device=dev)
    L = sph.lib()
    sim.step(20)
    out = {}
    for label, sample in (("step", False), ("step_and_sensors", True)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for k in range(steps):
            sim.step_async(1)
            if sample:
                L.sph_probe_pressure(sim.ctx, pts.data_ptr(), len(pts), p[k].data_ptr(), w[k].data_ptr(),
                                     sph.SPH_DEVICE)
                L.sph_gauge_height(sim.ctx, lines.data_ptr(), len(lines), 0.25 * sc.dp, H[k].data_ptr(),
                                   sph.SPH_DEVICE)
        e1.record(stream)
        sim.sync()
        out[label + "_ms"] = e0.elapsed_time(e1) / steps
    sim.close()
    out["sensors_us_per_sample"] = 1e3 * (out["step_and_sensors_ms"] - out["step_ms"])
    out.update({"workload": "dam_break_obstacle_123k", "n_fluid": sc.n_fluid, "n_wall": sc.n_wall,
                "sensors": len(pts), "gauges": len(lines), "steps": steps,
                "H_last": [round(float(v), 4) for v in H[-1].cpu()]})
    return out


def e2e(sc, steps, precision, stream, active_mean):
    """The same metric through the public C ABI with host buffers: create from
    pinned host arrays (H2D inside), then per step sph_step plus a device-to-
    host read of the FP64 diagnostics, then the final state back to the host."""
    import torch
    from paper_2110_02621_gb300 import sph

    def pinned(a, dtype):
        t = torch.empty(a.shape, dtype=dtype, pin_memory=True)
        t.numpy()[...] = a
        return t

    x = pinned(sc.fluid_pos, torch.float64)
    v = pinned(sc.fluid_vel, torch.float64)
    ph = pinned(sc.fluid_phase, torch.int32)
    xw = pinned(sc.wall_pos, torch.float64)
    nf, nw = sc.n_fluid, sc.n_wall
    outs = {k: torch.empty(shape, dtype=torch.float64, pin_memory=True)
            for k, shape in (("x", (nf, 3)), ("v", (nf, 3)), ("rho", (nf,)), ("p", (nf,)),
                             ("pw", (nw,)))}
    diag = torch.empty((steps, 8), dtype=torch.float64, pin_memory=True)
    params = sph.make_params(sc, precision)
    fluid = sph.sph_fluid(nf, x.data_ptr(), v.data_ptr(), None, ph.data_ptr())
    wall = sph.sph_wall(nw, xw.data_ptr())
    out = sph.sph_state_out(outs["x"].data_ptr(), outs["v"].data_ptr(), outs["rho"].data_ptr(),
                            outs["p"].data_ptr(), None, None, None, outs["pw"].data_ptr(), None, None)
    L = sph.lib()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st, ctx = sph.sph_create(params, fluid, wall, stream.cuda_stream)
    assert st == sph.SPH_OK, sph.sph_last_error(None)
    # per step: enqueue the step and the copy of its FP64 diagnostics into a
    # pinned ring; the host does not wait inside the loop
    for k in range(steps):
        assert L.sph_step_async(ctx, 1, 0.0) == sph.SPH_OK
        assert L.sph_diagnostics_async(ctx, diag[k].data_ptr(), sph.SPH_HOST) == sph.SPH_OK
    assert L.sph_sync(ctx, None) == sph.SPH_OK
    assert sph.sph_get_state(ctx, out, sph.SPH_HOST) == sph.SPH_OK
    el = time.perf_counter() - t0
    sph.sph_destroy(ctx)
    h2d = nf * (3 + 3) * 8 + nf * 4 + nw * 3 * 8
    d2h = 8 * 8 * steps + sum(t.numel() * 8 for t in outs.values())
    return {"value": (nf + active_mean) * steps / el / 1e6, "unit": UNIT,
            "h2d_bytes_per_step": h2d / steps, "d2h_bytes_per_step": d2h / steps,
            "seconds": el, "mass_drift": float(abs(diag[-1, 0] - diag[0, 0]) / diag[0, 0]),
            "includes": "sph_create (upload, sort, normals) + steps x (sph_step_async + "
                        "sph_diagnostics_async D2H of 8 doubles into a pinned ring) + sph_sync + "
                        "sph_get_state(HOST)"}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.adjoint_only:
        import torch
        from paper_2110_02621_gb300 import build
        build.build()
        torch.cuda.set_device(0)
        print(json.dumps({"adjoint": adjoint_block(torch.cuda.current_stream())}), flush=True)
        return 0
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
