#!/usr/bin/env python
"""Benchmark: particle-pair interactions/s and steps/s of the SPH advection-dispersion step.

A *step* is one predictor-corrector step (Eq. 8-9) of the whole hot path on one plume: cell-key
hash, radix sort, reorder and cell table, the rate evaluation at level l with the fused predictor,
the rate evaluation at level l+1/2 with the fused corrector and the FP64 reductions.  An
*interaction* is one ordered in-support pair (b != a, |x_ab| < H) evaluated once; a step evaluates
2 x pairs.  Inputs are synthetic and seeded (inputs.py): the default workload is the largest
single-GPU configuration, the 3D plume on a 128^3 lattice in the unit cube (2,097,152 particles,
h = 2 dx, about 250 neighbours, flow along the diagonal); --workload selects the others (the 2D
convergence ladder, the batched plumes, the sweep, the adjoint, paper scale).  The L2 cache is
flushed (256 MiB write) before every timed step.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload W]
Under torchrun (N > 1) every rank runs an independent replica of the workload (the single-plume
path has no exchange step); value = all ranks' interactions / max-over-ranks time.
``--impl reference`` times the FP64 CPU oracle on the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import csv
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2108_09488_gb300 import inputs, sharding  # noqa: E402

WORKLOADS = {
    "ladder-1024-n120-r10": lambda: inputs.ladder_2d(1024, 10),
    "ladder-512-n60-r10": lambda: inputs.ladder_2d(512, 10),
    "ladder-256-n28-r10": lambda: inputs.ladder_2d(256, 10),
    "lattice-64-h1.3": inputs.lattice_2d_64,
    "cube-128-h2": inputs.cube_3d_128,
    "field-1024-n120-r10": lambda: inputs.ladder_2d(1024, 10),   # + per-particle velocity field
    # Table 1 resolutions of the Sec. 3 test model (C4, support h, irregular particles)
    "paper-1m-n31k-c4": lambda: inputs.paper_plume(1000, 0.1),
    "paper-2m-n50k-c4": lambda: inputs.paper_plume(1414, 0.1),
    "paper-4m-n80k-c4": lambda: inputs.paper_plume(2000, 0.1),
    "batched-64": None,          # 64 uneven 2D plumes in one batch (inputs.batched_2d)
    "sweep-512-8": None,         # 8 dispersivity sets on the 512^2 rung sharing one cell list
    "cattaneo-1024-n120-r10": lambda: inputs.ladder_2d(1024, 10),   # Eq. 14 with tau = 2 dt
    "adjoint-512": None,         # gradient of the misfit: 512^2, 400 steps, checkpoints every 40
}
# velocity-field workloads: vmax of the smooth seeded field (inputs.velocity_field, speed 0.1,
# relative amplitude 0.5, so max |v| ~ 0.17)
FIELD_VMAX = {"field-1024-n120-r10": 0.2}
# dispersivity sweep: alpha_T = 1e-3, alpha_L / alpha_T = 1 .. 100, D_m = 1e-6, on the 512^2 rung
SWEEP_RATIOS = (1, 2, 5, 10, 20, 30, 50, 100)
# minimum FP32-pipe instructions of the sweep kernel: 12 per pair for the shared geometry
# (separation, r^2, r, 1 - q, f, u = (vhat . e)^2) and 4 per pair and set (a u + b, f s, C_a - C_b,
# accumulation)
SWEEP_GEOM, SWEEP_PER_SET = 12, 4
ADJ_THETA = (1e-2, 1e-3, 1e-6)
ADJ_THETA_STAR = (2e-2, 2e-3, 1e-6)
ADJ_STEPS, ADJ_CKPT = 400, 40


def adjoint_plume():
    return inputs.Plume(dim=2, side=512, h_over_dx=1.3, alpha_L=ADJ_THETA[0], alpha_T=ADJ_THETA[1],
                        D_m=ADJ_THETA[2], name="2d-512^2-h1.3dx-adjoint-400steps")
DEFAULT_WORKLOAD = "cube-128-h2"
METRIC = "particle-pair interactions/s"
UNIT = "interactions/s"

# ALU roof of the uniform-D pair term: instructions per in-support ordered pair issued to the
# FP32 lanes (SMs x 128 lanes x clock / count pairs per second).  I_PAIR is the per-pair count of
# the scope table the measurement is defined against (2D 20, 3D 26: the separation from the
# fixed-point words, r^2, r, 1 - q, the kernel shape, the pair factor of Eq. 5, the weight,
# C_a - C_b and the accumulation); I_FP32 is the FP32 arithmetic alone of the form the kernels
# evaluate (2D 14, 3D 16: r^2 2/3, 1 - q 2, its clamp 1, the dot product (sqrt|a| vhat . x) 2/3,
# its product with 1/r 1, t^2 + b 1, the shape 2, the weight 1, C_a - C_b 1, the accumulation 1),
# a stricter floor that leaves out the integer separations and their conversion to FP32.
I_PAIR = {2: 20, 3: 26}
I_FP32 = {2: 14, 3: 16}
# Velocity-field pair term (per-particle D, harmonic means, convective term): minimum FP32-pipe
# instructions and MUFU operations (rsqrt + one reciprocal per tensor component) per pair; the
# roof takes the slower of the two pipes (128 FP32 lanes and 16 MUFU lanes per SM).
FIELD_PIPE_COST = {2: (33, 4), 3: (51, 7)}
MUFU_LANES_PER_SM = 16

# DRAM bytes (read + write) per launch of the dominant kernel, mean of one predictor and one
# corrector launch, from the ncu capture summarised in the named profile, keyed by workload and
# walk, with the digest of the kernel sources the capture was taken of: a walk without a capture,
# or whose sources have changed since, reports null traffic.
# The source files each rate kernel is built from: a capture is tied to a digest of its own files.
KERNEL_FILES = {
    "pair": ("rate_pair.cu", "rate_walk.cuh", "rate_common.cuh", "ade_internal.h"),
    "batch": ("rate.cu", "rate_walk.cuh", "rate_common.cuh", "ade_internal.h"),
    "field": ("rate_field.cu", "rate_common.cuh", "ade_internal.h"),
    "sweep": ("sweep.cu", "rate_common.cuh", "ade_internal.h"),
}
# (workload, walk) -> (DRAM bytes read + written per launch, mean of one predictor and one corrector
# from an ncu --set full capture, the profile that records it, kernel family, digest of its files)
TRAFFIC_PER_LAUNCH = {
    ("cube-128-h2", "direct-branch-free-trimmed-paired"): (53.62e6, "profiles/k_rate_cube128.md", "pair", "dd0f33488e40561a"),
    ("ladder-1024-n120-r10", "direct-branch-free-trimmed-paired"): (25.13e6, "profiles/k_rate_ladder1024.md", "pair",
                                                              "dd0f33488e40561a"),
    ("batched-64", None): (42.19e6, "profiles/k_rate_batch_batched64.md", "batch", "f85a9b4952214a0c"),
    ("paper-1m-n31k-c4", "direct-branch-free-trimmed-paired"): (16.09e6, "profiles/k_rate_paper1m.md", "pair",
                                                          "dd0f33488e40561a"),
    ("field-1024-n120-r10", "velocity-field-direct"): (82.34e6, "profiles/k_rate_field_field1024.md", "field",
                                                       "33d53e1a706f6232"),
    ("sweep-512-8", None): (18.25e6, "profiles/k_rate_sweep_sweep512.md", "sweep", "3fed28905bd475a7"),
}


def kernel_digest(family="pair"):
    """Digest of one rate kernel family's source files (ties a traffic capture to a kernel revision)."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_FILES[family]:
        with open(os.path.join(ROOT, "paper_2108_09488_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_entry(workload, walk):
    """(bytes per launch or None, source note) for the roofline line."""
    e = TRAFFIC_PER_LAUNCH.get((workload, walk))
    if e is None or e[0] is None:
        return None, "no ncu capture of this walk on this workload"
    nbytes, profile, family, digest = e
    if digest != kernel_digest(family):
        return None, f"stale: the kernel sources changed since the capture in {profile}"
    return nbytes, f"{profile} (kernel sources {digest})"


# interaction walks (ade flags) selectable with --variant; "auto" autotunes grid and walk
VARIANT_FLAGS = {"direct-branch-free": 1, "tiled": 2, "direct-branched": 4,
                 "direct-branch-free-trimmed": 9, "direct-branched-trimmed": 12,
                 "direct-branch-free-paired": 17, "direct-branch-free-trimmed-paired": 25,
                 "direct-branched-paired": 20, "direct-branched-trimmed-paired": 28}
VARIANT_NAMES = {0: "direct-branch-free", 1: "tiled", 2: "direct-branched", 3: "direct-branch-free-trimmed",
                 4: "direct-branched-trimmed", 5: "direct-branch-free-paired",
                 6: "direct-branch-free-trimmed-paired", 7: "direct-branched-paired",
                 8: "direct-branched-trimmed-paired"}
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 256 << 20


# ---------------------------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    def __init__(self, world, use_cuda):
        self.world = world
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("nccl" if use_cuda else "gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x, device):
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for r in csv.reader(f):
                if len(r) >= 10:
                    rows.append([c.strip() for c in r])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(s):
            try:
                return float(s)
            except ValueError:
                return float("nan")
        load = [r for r in rows if num(r[4]) >= 50.0] or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[6 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(num(r[1]) for r in load),
                "sm_max_mhz": max(num(r[2]) for r in rows),
                "power_w_max": max(num(r[3]) for r in rows),
                "samples": len(rows), "samples_under_load": len(load), "reasons": reasons}


# ---------------------------------------------------------------------------------------------
def field_setup(workload, plume, xq):
    """(velocity field float32 [dim][n], vmax, plume renamed) of a velocity-field workload, or
    (None, 0, plume)."""
    import dataclasses
    vmax = FIELD_VMAX.get(workload)
    if vmax is None:
        return None, 0.0, plume
    v = inputs.velocity_field(inputs.from_fixed(xq, plume.boxv), plume.boxv)
    return v, vmax, dataclasses.replace(plume, name=f"{plume.name}-velocity-field-vmax{vmax}")


def oracle_sample(plume, requested):
    """Particles the CPU oracle evaluates per rate evaluation: the requested sample, capped at
    about 2e8 pairs (about a second of FP64 work on the host cores) for wide kernels."""
    neighbours = max(sharding.plume_cost(plume) / plume.n, 1.0)
    return int(max(256, min(requested, 2e8 / neighbours, plume.n)))


def cpu_oracle_rate(plume, xq, C, sample, min_seconds, max_steps=None, v=None):
    """Time the FP64 oracle: each step evaluates Eq. 4 twice (predictor and corrector
    evaluation) for a fixed random sample of particles.  Returns (interactions/s, steps, secs).
    v: per-particle velocities (float32 [dim][n]) of a velocity-field workload."""
    import oracle
    oracle.build()
    x = inputs.from_fixed(xq, plume.boxv)
    Cd = np.asarray(C, dtype=np.float64)
    sel = np.sort(np.random.default_rng(12345).choice(plume.n, min(sample, plume.n), replace=False))
    vel = plume.velocity if v is None else np.ascontiguousarray(v.T, dtype=np.float64)
    args = (vel, Cd, plume.mass, plume.rho, plume.boxv, plume.kernel, plume.support,
            plume.dim + 2.0, plume.alpha_L, plume.alpha_T, plume.D_m)
    pairs = 0
    steps = 0
    t0 = time.perf_counter()
    while True:
        for _ in range(2):
            _, p = oracle.rate_at(sel, x, *args)
            pairs += p
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and steps >= max_steps) or (max_steps is None and el >= min_seconds):
            break
    return pairs / el, steps, el, int(sel.size)


def host_cpu_model():
    """CPU model string of this host (for the CPU-baseline record)."""
    import platform
    try:
        fields = {}
        for line in open("/proc/cpuinfo"):
            if ":" in line:
                k, v = line.split(":", 1)
                fields.setdefault(k.strip(), v.strip())
        name = fields.get("model name") or fields.get("Model") or (
            f"implementer {fields.get('CPU implementer', '?')} part {fields.get('CPU part', '?')}")
    except OSError:
        name = platform.processor() or "unknown"
    return f"{name} ({platform.machine()})"


def single_core_baseline(plume, xq, C, sample, seconds=3.0, v=None):
    """The oracle on one host thread (a smaller sample), next to the all-core figure."""
    import oracle
    oracle.build()
    threads = oracle.max_threads()
    oracle.set_threads(1)
    try:
        value, steps, secs, ns = cpu_oracle_rate(plume, xq, C, max(256, sample // 16), seconds, v=v)
    finally:
        oracle.set_threads(threads)
    return {"value": value, "unit": UNIT, "cores": 1,
            "sample": f"Eq. 4 evaluated twice per step on {ns} particles; {steps} steps in {secs:.1f} s"}


def cpu_oracle_batch(plumes, states, per_plume, min_seconds, max_steps=None):
    """Oracle timing for a batch: Eq. 4 twice per step on a fixed sample of each plume."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(12345)
    prepared = []
    for p, (xq, C) in zip(plumes, states):
        sel = np.sort(rng.choice(p.n, min(per_plume, p.n), replace=False))
        args = (p.velocity, np.asarray(C, dtype=np.float64), p.mass, p.rho, p.boxv, p.kernel,
                p.support, p.dim + 2.0, p.alpha_L, p.alpha_T, p.D_m)
        prepared.append((sel, inputs.from_fixed(xq, p.boxv), args))
    pairs = steps = 0
    t0 = time.perf_counter()
    while True:
        for sel, x, args in prepared:
            for _ in range(2):
                pairs += oracle.rate_at(sel, x, *args)[1]
        steps += 1
        el = time.perf_counter() - t0
        if (max_steps is not None and steps >= max_steps) or (max_steps is None and el >= min_seconds):
            break
    return pairs / el, steps, el, sum(int(p[0].size) for p in prepared)


def batched_config(plumes):
    return {"workload": "batched-2d-64-plumes-seed20210821", "plumes": len(plumes),
            "particles": int(sum(p.n for p in plumes)), "dim": 2, "kernel": "wendland-c2",
            "side_range": [min(p.side for p in plumes), max(p.side for p in plumes)],
            "l2": "flushed (256 MiB write) before every timed step"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload == "batched-64":
        plumes = inputs.batched_2d()
        states = [p.initial_state() for p in plumes]
        cpu_oracle_batch(plumes, states, args.cpu_sample // 64, 0.0, max_steps=args.warmup)
        value, steps, secs, ns = cpu_oracle_batch(plumes, states, args.cpu_sample // 64, 0.0,
                                                  max_steps=args.steps)
        line = {
            "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": batched_config(plumes),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"Eq. 4 evaluated twice per step on {ns} particles sampled "
                                       f"across the 64 plumes"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        }
        print(json.dumps(line))
        return 0
    if args.workload == "adjoint-512":
        plume = adjoint_plume()
    elif args.workload == "sweep-512-8":
        plume = sweep_setup()[0]          # the oracle evaluates one set at a time
    else:
        plume = WORKLOADS[args.workload]()
    xq, C = plume.initial_state()
    v, _, plume = field_setup(args.workload, plume, xq)
    sample = oracle_sample(plume, args.cpu_sample)
    cpu_oracle_rate(plume, xq, C, sample, 0.0, max_steps=args.warmup, v=v) if args.warmup else None
    value, steps, secs, ns = cpu_oracle_rate(plume, xq, C, sample, 0.0, max_steps=args.steps, v=v)
    cores = os.cpu_count()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / max(steps, 1),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(plume),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "cpu_model": host_cpu_model(),
                         "sample": f"Eq. 4 evaluated twice per step on {ns} of {plume.n} particles"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def workload_config(plume):
    return {"workload": plume.name, "particles": plume.n, "dim": plume.dim,
            "kernel": "wendland-c2" if plume.kernel == inputs.WENDLAND_C2 else "wendland-c4",
            "support_over_dx": round(plume.support / plume.dx, 6),
            "alpha_L_over_alpha_T": round(plume.alpha_L / plume.alpha_T, 6),
            "l2": "flushed (256 MiB write) before every timed step"}


def run_batched(args):
    """64 uneven plumes in one batch (autotuned, graph replay) against one context per plume."""
    import torch

    from paper_2108_09488_gb300 import ade

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = Dist(world, True)
    all_plumes = inputs.batched_2d()
    # independent plumes: whole plumes are sharded over ranks (no collective on the data path)
    mine = sharding.shard_plumes([sharding.plume_cost(p) for p in all_plumes], world)[rank]
    plumes = [all_plumes[i] for i in mine]
    states = [p.initial_state() for p in plumes]
    plist = [ade.params_for(p) for p in plumes]
    b = ade.Batch(plist, [s[0] for s in states], [s[1] for s in states], device=device)
    pairs = b.count_pairs()
    tune_ms = b.autotune()
    info0 = b.plume_info(0)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    for _ in range(args.warmup):
        flush.zero_()
        b.step_timed()
    torch.cuda.synchronize()
    dist.barrier()
    stream = torch.cuda.current_stream(device)
    for _ in range(args.warmup):
        flush.zero_()
        b.run(1)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    # the timed steps: one graph replay of the whole batched step (ade_batch_run) per step,
    # bracketed by events, the L2 flush outside; per-phase times from ade_batch_step_timed
    marks = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(1)
        e1.record(stream)
        marks.append((e0, e1))
    phases = []
    for _ in range(args.steps):
        flush.zero_()
        phases.append(b.step_timed())
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    agg_dev = device if world > 1 else None
    value, total_ms, all_units = sharding.aggregate(2.0 * pairs * args.steps,
                                                    sum(a.elapsed_time(z) for a, z in marks), device=agg_dev)

    # the same plumes as 64 separate contexts (same cell subdivision), one graph launch each
    sims = [ade.Simulation(ade.params_for(p, cell_subdiv=b.plume_info(i).cell_subdiv,
                                          flags=ade.FLAG_DIRECT), *states[i], device=device)
            for i, p in enumerate(plumes)]
    for _ in range(args.warmup):
        flush.zero_()
        for sm in sims:
            sm.run(1, stats=False)
    torch.cuda.synchronize()
    pp_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sm in sims:
            sm.run(1, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        pp_ms += e0.elapsed_time(e1)
    pp_value, pp_ms, _ = sharding.aggregate(2.0 * pairs * args.steps, pp_ms, device=agg_dev)
    pp_launches = sum(ade.launches_per_step(sm.ctx) for sm in sims)
    for sm in sims:
        sm.close()

    rate_ms = [p[1] for p in phases] + [p[2] for p in phases]
    rate_avg_ms = sum(rate_ms) / len(rate_ms)
    props = torch.cuda.get_device_properties(device)
    f_max = clk.get("sm_max_mhz") or 2070.0
    peak = props.multi_processor_count * FP32_LANES_PER_SM * f_max * 1e6 / I_PAIR[2] / 1e9
    achieved = pairs / (rate_avg_ms * 1e-3) / 1e9
    traffic, tsrc = traffic_entry("batched-64", None)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": tsrc,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "kernel": "k_rate_batch (predictor + corrector)",
                "peak_basis": f"{props.multi_processor_count} SMs x {FP32_LANES_PER_SM} FP32 lanes x "
                              f"{f_max:.0f} MHz / {I_PAIR[2]} instructions per pair",
                "frac_fp32_floor": achieved / (peak * I_PAIR[2] / I_FP32[2]),
                "rate_kernel_ms": rate_avg_ms,
                "phase_ms_per_step": {k: sum(p[i] for p in phases) / len(phases)
                                      for i, k in enumerate(("cells", "predictor", "corrector"))}}

    # end to end: H2D of every plume's x and C, one graph-replayed step, D2H of C; as for the
    # single plume, a second batch given the first one's autotuned configuration alternates with
    # it so that one's copies (on their own streams) overlap the other's step
    xq_pin = b.xq.cpu().pin_memory()
    C_pin = b.C.cpu().pin_memory()
    C_out = torch.empty_like(C_pin).pin_memory()
    b2 = ade.Batch(plist, [s_[0] for s_ in states], [s_[1] for s_ in states], device=device)
    b2.set_config(b.config())
    batches = (b, b2)
    h2d, d2h = torch.cuda.Stream(device), torch.cuda.Stream(device)
    ev = {k: [torch.cuda.Event() for _ in batches] for k in ("in", "ran", "out")}
    for e in ev["out"]:
        e.record(d2h)

    def e2e_step(k):
        q, bx = k % 2, batches[k % 2]
        h2d.wait_event(ev["out"][q])
        with torch.cuda.stream(h2d):
            bx.xq.copy_(xq_pin, non_blocking=True)
            bx.C.copy_(C_pin, non_blocking=True)
        ev["in"][q].record(h2d)
        stream.wait_event(ev["in"][q])
        with torch.cuda.stream(stream):
            bx.run(1)
        ev["ran"][q].record(stream)
        d2h.wait_event(ev["ran"][q])
        with torch.cuda.stream(d2h):
            C_out.copy_(bx.C, non_blocking=True)
        ev["out"][q].record(d2h)

    for k in range(max(args.warmup, 1)):
        e2e_step(k)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d.wait_stream(stream)
    d2h.wait_stream(stream)
    for k in range(args.steps):
        e2e_step(k)
    stream.wait_stream(d2h)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, e2e_ms, _ = sharding.aggregate(2.0 * pairs * args.steps, e0.elapsed_time(e1), device=agg_dev)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(xq_pin.numel() * 4 + C_pin.numel() * 4),
           "d2h_bytes_per_step": int(C_out.numel() * 4), "ms_per_step": e2e_ms / args.steps,
           "path": "ade_batch_run (graph replay) via ctypes; two batches of one configuration "
                   "alternate, H2D and D2H on their own streams overlapping the other batch's step"}
    b2.close()
    ms_per_step = total_ms / args.steps
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": batched_config(all_plumes),
        "timing": "CUDA events around one graph replay (ade_batch_run) per step; per-phase times from "
                  "ade_batch_step_timed",
        "batch": {"autotune_best_ms": tune_ms, "paired_walk": bool(b.config()[3]),
                  "work_item_particles": info0.tile[0],
                  "persistent_grid": info0.tile[1], "work_items": info0.tile[2],
                  "cell_subdiv": [b.plume_info(i).cell_subdiv for i in range(len(plumes))]},
        "per_plume_launches": {"value": pp_value, "ms_per_step": pp_ms / args.steps,
                               "launches_per_step": pp_launches,
                               "batched_speedup": value / pp_value},
        "steps_per_s": 1e3 / ms_per_step, "interactions_per_step": all_units / args.steps,
        "roofline": roofline, "e2e": e2e, "clocks": clk,
        "cell_build": cell_build_roof(sum(b.ns), sum(b.plume_info(i).ncells for i in range(len(plumes))), 2,
                                      roofline["phase_ms_per_step"]["cells"]),
        "gpu_launches": b.launches_per_step() * args.steps,
        "shard": {"rank0_plumes": len(mine), "ranks": world},
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, steps, secs, ns = cpu_oracle_batch(plumes, states, args.cpu_sample // 64, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"Eq. 4 evaluated twice per step on {ns} particles sampled "
                                          f"across the 64 plumes; {steps} steps in {secs:.1f} s"}
    b.close()
    if rank == 0:
        print(json.dumps(line))
    dist.close()
    return 0


def run_adjoint(args):
    """One bench step = one gradient evaluation: the 400-step forward run with checkpoints and the
    adjoint sweep (ade_adjoint).  Interactions counted: pair evaluations of every operator
    application (forward 2 per step, recomputation 2 per step except each segment's last, backward
    2 three-output and 2 single applications per step)."""
    import torch

    from paper_2108_09488_gb300 import ade

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = Dist(world, True)
    p = adjoint_plume()
    xq, C = p.initial_state()
    sim = ade.Simulation(ade.params_for(p), xq, C, device=device)
    pairs = sim.count_pairs()
    # target: the same run with theta* (generated here on the GPU; the tests generate it with the
    # oracle at smaller sizes)
    sim.set_dispersivity(*ADJ_THETA_STAR)
    _, _, _, target = sim.adjoint(np.zeros(p.n, np.float32), ADJ_STEPS, ADJ_CKPT, want_dC0=False,
                                  want_final=True)
    target = target.clone()
    sim.set_dispersivity(*ADJ_THETA)
    passes = 2 * ADJ_STEPS + 2 * (ADJ_STEPS - ADJ_STEPS // ADJ_CKPT) + 4 * ADJ_STEPS
    for _ in range(args.warmup):
        sim.adjoint(target, ADJ_STEPS, ADJ_CKPT)
    torch.cuda.synchronize()
    dist.barrier()
    stream = torch.cuda.current_stream(device)
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        J, g, _, _ = sim.adjoint(target, ADJ_STEPS, ADJ_CKPT)
    e1.record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    ms = dist.max(e0.elapsed_time(e1), device) / args.steps
    value = world * passes * pairs / (ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": p.name, "particles": p.n, "time_steps": ADJ_STEPS,
                   "checkpoint_every": ADJ_CKPT, "theta": ADJ_THETA, "theta_star": ADJ_THETA_STAR,
                   "step": "one gradient evaluation (forward + adjoint)"},
        "gradient": {"J": J, "dJ_dalpha_L": g[0], "dJ_dalpha_T": g[1], "dJ_dD_m": g[2]},
        "interactions_per_step": passes * pairs, "clocks": clk,
        # cell build (6) and set-up gathers (3); forward 2 per step; recomputation 2 per step but
        # each segment's last; backward 4 applications and 1 dot-product kernel per step
        "gpu_launches": args.steps * (9 + 2 * ADJ_STEPS + 2 * (ADJ_STEPS - ADJ_STEPS // ADJ_CKPT)
                                      + 5 * ADJ_STEPS),
    }
    if rank == 0:
        print(json.dumps(line))
    dist.close()
    return 0


def hbm_peak_gbs():
    """HBM copy bandwidth measured on this machine's GPUs (MEASURED_PEAKS.json), else 6800 GB/s."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs, a device copy)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6800 GB/s"


def cell_build_roof(n, ncells, dim, cells_ms):
    """The cell build against HBM bandwidth.  Algorithmic bytes per particle: k_count reads the dim
    position words and writes key and rank (4 dim + 8); k_place reads key and rank, gathers the
    cell's start and writes the provisional slot (16); k_order reads that slot, gathers the position
    words and C and writes the permutation and the 16-byte sorted record (4 dim + 28).  Per cell:
    the counting atomics read and write the count (8), the scan reads it, clears it and writes the
    start (12), k_order reads the start (4)."""
    nbytes = n * (8 * dim + 52) + ncells * 24
    gbs = nbytes / (cells_ms * 1e-3) / 1e9
    peak, src = hbm_peak_gbs()
    return {"bound": "hbm", "bytes_per_build": nbytes, "ms": cells_ms, "achieved": gbs, "peak": peak,
            "unit": "GB/s", "frac": gbs / peak, "peak_source": src,
            "bytes_basis": "n (8 dim + 52) + 24 ncells"}


def measured_alu_roof(ade, dim, field, achieved, sms):
    """The pair roof re-derived from the FFMA and MUFU.RSQ issue rates measured on this device
    (ade_alu_peaks, outside the timed region)."""
    ffma, rsq = ade.alu_peaks()
    if field:
        n32, nmufu = FIELD_PIPE_COST[dim]
        roof = min(ffma / n32, rsq / nmufu) / 1e9
    else:
        n32, nmufu = I_PAIR[dim], 1
        roof = min(ffma / n32, rsq / nmufu) / 1e9
    return {"ffma_per_s": ffma, "rsqrt_per_s": rsq,
            "ffma_per_sm_per_ns": ffma / sms / 1e9, "rsqrt_per_sm_per_ns": rsq / sms / 1e9,
            "pair_roof": roof, "unit": "Gpair/s", "frac": achieved / roof,
            "basis": f"min(FFMA/s / {n32}, RSQRT/s / {nmufu}) per pair"}


def sweep_setup():
    plume = inputs.ladder_2d(512, 10)
    theta = np.array([[1e-3 * r, 1e-3, 1e-6] for r in SWEEP_RATIOS])
    return plume, theta


def run_sweep(args):
    """8 dispersivity sets on one 512^2 plume in one sweep, against one context per set."""
    import torch

    from paper_2108_09488_gb300 import ade

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = Dist(world, True)
    plume, theta = sweep_setup()
    P = len(theta)
    xq, C = plume.initial_state()
    sw = ade.Sweep(ade.params_for(plume), xq, np.broadcast_to(C, (P, plume.n)), theta, device=device)
    pairs = sw.count_pairs()
    units_per_step = 2.0 * pairs * P          # every set evaluates every pair twice per step
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    for _ in range(args.warmup):
        flush.zero_()
        sw.step_timed()
    torch.cuda.synchronize()
    dist.barrier()
    stream = torch.cuda.current_stream(device)
    for _ in range(args.warmup):
        flush.zero_()
        sw.run(1)
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    # the timed steps: one graph replay of the whole sweep step (ade_sweep_run) per step,
    # bracketed by events, the L2 flush outside; per-phase times from ade_sweep_step_timed
    marks = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sw.run(1)
        e1.record(stream)
        marks.append((e0, e1))
    phases = []
    for _ in range(args.steps):
        flush.zero_()
        phases.append(sw.step_timed())
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    agg_dev = device if world > 1 else None
    value, total_ms, _ = sharding.aggregate(units_per_step * args.steps, sum(a.elapsed_time(z) for a, z in marks),
                                            device=agg_dev)
    ms_per_step = total_ms / args.steps

    # the same sets as P single-plume contexts (same dt and grid), one graph launch each
    sims = [ade.Simulation(ade.params_for(plume, alpha_L=t[0], alpha_T=t[1], D_m=t[2], dt=sw.info.dt,
                                          cell_subdiv=sw.info.cell_subdiv, flags=ade.FLAG_DIRECT),
                           xq, C, device=device) for t in theta]
    for _ in range(args.warmup):
        flush.zero_()
        for sm in sims:
            sm.run(1, stats=False)
    torch.cuda.synchronize()
    ps_ms = 0.0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for sm in sims:
            sm.run(1, stats=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ps_ms += e0.elapsed_time(e1)
    ps_value, ps_ms, _ = sharding.aggregate(units_per_step * args.steps, ps_ms, device=agg_dev)
    for sm in sims:
        sm.close()

    rate_ms = (sum(p[1] for p in phases) + sum(p[2] for p in phases)) / (2 * len(phases))
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    f_max = clk.get("sm_max_mhz") or 2070.0
    per_set = SWEEP_PER_SET + SWEEP_GEOM / P
    peak = sms * FP32_LANES_PER_SM * f_max * 1e6 / per_set / 1e9
    achieved = pairs * P / (rate_ms * 1e-3) / 1e9
    traffic, tsrc = traffic_entry("sweep-512-8", None)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair-sets/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": tsrc,
                "traffic_unit": "bytes per evaluation (ncu dram read + write, all groups)",
                "kernel": "k_rate_sweep (predictor + corrector, one group of 8 sets)",
                "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {f_max:.0f} MHz / "
                              f"({SWEEP_PER_SET} + {SWEEP_GEOM}/{P}) FP32-pipe instructions per pair and set",
                "rate_evaluation_ms": rate_ms,
                "phase_ms_per_step": {k: sum(p[i] for p in phases) / len(phases)
                                      for i, k in enumerate(("cells", "predictors", "correctors"))}}
    roofline["measured_alu"] = {"ffma_per_s": ade.alu_peaks()[0]}
    roofline["measured_alu"]["pair_set_roof"] = roofline["measured_alu"]["ffma_per_s"] / per_set / 1e9
    roofline["measured_alu"]["frac"] = achieved / roofline["measured_alu"]["pair_set_roof"]

    # end to end: H2D of x and the P fields, one graph-replayed step, D2H of the P fields; as for
    # the single plume, two sweeps of the same configuration alternate so that one's copies (on
    # their own streams) overlap the other's step
    xq_pin = sw.xq.cpu().pin_memory()
    C_pin = sw.C.cpu().pin_memory()
    C_out = torch.empty_like(C_pin).pin_memory()
    sw2 = ade.Sweep(ade.params_for(plume), xq, np.broadcast_to(C, (P, plume.n)), theta, device=device)
    assert sw2.info.cell_subdiv == sw.info.cell_subdiv and sw2.info.dt == sw.info.dt
    sweeps = (sw, sw2)
    h2d, d2h = torch.cuda.Stream(device), torch.cuda.Stream(device)
    ev = {k: [torch.cuda.Event() for _ in sweeps] for k in ("in", "ran", "out")}
    for e in ev["out"]:
        e.record(d2h)

    def e2e_step(k):
        q, sx = k % 2, sweeps[k % 2]
        h2d.wait_event(ev["out"][q])
        with torch.cuda.stream(h2d):
            sx.xq.copy_(xq_pin, non_blocking=True)
            sx.C.copy_(C_pin, non_blocking=True)
        ev["in"][q].record(h2d)
        stream.wait_event(ev["in"][q])
        with torch.cuda.stream(stream):
            sx.run(1)
        ev["ran"][q].record(stream)
        d2h.wait_event(ev["ran"][q])
        with torch.cuda.stream(d2h):
            C_out.copy_(sx.C, non_blocking=True)
        ev["out"][q].record(d2h)

    for k in range(max(args.warmup, 1)):
        e2e_step(k)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h2d.wait_stream(stream)
    d2h.wait_stream(stream)
    for k in range(args.steps):
        e2e_step(k)
    stream.wait_stream(d2h)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_value, e2e_ms, _ = sharding.aggregate(units_per_step * args.steps, e0.elapsed_time(e1), device=agg_dev)
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(xq_pin.numel() * 4 + C_pin.numel() * 4),
           "d2h_bytes_per_step": int(C_out.numel() * 4), "ms_per_step": e2e_ms / args.steps,
           "path": "ade_sweep_run (graph replay) via ctypes; two sweeps alternate, H2D and D2H on their "
                   "own streams overlapping the other sweep's step"}
    sw2.close()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**workload_config(plume), "workload": f"sweep-{plume.name}-{P}-sets",
                   "sets": P, "alpha_L_over_alpha_T": list(SWEEP_RATIOS), "interaction": "one pair for one set"},
        "timing": "CUDA events around one graph replay (ade_sweep_run) per step; per-phase times from "
                  "ade_sweep_step_timed",
        "grid": {"cell_subdiv": sw.info.cell_subdiv, "cells": sw.info.ncells, "dt": sw.info.dt,
                 "launches_per_evaluation": sw.info.tile[0]},
        "per_set_contexts": {"value": ps_value, "ms_per_step": ps_ms / args.steps,
                             "sweep_speedup": value / ps_value},
        "steps_per_s": 1e3 / ms_per_step * world, "interactions_per_step": units_per_step,
        "roofline": roofline, "e2e": e2e, "clocks": clk,
        "gpu_launches": sw.launches_per_step() * args.steps,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cv, steps, secs, ns = cpu_oracle_rate(plume, xq, C, oracle_sample(plume, args.cpu_sample // P),
                                              args.cpu_seconds)
        line["cpu_baseline"] = {"value": cv, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"Eq. 4 evaluated twice per step for one set on {ns} of "
                                          f"{plume.n} particles; {steps} steps in {secs:.1f} s "
                                          "(the oracle evaluates each set separately)"}
    sw.close()
    if rank == 0:
        print(json.dumps(line))
    dist.close()
    return 0


def closed_form_images(plume, t):
    """Periodic image shells of the closed form at time t: every omitted image lies more than 12
    plume widths away (width^2 = w^2 + 2 lambda_max t, lambda_max = max(alpha_L, alpha_T)|v| + D_m)."""
    import math
    lam = max(plume.alpha_L, plume.alpha_T) * plume.speed + plume.D_m
    sigma = math.sqrt(plume.w ** 2 + 2.0 * lam * t)
    return int(math.ceil(12.0 * sigma / plume.box)) + 1


def accuracy_run(ade, plume, device, steps=None, **over):
    """The configured run of a uniform-velocity plume (steps of Eq. 8-9 from the initial state
    through the library, FP32) and its error against the closed form of Sec. 3 (Eq. 12-13, FP64 on
    the device): L2, Linf, RMSE of C/C0, C_min, C_max and the relative change of sum m C."""
    import torch
    steps = plume.steps if steps is None else steps
    xq, C = plume.initial_state()
    sim = ade.Simulation(ade.params_for(plume, **over), xq, C, device=device)
    m0 = sim.stats().mass
    if steps:
        sim.run(steps, stats=False)
    torch.cuda.synchronize()
    st = sim.stats()
    t = steps * sim.info.dt
    nimg = closed_form_images(plume, t)
    cf = sim.closed_form_error(np.asarray(plume.x0[: plume.dim]), plume.w, plume.C0, nimg=nimg)
    out = {"steps": steps, "t": t, "dt": sim.info.dt, "l2": cf["l2"], "linf": cf["linf"], "rmse": cf["rmse"],
           "c_an_max": cf["c_an_max"], "c_min": st.c_min, "c_max": st.c_max,
           "mass_rel_change": (st.mass - m0) / m0, "closed_form_images": nimg,
           "status": st.status}
    sim.close()
    return out


ACCURACY_CONFIGS = [("lattice-64-h1.3", inputs.lattice_2d_64)] + [
    (f"ladder-{s}-n{inputs.LADDER_NEIGHBOURS[s]}-r{r}", (lambda s=s, r=r: inputs.ladder_2d(s, r)))
    for s in (256, 512, 1024) for r in (1, 10, 100)] + [("cube-128-h2", inputs.cube_3d_128)]


def run_accuracy(args):
    """One JSON line per configured plume: its full run against the closed form (FP32 state,
    FP64 norms); the FP64-oracle drift of the same runs is checked in tests/test_gpu_precision.py."""
    import torch

    from paper_2108_09488_gb300 import ade
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    for name, make in ACCURACY_CONFIGS:
        plume = make()
        acc = accuracy_run(ade, plume, device)
        print(json.dumps({"workload": name, "config": plume.name, "particles": plume.n, "dtype": "f32",
                          "norms": "f64", **acc}), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2108_09488_gb300 import ade

    world, rank, local = dist_env()
    if args.workload == "batched-64":
        return run_batched(args)
    if args.workload == "sweep-512-8":
        return run_sweep(args)
    if args.workload == "adjoint-512":
        return run_adjoint(args)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = Dist(world, True)

    plume = WORKLOADS[args.workload]()
    xq, C = plume.initial_state()
    v, vmax, plume = field_setup(args.workload, plume, xq)
    tau = 0.0
    if args.workload.startswith("cattaneo-"):
        # relaxation time of Eq. 14: twice the parabolic step 0.1 h^2 / lambda_max(D)
        lam = max(plume.alpha_L, plume.alpha_T) * plume.speed + plume.D_m
        tau = 2.0 * 0.1 * plume.h ** 2 / lam
    pinned = args.variant != "auto" or args.cell_subdiv > 0
    if pinned and v is not None and args.variant not in ("auto", "direct-branch-free"):
        raise SystemExit("velocity-field mode has one walk (direct-branch-free)")
    extra = {} if not pinned else {"flags": VARIANT_FLAGS.get(args.variant, 0), "cell_subdiv": args.cell_subdiv}
    sim = ade.Simulation(ade.params_for(plume, vmax=vmax, tau=tau, **extra), xq, C, device=device)
    if v is not None:
        sim.set_velocity_field(v)
    if tau > 0.0:
        sim.set_flux()            # Q(0) = R(C(0)); the flux stays resident between e2e steps
    tune_ms = None if pinned else sim.autotune()
    walk = "velocity-field-direct" if v is not None else VARIANT_NAMES[sim.info.variant]
    pairs = sim.count_pairs()
    launches = ade.launches_per_step(sim.ctx)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)

    stream = torch.cuda.current_stream(device)
    for _ in range(args.warmup):
        flush.zero_()
        sim.run(1, stats=False)
        flush.zero_()
        sim.step_timed()
    torch.cuda.synchronize()
    dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    # the timed steps: one graph replay of the whole step (ade_run: cell build, predictor,
    # corrector, fold of the diagnostics) per step, bracketed by events, the L2 flush outside
    marks = []
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.run(1, stats=False)
        e1.record(stream)
        marks.append((e0, e1))
    # per-phase device times of the same step (events between the phases) for the roofline
    phases = []
    for _ in range(args.steps):
        flush.zero_()
        phases.append(sim.step_timed())
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    step_ms = sum(a.elapsed_time(b) for a, b in marks)

    # replicas: every rank steps its own copy of the plume; all ranks' work / slowest rank's time
    value, total_ms, _ = sharding.aggregate(2.0 * pairs * args.steps, step_ms,
                                            device=device if world > 1 else None)
    ms_per_step = total_ms / args.steps

    # dominant kernel: the rate kernel (predictor and corrector launches)
    rate_ms = [p[1] for p in phases] + [p[2] for p in phases]
    rate_avg_ms = sum(rate_ms) / len(rate_ms)
    props = torch.cuda.get_device_properties(device)
    sms = props.multi_processor_count
    f_max = clk.get("sm_max_mhz") or 2070.0
    if v is None:
        peak = sms * FP32_LANES_PER_SM * f_max * 1e6 / I_PAIR[plume.dim] / 1e9
        basis = (f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x {f_max:.0f} MHz / "
                 f"{I_PAIR[plume.dim]} instructions per pair")
        kname = "k_rate (predictor + corrector)"
    else:
        n32, nmufu = FIELD_PIPE_COST[plume.dim]
        cyc = max(n32 / FP32_LANES_PER_SM, nmufu / MUFU_LANES_PER_SM)
        peak = sms * f_max * 1e6 / cyc / 1e9
        basis = (f"{sms} SMs x {f_max:.0f} MHz / max({n32} FP32-pipe instr / {FP32_LANES_PER_SM} lanes, "
                 f"{nmufu} MUFU ops / {MUFU_LANES_PER_SM} lanes) per pair")
        kname = "k_rate_field (predictor + corrector)"
    achieved = pairs / (rate_avg_ms * 1e-3) / 1e9
    traffic, tsrc = traffic_entry(args.workload, walk)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gpair/s",
                "frac": achieved / peak, "traffic": traffic, "traffic_source": tsrc,
                "traffic_unit": "bytes per launch (ncu dram read + write)",
                "kernel": kname,
                "peak_basis": basis,
                "rate_kernel_ms": rate_avg_ms,
                "phase_ms_per_step": {k: sum(p[i] for p in phases) / len(phases)
                                      for i, k in enumerate(("cells", "predictor", "corrector", "reduce"))}}
    if clk.get("sm_mhz"):
        roofline["frac_at_sampled_clock"] = achieved / (peak * clk["sm_mhz"] / f_max)
    roofline["measured_alu"] = measured_alu_roof(ade, plume.dim, v is not None, achieved, sms)
    if v is None:
        roofline["frac_fp32_floor"] = achieved / (peak * I_PAIR[plume.dim] / I_FP32[plume.dim])

    # end to end through the C ABI with host buffers: every step copies its inputs (x, C) from
    # pinned host memory, runs one graph-replayed step and reads C back.  The steps are independent
    # instances (each starts from the same inputs), so two contexts of the same configuration
    # alternate and the copies of one overlap the other's step: H2D on one copy stream, the step
    # on the compute stream, D2H on a second copy stream, ordered per instance by events.
    xq_pin = torch.from_numpy(np.ascontiguousarray(xq).view(np.int32)).pin_memory()
    C_pin = torch.from_numpy(np.ascontiguousarray(C)).pin_memory()
    C_out = torch.empty_like(C_pin).pin_memory()
    sim2 = ade.Simulation(ade.params_for(plume, vmax=vmax, tau=tau, flags=VARIANT_FLAGS.get(walk, 0)
                                         if v is None else 0, cell_subdiv=sim.info.cell_subdiv),
                          xq, C, device=device)
    if v is not None:
        sim2.set_velocity_field(v)
    if tau > 0.0:
        sim2.set_flux()
    assert sim2.info.variant == sim.info.variant and sim2.info.ncells == sim.info.ncells
    sims = (sim, sim2)
    h2d, d2h = torch.cuda.Stream(device), torch.cuda.Stream(device)
    ev = {k: [torch.cuda.Event() for _ in sims] for k in ("in", "ran", "out")}
    for e in ev["out"]:
        e.record(d2h)

    def e2e_step(k):
        q, sm = k % 2, sims[k % 2]
        h2d.wait_event(ev["out"][q])                 # the slot's previous read-back is done
        with torch.cuda.stream(h2d):
            sm.xq.copy_(xq_pin, non_blocking=True)
            sm.C.copy_(C_pin, non_blocking=True)
        ev["in"][q].record(h2d)
        stream.wait_event(ev["in"][q])
        with torch.cuda.stream(stream):
            sm.run(1, stats=False)
        ev["ran"][q].record(stream)
        d2h.wait_event(ev["ran"][q])
        with torch.cuda.stream(d2h):
            C_out.copy_(sm.C, non_blocking=True)
        ev["out"][q].record(d2h)

    for k in range(max(args.warmup, 1)):
        e2e_step(k)
    torch.cuda.synchronize()
    dist.barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    h2d.wait_stream(stream)
    d2h.wait_stream(stream)
    for k in range(args.steps):
        e2e_step(k)
    stream.wait_stream(d2h)
    ev1.record(stream)
    torch.cuda.synchronize()
    e2e_value, e2e_ms, _ = sharding.aggregate(2.0 * pairs * args.steps, ev0.elapsed_time(ev1),
                                              device=device if world > 1 else None)
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(xq_pin.numel() * 4 + C_pin.numel() * 4),
           "d2h_bytes_per_step": int(C_out.numel() * 4),
           "ms_per_step": e2e_ms / args.steps,
           "path": "ade_run (graph replay) via ctypes; two contexts alternate, H2D and D2H on their "
                   "own streams overlapping the other context's step"}
    sim2.close()

    line_extra = {}
    # a whole run of consecutive steps through one ade_run call (graph replays of 32 steps each,
    # no gap between them; L2 flushed once before the run): steps per second of a simulation
    run_steps = 256 if plume.n <= (1 << 22) else 32
    flush.zero_()
    r0 = torch.cuda.Event(enable_timing=True)
    r1 = torch.cuda.Event(enable_timing=True)
    sim.run(run_steps, stats=False)              # graphs captured outside the timed region
    torch.cuda.synchronize()
    flush.zero_()
    r0.record(stream)
    sim.run(run_steps, stats=False)
    r1.record(stream)
    torch.cuda.synchronize()
    run_ms = r0.elapsed_time(r1)
    line_extra["graph_run"] = {"steps": run_steps, "ms": run_ms, "steps_per_s": 1e3 * run_steps / run_ms,
                               "interactions_per_s": 2.0 * pairs * run_steps / (run_ms * 1e-3),
                               "how": "one ade_run call of consecutive steps (graphs of 32 steps), "
                                      "CUDA events around it, L2 flushed before"}
    if v is None and tau == 0.0 and not args.workload.startswith("paper-") and not args.no_accuracy:
        # the configured run of this plume against the closed form (untimed)
        line_extra["accuracy"] = accuracy_run(ade, plume, device, flags=VARIANT_FLAGS.get(walk, 0),
                                              cell_subdiv=sim.info.cell_subdiv)
    if args.workload.startswith("paper-"):
        N = 4000000 if plume.n > 3000000 else (2000000 if plume.n > 1500000 else 1000000)
        line_extra["paper_context"] = {
            "paper_cpu_time_s": inputs.PAPER_CPU_TIME_S[N],
            "paper_hardware": "Intel Xeon E5-2690 v3, 2.6 GHz, 12 cores (modified DualSPHysics)",
            "paper_steps": "not stated",
            "run_of_300_days_at_dt_1_day_s": 300 * ms_per_step / 1e3 / world}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(plume),
        "timing": "CUDA events around one graph replay (ade_run) per step; per-phase times from "
                  "ade_step_timed",
        "grid": {"cell_subdiv": sim.info.cell_subdiv, "cells": sim.info.ncells,
                 "stencil_rows": sim.info.stencil_rows, "sort_passes": sim.info.sort_passes,
                 "variant": walk,
                 "autotune_best_ms": tune_ms, "dt": sim.info.dt, "skin": sim.info.skin},
        "steps_per_s": 1e3 / ms_per_step * world,
        "interactions_per_step": 2 * pairs,
        "roofline": roofline, "e2e": e2e, "clocks": clk,
        "cell_build": cell_build_roof(plume.n, sim.info.ncells, plume.dim,
                                      roofline["phase_ms_per_step"]["cells"]),
        "gpu_launches": launches * args.steps,
        **line_extra,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cv, steps, secs, ns = cpu_oracle_rate(plume, xq, C, oracle_sample(plume, args.cpu_sample),
                                              args.cpu_seconds, v=v)
        line["cpu_baseline"] = {"value": cv, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"Eq. 4 evaluated twice per step on a fixed sample of {ns} "
                                          f"of {plume.n} particles; {steps} steps in {secs:.1f} s",
                                "cpu_model": host_cpu_model(),
                                "single_core": single_core_baseline(plume, xq, C, oracle_sample(plume, args.cpu_sample),
                                                                    v=v)}
    sim.close()
    if rank == 0:
        print(json.dumps(line))
    dist.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default=DEFAULT_WORKLOAD)
    ap.add_argument("--cpu-sample", type=int, default=131072)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", choices=("auto",) + tuple(VARIANT_FLAGS), default="auto",
                    help="interaction walk of the single-plume workloads (default: autotuned)")
    ap.add_argument("--cell-subdiv", type=int, default=0,
                    help="cells per support radius with --variant (0: the library's choice)")
    ap.add_argument("--accuracy", action="store_true",
                    help="run every configured plume to its step count and print its error against "
                         "the closed form (one JSON line per plume), instead of timing")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="leave the configured run against the closed form out of the bench line")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)       # at least 3 untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.accuracy:
        return run_accuracy(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
