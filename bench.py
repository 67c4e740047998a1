"""Throughput of the differentiable magneto-elastic MPM on one GB300.

One bench step = one design iteration of a workload (default: the 3D
locomotion configuration, about 1,000,000 particles on 128^3 for 5,000
substeps, the largest single-GPU configuration): the forward pass over the
whole horizon (cell sort, P2G, grid operation, G2P, objective) plus the
checkpointed adjoint (recomputation and the reverse kernels), producing
dL/dphi, dL/dB~_r and dL/dB_applied.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload walker3d_128|walker2d_128|beam2d_64|plate3d_64|walker2d_batch64]

Prints one JSON line (rank 0).  ``value`` is particle-steps per second of
forward+adjoint over all ranks (sum of particles x substeps / max time);
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload instead.  Several GPUs run independent replicas (a single simulation
does not shard without a halo exchange every substep).
"""
from __future__ import annotations

import argparse
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

from paper_2503_22767_gb300 import workloads as W  # noqa: E402

METRIC = "particle-steps/s fwd+adjoint (and ms/design iter) vs oracle, % HBM roofline"
UNIT = "particle-steps/s"
CLASS_NAMES = ["forward particle (G2P+P2G)", "adjoint particle (P2G^T+G2P^T)", "grid operation",
               "grid adjoint"]


# the paper's five workload shapes: generator and full horizon.  The default,
# walker3d_128, is the largest configuration that fits one GPU; the others
# measure the same step on the other shapes.
WORKLOADS = {
    "walker2d_128": (lambda seed, n: W.walker_2d(seed=seed, n_steps=n, checkpoint_every=100), 4000),
    "beam2d_64": (lambda seed, n: W.beam_2d(seed=seed, n_steps=n), 200),
    "plate3d_64": (lambda seed, n: W.with_steps(W.plate_3d(seed=seed, n_steps=n), n, checkpoint_every=100), 1000),
    "walker3d_128": (lambda seed, n: W.walker_3d(seed=seed, n_steps=n, checkpoint_every=100), 5000),
    "walker2d_batch64": (lambda seed, n: W.walker_batch_2d(seed=seed, n_steps=n, checkpoint_every=100), 2000),
}


# Device memory a design iteration may hold (bytes): the 3D locomotion
# configuration's 180 GB allowance, used by every workload to keep its last
# checkpoint segments resident (their recomputation skipped), except the 2D
# locomotion workload, whose configuration fixes recomputation every 100
# substeps.
RESIDENT_BUDGET = {"walker2d_128": 0}
TUNE_SUBSTEPS = 1000  # autotuner sample (substeps from the start of the horizon)
DEFAULT_BUDGET = 180e9


def workload(name="walker3d_128", seed=0, substeps=None, checkpoint_every=None):
    """A named workload; ``substeps`` shortens the horizon and
    ``checkpoint_every`` overrides the segment length (profiling runs on a
    few GB of device memory)."""
    make, full = WORKLOADS[name]
    w = make(seed, substeps if substeps else full)
    if checkpoint_every:
        w = W.with_steps(w, w.cfg.n_steps, checkpoint_every=checkpoint_every)
    return w


def workload_desc(w, name):
    c = w.cfg
    contact = f"Coulomb floor mu={c.floor_mu}" if c.wall_mode == 1 else "non-slip walls"
    loss = "locomotion loss (Eq. 40)" if c.loss_kind == 1 else "final-position MSE (Eq. 38)"
    inst = (f"{c.n_instances} instances sharing {c.n_designs} design(s)" if c.n_instances > 1
            else "one instance")
    ckpt = f"checkpoint every {c.checkpoint_every}" if c.checkpoint_every else "every substep stored"
    return {
        "workload": (f"{name}: {c.dim}D, {c.res}^{c.dim} grid, {c.n_total} particles, {inst}, "
                     f"{c.n_steps} substeps dt={c.dt}, {contact}, {loss}, {ckpt}"),
        "particles": c.n_total,
        "instances": c.n_instances,
        "substeps": c.n_steps,
        "grid": f"{c.res}^{c.dim}",
        "checkpoint_every": c.checkpoint_every,
        "step": "one design iteration: forward over the horizon + checkpointed adjoint",
    }


def method_bytes(dim):
    """Algorithmic bytes per particle-substep that the method itself must move
    (float32), by pass: what the roofline fractions are computed with.

    forward: read the state (x, v, C, F) and write it, read the design
    (phi, B~_r): 108 B in 2D, 208 B in 3D; plus the grid per active node (P2G
    write, grid read and write, G2P read: 40 B / 56 B) over the particles per
    cell (4 / 8): +10 B / +7 B.  adjoint: read the stored state, read the
    adjoint of n+1 and write that of n, read the design and read-modify-write
    its gradients: 180 B / 336 B, plus twice the forward grid term.
    Recomputation and sort traffic are not counted, so they count against the
    fractions.  Returns (forward, adjoint, forward + adjoint).
    """
    if dim == 2:
        fwd, adj = 108 + 10, 180 + 20
    else:
        fwd, adj = 208 + 7, 336 + 14
    return fwd, adj, fwd + adj


def kernel_bytes(cfg):
    """Bytes per particle and launch of this build's fused kernels (float32):
    the lean forward (G2P n + P2G n+1) reads and writes x and E and reads phi,
    B~_r; the store pass of the recomputation writes the full state instead;
    the fused adjoint reads state n, (x, E) of state n-1, the partial adjoint
    in and out, the design, and read-modify-writes the design gradients.
    Reported beside the method's bytes."""
    d = cfg.dim
    xf, full, design = d + d * d, 2 * d + 2 * d * d, 1 + d
    lean = 4 * (xf + xf + design)
    store = 4 * (xf + full + design)
    adjoint = 4 * (full + xf + 2 * xf + design + 2 * design)
    return {"forward lean": lean, "forward store": store, "adjoint": adjoint}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            p = json.load(fh)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM traffic per launch of the dominant kernel, from an ncu capture summarised
# under profiles/ (traffic.json).  A figure is used only while the particle
# kernels' sources hash to the value stored beside it, i.e. while the kernel
# is the one the counters were taken on; otherwise traffic is null.
KERNEL_SOURCES = ("particle_kernels.cuh", "mpm_device.cuh", "particle_io.cuh", "warp_scatter.cuh")


def kernel_source_hash():
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2503_22767_gb300", "csrc", name), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, kernel_class):
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            rec = json.load(fh)
        e = rec[workload][kernel_class]
        if e["kernel_sources_sha256_16"] != kernel_source_hash():
            return None, "kernel changed since the capture"
        return float(e["dram_bytes_per_launch"]), e["profile"]
    except (OSError, KeyError, ValueError, TypeError):
        return None, "no capture recorded for this workload and kernel"


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return None
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[4:8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, flags in rows for i, f in enumerate(flags)
                          if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", torch.cuda.current_device())
    from paper_2503_22767_gb300.sim import Simulator

    # A batch (several instances) is sharded by instance across the ranks,
    # and tasks of one design on several ranks sum their gradients (Eq. 35).
    # A single instance runs as one replica per rank, seeded by rank.
    plan = None
    if world > 1:
        full = workload(args.workload, seed=0, substeps=args.substeps, checkpoint_every=args.checkpoint_every)
        if full.cfg.n_instances >= world:
            from paper_2503_22767_gb300 import shard
            plan = shard.plan(full.cfg.counts, full.cfg.design_of_instance, world)
            w = shard.local_workload(full, plan, rank)
            total_ps = full.cfg.n_total * full.cfg.n_steps
    if plan is None:
        w = workload(args.workload, seed=rank, substeps=args.substeps, checkpoint_every=args.checkpoint_every)
        total_ps = w.cfg.n_total * w.cfg.n_steps * world
    cfg = w.cfg
    sim = Simulator(cfg)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    x0, phi, mag, field = t(w.x0), t(w.phi), t(w.mag), t(w.field)
    target, v0 = t(w.target), t(w.v0)
    dloss = torch.ones(cfg.n_instances, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def iteration():
        loss, _ = sim.forward(x0, phi, mag, field, target=target, v0=v0)
        g = sim.backward(dloss)
        if plan is not None:
            shard.reduce_design_grads(plan, rank, cfg.dim, g[0], g[1])
        return loss, g

    # launch configuration picked by the library's autotuner (outside the timed region)
    tuned = None
    if not args.no_autotune:
        sim.forward(x0, phi, mag, field, target=target, v0=v0)
        t0 = time.perf_counter()
        # the sample reaches 1,000 substeps: on a deforming body the particle
        # kernels slow down over the first thousand (uneven cells), and the
        # choice made on the first 200 alone flipped between runs
        tuned = sim.autotune(sample_substeps=min(cfg.n_steps, TUNE_SUBSTEPS))
        tuned["tuning_s"] = round(time.perf_counter() - t0, 2)

    if args.options:
        keys = {"block": 2, "fuse_grid": 3, "graphs": 4, "streams": 6, "pdl": 7, "adjoint_blocks": 8, "grid_blocks": 10, "persistent": 11,
                "scatter_2d": 13}
        for item in args.options.split(","):
            name, value = item.split("=")
            sim.set_option(keys[name.strip()], int(value))
        if tuned is not None:
            tuned = {**sim.options(), "tuning_s": tuned["tuning_s"], "overridden": args.options}

    budget = (args.resident_budget_gb * 1e9 if args.resident_budget_gb is not None
              else RESIDENT_BUDGET.get(args.workload, DEFAULT_BUDGET))
    resident = sim.set_resident_budget(budget) if budget > 0 else 0
    if tuned is not None:
        tuned["resident_segments"] = resident

    # the timed region runs the passes as a user would: no timing events inside
    # the captured graphs (they would break the launch overlap they measure)
    sim.set_option(1, 0)
    for _ in range(args.warmup):
        iteration()
    torch.cuda.synchronize()
    sim.reset_stats()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev.index) as clocks:
        for i in range(args.steps):
            flush.zero_()  # evict L2 between timed iterations (outside the events)
            ev[i][0].record(stream)
            loss, g = iteration()
            ev[i][1].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(ms)
    launches = sim.stats()["launches"]
    sim_options = sim.options()

    # Per-kernel durations: one more design iteration after the timed region,
    # on one stream and with programmatic dependent launch off, with CUDA
    # events around every k-th launch of each kernel class.  With PDL on, a
    # kernel's start event would fire while its predecessor still runs (its
    # CTAs wait inside it), and on two streams a kernel shares the GPU with
    # the other stream's; here each timed launch runs alone, so its events
    # bracket its own duration.  Class time per iteration = average duration
    # x the class's launches in one iteration; the sum over classes is
    # reported beside the timed step.
    sim.set_option(6, 1)
    sim.set_option(7, 0)
    sim.set_option(1, args.timing_stride)
    iteration()  # captures the instrumented graphs
    torch.cuda.synchronize()
    sim.reset_stats()
    flush.zero_()
    tp0, tp1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tp0.record(stream)
    iteration()
    tp1.record(stream)
    torch.cuda.synchronize()
    timing_pass_ms = tp0.elapsed_time(tp1)
    stats = sim.stats()
    sim.set_option(1, 0)
    sim.set_option(6, sim_options["streams"])
    sim.set_option(7, sim_options["pdl"])
    if dist:
        tt = torch.tensor([total_ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
    ms_per_step = total_ms / args.steps
    ps = cfg.n_total * cfg.n_steps
    value = total_ps / (ms_per_step / 1000.0)
    loss_val = float(loss.sum().item())

    # dominant kernel class by its time per design iteration
    avg_ms = [stats["timed_ms"][c] / stats["timed_launches"][c] if stats["timed_launches"][c] else 0.0
              for c in range(4)]
    class_ms = [avg_ms[c] * stats["class_launches"][c] for c in range(4)]
    dom = int(np.argmax(class_ms))
    peak, peak_kind = load_peaks()
    fwd_b, adj_b, step_b = method_bytes(cfg.dim)
    kb = kernel_bytes(cfg)
    # bytes per launch: every particle kernel launch covers all particles of
    # the batch, one substep of its pass
    per_particle = {0: fwd_b, 1: adj_b}.get(dom)
    if per_particle is not None:
        bytes_launch = per_particle * cfg.n_total
        what = (f"{per_particle} B per particle-substep (the method's {'forward' if dom == 0 else 'adjoint'} "
                f"bytes) x {cfg.n_total} particles")
    else:  # a grid class: 48 B (64 B adjoint) per node of every instance's grid
        per_node = 48 if dom == 2 else 64
        bytes_launch = per_node * cfg.n_instances * cfg.res ** cfg.dim
        what = f"{per_node} B per grid node x {cfg.n_instances * cfg.res ** cfg.dim} nodes"
    dur_s = avg_ms[dom] / 1e3
    achieved = bytes_launch / 1e9 / dur_s if dur_s > 0 else 0.0
    launches_timed = stats["timed_launches"][dom]
    roofline = {
        "bound": "hbm",
        "kernel": CLASS_NAMES[dom],
        "achieved": round(achieved, 1),
        "peak": peak,
        "unit": "GB/s",
        "frac": round(achieved / peak, 4),
        "peak_source": f"{peak_kind} hbm_gbs (burst copy; the kernel is timed alone)",
        "traffic": None,
        "avg_launch_us": round(1e3 * avg_ms[dom], 2),
        "algorithmic_bytes_per_launch": round(bytes_launch),
        "algorithmic_bytes": what,
        "timed_launches": launches_timed,
        "class_ms_per_iteration": {CLASS_NAMES[c]: round(class_ms[c], 3) for c in range(4)},
        "class_launches_per_iteration": {CLASS_NAMES[c]: int(stats["class_launches"][c]) for c in range(4)},
        "avg_launch_us_by_class": {CLASS_NAMES[c]: round(1e3 * avg_ms[c], 2) for c in range(4)},
        "class_ms_sum": round(sum(class_ms), 3),
        "class_ms_sum_over_step": round(sum(class_ms) / ms_per_step, 4),
        "timing_pass_ms": round(timing_pass_ms, 3),
        "time_share_by_class": {CLASS_NAMES[c]: round(class_ms[c] / ms_per_step, 4) for c in range(4)},
    }
    if dom in (0, 1):
        kname = "forward lean" if dom == 0 else "adjoint"
        kach = kb[kname] * cfg.n_total / 1e9 / dur_s if dur_s > 0 else 0.0
        roofline["fused_kernel_bytes"] = {"bytes_per_particle": kb[kname], "achieved": round(kach, 1),
                                          "frac": round(kach / peak, 4),
                                          "what": f"{kname} kernel's own loads and stores per particle"}
    roofline["timing"] = (f"CUDA events around every {args.timing_stride}th launch of each kernel class, "
                          "in one extra design iteration after the timed region: one stream, programmatic "
                          "dependent launch off")
    if args.traffic_bytes:
        roofline["traffic"] = args.traffic_bytes
        roofline["traffic_source"] = "--traffic-bytes"
    else:
        roofline["traffic"], roofline["traffic_source"] = recorded_traffic(args.workload, CLASS_NAMES[dom])
    # the whole design iteration against the same peak: the method's bytes of
    # every particle-substep (forward + adjoint) over the timed step
    step_achieved = ps * step_b / 1e9 / (ms_per_step / 1e3)
    step_roofline = {"bound": "hbm", "achieved": round(step_achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(step_achieved / peak, 4), "bytes_per_particle_step": step_b,
                     "what": "the method's forward + adjoint bytes of every particle-substep over the timed "
                             "design iteration (recomputation, sort and full-grid traffic count against it)"}

    # end to end through the host-buffer entry points (pinned memory)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    hx0, hphi, hmag, hfield = pin(w.x0), pin(w.phi), pin(w.mag), pin(w.field)
    htarget = pin(w.target) if w.target is not None else None
    hv0 = pin(w.v0) if w.v0 is not None else None
    hloss = torch.empty(cfg.n_instances).pin_memory()
    hdl = torch.ones(cfg.n_instances).pin_memory()
    hgp = torch.empty(phi.shape).pin_memory()
    hgm = torch.empty(mag.shape).pin_memory()
    hgf = torch.empty(field.shape).pin_memory()
    e2e_steps = args.e2e_steps if args.e2e_steps else max(1, min(args.steps, 3))
    # the device-buffer iteration timed the same way (host wall clock around
    # synchronised iterations), so the two paths compare directly; its first,
    # untimed call re-captures the graphs without timing events
    iteration()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        iteration()
    torch.cuda.synchronize()
    dev_wall_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    # one untimed pass through the host entry points
    sim.forward_host(hx0, hphi, hmag, hfield, htarget, hv0, None, hloss)
    sim.backward_host(hdl, hgp, hgm, hgf)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sim.forward_host(hx0, hphi, hmag, hfield, htarget, hv0, None, hloss)
        sim.backward_host(hdl, hgp, hgm, hgf)
    torch.cuda.synchronize()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / e2e_steps
    h2d = 4 * (w.x0.size + w.phi.size + w.mag.size + w.field.size + cfg.n_instances
               + (w.target.size if w.target is not None else 0) + (w.v0.size if w.v0 is not None else 0))
    d2h = 4 * (cfg.n_instances + w.phi.size + w.mag.size + w.field.size)
    e2e = {"value": round(ps / (e2e_ms / 1e3), 1), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
           "d2h_bytes_per_step": int(d2h), "ms_per_step": round(e2e_ms, 3), "steps": e2e_steps,
           "device_buffers_wall_ms_per_step": round(dev_wall_ms, 3),
           "api": "mpm_forward_host + mpm_backward_host (C ABI, pinned host buffers)"}
    if dist:
        t2 = torch.tensor([e2e_ms], device=dev)
        dist.all_reduce(t2, op=dist.ReduceOp.MAX)
        e2e["value"] = round(total_ps / (float(t2.item()) / 1e3), 1)

    sequential = None
    if cfg.n_instances > 1 and not args.no_sequential and world == 1:
        # the single-instance runs keep as many segments resident as the batch
        # did; the batch's sets are released meanwhile
        sim.set_option(14, 0)
        sequential = run_sequential(w, dev, g, ps, resident)
        sim.set_option(14, resident)
    codesign = None
    if cfg.n_designs == 1 and not args.no_codesign and world == 1:
        codesign = run_codesign(w, sim, dev, args.steps)
    sim.close()
    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    out = {
        "metric": METRIC,
        "value": round(value, 1),
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 3),
        "higher_is_better": True,
        "scaling": "strong" if plan is not None else "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": f"synthetic (seeded bodies, designs and field schedules; workloads.py, {args.workload})",
        "config": {**workload_desc(w, args.workload), "parallelism": (f"instances sharded over {world} ranks" if plan is not None else
                                   f"replicas x{world}" if world > 1 else "single GPU"),
                   "launch": tuned if tuned else sim_options,
                   "resident_budget_gb": round(budget / 1e9, 1),
                   "l2": "256 MB buffer written between timed iterations (outside the timed events)"},
        "ms_per_design_iteration": round(ms_per_step, 3),
        "loss": loss_val,
        "roofline": roofline,
        "step_roofline": step_roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
        "device_bytes": stats["device_bytes"],
    }
    if sequential is not None:
        sequential["batched_speedup"] = round(value / world / sequential["value"], 3)
        out["sequential"] = sequential
    if codesign is not None:
        out["codesign"] = codesign
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w, args.cpu_sample_steps)
    print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


def run_sequential(w, dev, batched_grads, ps, resident=0):
    """The batch's instances as single-instance simulations run one after
    another on the same stream: same kernels, launch options tuned once on the
    first instance.  Returns their throughput and the gradient difference
    from the batched run (equal accuracy check)."""
    import torch
    from paper_2503_22767_gb300 import shard
    from paper_2503_22767_gb300.sim import Simulator

    cfg = w.cfg
    p = shard.plan(cfg.counts, cfg.design_of_instance, cfg.n_instances)  # one instance per slot
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    runs = []
    for r in range(cfg.n_instances):
        lw = shard.local_workload(w, p, r)
        runs.append((p.local[r][0], Simulator(lw.cfg), (t(lw.x0), t(lw.phi), t(lw.mag), t(lw.field)),
                     dict(target=t(lw.target), v0=t(lw.v0))))
    first = runs[0]
    first[1].forward(*first[2], **first[3])
    tuned = first[1].autotune(sample_substeps=min(cfg.n_steps, TUNE_SUBSTEPS))
    for _, sim, _, _ in runs[1:]:
        for key, name in ((2, "block"), (3, "fuse_grid"), (8, "adjoint_blocks"), (13, "scatter_2d")):
            sim.set_option(key, tuned[name])
    for _, sim, _, _ in runs:
        try:
            sim.set_option(14, resident)
        except Exception:  # device memory short: recompute every segment
            resident = 0
            for _, s2, _, _ in runs:
                s2.set_option(14, 0)
            break
    one = torch.ones(1, device=dev)

    def sweep():
        grads = {}
        for i, sim, a, kw in runs:
            sim.forward(*a, **kw)
            grads[i] = sim.backward(one)
        return grads

    sweep()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    grads = sweep()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    # per-design gradients (tasks sharing a design add up, Eq. 35) against
    # the batched run's
    gp_b = batched_grads[0].cpu().numpy()
    doff = np.concatenate([[0], np.cumsum(cfg.design_counts())]).astype(int)
    gp_s = np.zeros_like(gp_b)
    for i, (gp, _, _) in grads.items():
        d = cfg.designs[i]
        gp_s[doff[d]:doff[d + 1]] += gp.cpu().numpy()
    num = float(np.sum((gp_s - gp_b) ** 2))
    den = float(np.sum(gp_b ** 2))
    for _, sim, _, _ in runs:
        sim.close()
    return {"value": round(ps / (ms / 1e3), 1), "unit": UNIT, "ms_per_step": round(ms, 3),
            "instances": cfg.n_instances,
            "launch": {**{k: tuned[k] for k in ("block", "fuse_grid", "adjoint_blocks", "scatter_2d")},
                       "resident_segments": resident},
            "g_phi_rel_l2_vs_batched": float(np.sqrt(num / max(den, 1e-300))),
            "what": "each instance as its own single-instance simulation, one after another"}


def run_codesign(w, sim, dev, steps):
    """Whole design iterations of Section 3 on the workload: design maps
    (filter radius 1.5 dx, per-particle magnetisation, one harmonic stimulus
    per task), the simulation forward + adjoint, the reverse maps and Adam.
    The maps' share is timed on its own."""
    import torch
    from paper_2503_22767_gb300.design import CoDesign, DesignMaps

    cfg = w.cfg
    N = cfg.design_counts()[0]
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).to(dev)
    Br_max = float(np.max(np.linalg.norm(w.mag, axis=0)))
    maps = DesignMaps(t(w.x0[:, :N]), cfg.n_instances, cfg.n_steps, cfg.dt, 1.5 / cfg.res, Br_max, 0.02, 1.0,
                      20.0, delta=1e-6)
    rng = np.random.default_rng(0)
    zeta = w.mag / np.maximum(np.linalg.norm(w.mag, axis=0), 1e-12)
    params = {"phi": t(w.phi), "Br": t(np.ones(N)), "zeta": t(zeta), "Ba": t(np.full(cfg.n_instances, 0.5)),
              "f": t(rng.uniform(0.2, 0.8, cfg.n_instances)),
              "eta": t(rng.uniform(-1, 1, (cfg.n_instances, cfg.dim)))}
    cd = CoDesign(sim, maps, t(w.x0), params, target=t(w.target), v0=t(w.v0), lr=0.01)
    cd.step()  # warm-up (captures the graphs for the new inputs)
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record()
    for _ in range(steps):
        cd.step()
    e[1].record()
    # the maps alone: forward and reverse at the current variables
    g = (torch.ones(N, device=dev), torch.ones((cfg.dim, N), device=dev),
         torch.ones((cfg.n_instances, cfg.n_steps, cfg.dim), device=dev))
    e[2].record()
    for _ in range(steps):
        maps.forward(cd.params, 1.0)
        maps.backward(*g)
    e[3].record()
    torch.cuda.synchronize()
    ms = e[0].elapsed_time(e[1]) / steps
    maps_ms = e[2].elapsed_time(e[3]) / steps
    maps.close()
    return {"ms_per_iteration": round(ms, 3), "maps_ms_per_iteration": round(maps_ms, 4),
            "maps_share": round(maps_ms / ms, 5), "iterations": steps, "objective": cd.history,
            "value": round(cfg.n_total * cfg.n_steps / (ms / 1e3), 1), "unit": UNIT,
            "what": "design iterations of Eq. 34/35: maps (Eq. 23-30), forward + checkpointed adjoint, "
                    "reverse maps, Adam with box clipping"}


# ---------------------------------------------------------------------------
# oracle arm (CPU baseline and --impl reference)
# ---------------------------------------------------------------------------
def _oracle_sample(w, n_steps, cores):
    """Forward + adjoint of the first n_steps substeps on `cores` host threads
    (the oracle's threaded passes give the serial results bit for bit)."""
    import oracle

    ws = W.with_steps(w, n_steps)
    with oracle.threads(cores) as used:
        t0 = time.perf_counter()
        oracle.forward(ws)
        oracle.backward(ws, ckpt_every=max(1, n_steps // 4))
        dt = time.perf_counter() - t0
    return ws.cfg.n_total * n_steps / dt, dt, used


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def sample_steps(w, n_steps, cores=1):
    """Oracle sample length: the requested substeps, or (0) a window of about
    7 million 2D particle-steps per core (a 3D particle-step costs about 5x
    as much; the threads scale at about half of ideal), some 10-30 s of host
    time."""
    if n_steps > 0:
        return min(n_steps, w.cfg.n_steps)
    cost = 1.0 if w.cfg.dim == 2 else 5.0
    budget = 7.0e6 * max(1.0, 0.5 * cores) / cost
    return int(max(1, min(w.cfg.n_steps, budget // max(w.cfg.n_total, 1))))


def cpu_baseline(w, n_steps):
    cores = host_cores()
    n_all = sample_steps(w, n_steps, cores)
    v_all, dt_all, used = _oracle_sample(w, n_all, cores)
    n_one = sample_steps(w, n_steps, 1)
    v_one, dt_one, _ = _oracle_sample(w, n_one, 1)
    return {"value": round(v_all, 1), "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": (f"window of the first {n_all} of {w.cfg.n_steps} substeps, all {w.cfg.n_total} particles, "
                       f"forward + adjoint of the FP64 C oracle on {used} host threads ({dt_all:.1f} s)"),
            "one_core": {"value": round(v_one, 1), "unit": UNIT, "cores": 1,
                         "sample": (f"window of the first {n_one} substeps, all particles, forward + adjoint, "
                                    f"one thread ({dt_one:.1f} s)")}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = workload(args.workload, substeps=args.substeps, checkpoint_every=args.checkpoint_every)
    cores = host_cores()
    # each step is a window of the workload, sized so that the whole run
    # (warm-up included) stays within a few minutes
    n = sample_steps(w, args.cpu_sample_steps, cores)
    n = max(1, n // max(1, (args.steps + args.warmup) // 4))
    used = cores
    for _ in range(args.warmup):
        _oracle_sample(w, 1, cores)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, _, used = _oracle_sample(w, n, cores)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = w.cfg.n_total * n / (ms / 1e3)
    sample = (f"each step: the first {n} of {w.cfg.n_steps} substeps, all {w.cfg.n_total} particles, "
              f"forward + adjoint of the FP64 C oracle on {used} host threads")
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": UNIT,
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")), "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms, 3), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {**workload_desc(w, args.workload), "parallelism": f"CPU, {used} host threads"},
        "cpu_baseline": {"value": round(value, 1), "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--timing-stride", type=int, default=32,
                    help="time every k-th launch of each kernel class with CUDA events")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="walker3d_128",
                    help="workload shape (default: the 3D locomotion configuration, 1M particles on 128^3)")
    ap.add_argument("--cpu-sample-steps", type=int, default=0,
                    help="substeps of the oracle window (0: sized to some 10-30 s of host time)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the library's default launch options")
    ap.add_argument("--no-codesign", action="store_true",
                    help="skip the whole-design-iteration measurement (maps + simulation + Adam)")
    ap.add_argument("--no-sequential", action="store_true",
                    help="skip the one-instance-at-a-time comparison of multi-instance workloads")
    ap.add_argument("--options", default="",
                    help="launch options applied after autotuning, e.g. block=64,fuse_grid=0 "
                         "(names as in Simulator.options())")
    ap.add_argument("--substeps", type=int, default=0,
                    help="horizon of the timed workload (0: the configuration's full horizon)")
    ap.add_argument("--resident-budget-gb", type=float, default=None,
                    help="device memory (GB) the handle may hold, the rest of it for resident checkpoint "
                         "segments (default: 180, 0 for walker2d_128)")
    ap.add_argument("--checkpoint-every", type=int, default=0,
                    help="checkpoint segment length (0: the configuration's own)")
    ap.add_argument("--e2e-steps", type=int, default=0, help="end-to-end iterations (default min(steps, 3))")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes per launch of the dominant kernel from an ncu capture")
    args = ap.parse_args(argv)
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
