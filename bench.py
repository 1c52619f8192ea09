"""Benchmark of the MLS-MPM substep library on GB300.

Headline: particle-substeps/s on the 1,048,576-particle elastoplastic tissue
block (256^3 grid, fixed-corotated + von Mises, dt = 5e-5), FP32, over the
block's whole 500-substep trajectory (fall, impact on the sticky floor and the
plastic flow after it).  One bench step = 25 substeps, so 20 steps are the
whole trajectory; the timed region starts from the initial state and restarts
it (a device copy, inside the timed region) every 20 steps.  Inputs are
synthetic and seeded.  The particle state (~100 MB read + ~100 MB written per
substep) and the grid exceed the 129 MB L2 between timed iterations, so no
separate L2 flush is done (stated in ``config``).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs an independent replica (the single-scene
substep does not shard); value = particle-substeps of all ranks / max time.
``--impl reference`` times the FP64 CPU oracle on a bounded sample instead.
"""
import argparse
import glob
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "particle-substeps/s at 1M particles FP32"
UNIT = "particle-substeps/s"
SUBSTEPS_PER_STEP = 25
# scan, scatter, P2G, grid update, accumulator reset, G2P
KERNELS_PER_SUBSTEP = 6
TRAJECTORY_STEPS = 20  # 20 x 25 = the block's 500-substep trajectory
FALL_SUBSTEPS = 150    # the block is still falling (F close to I) before this substep


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--particles", type=int, default=1048576)
    p.add_argument("--no-extras", action="store_true", help="skip e2e, batched and cpu-baseline legs")
    p.add_argument("--autotune", action="store_true")
    p.add_argument("--profile-substeps", type=int, default=0,
                   help="run this many substeps with direct launches and exit (the command profiles use)")
    p.add_argument("--profile-batched-substeps", type=int, default=0,
                   help="run the 256-scene batched workload for this many substeps with direct launches "
                        "(P2G passes of 576, 128-thread 64-register G2P) and exit")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------- replicas

class Replicas:
    """Host side of the replica mode: every rank simulates its own copy of the
    workload (no data-path collective); ranks meet at barriers around the
    timed region and the slowest rank's time is the job's time.  ``dist`` is
    torch.distributed with an initialised process group, or None for one
    process; ``device`` is where the reduction tensor lives (cuda for NCCL,
    cpu for gloo); ``sync`` drains the device queue on each side of a barrier."""

    def __init__(self, dist=None, device="cpu", sync=None):
        self.dist, self.device, self.sync = dist, device, sync

    def barrier(self):
        if self.sync:
            self.sync()
        if self.dist:
            self.dist.barrier()
        if self.sync:
            self.sync()

    def max_over_ranks(self, x):
        if not self.dist:
            return x
        import torch

        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(world, units_per_rank, ms):
    """Units of all ranks per second, timed by the slowest rank (weak scaling)."""
    return world * units_per_rank / (ms / 1e3)


# --------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

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
        self.t.join(timeout=2)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


# ----------------------------------------------------- algorithmic bytes
#
# The roofline is taken against the method's ALGORITHMIC bytes per
# particle-substep: FP32 structure-of-arrays state, each field read or written
# once per phase in which the algorithm needs it; P2G and G2P are separated by
# a grid-wide dependency, so x and F are read twice.
#   P2G   read x, v, C, F                                    96 B per particle
#   G2P   read x, F (48), write x, v, C, F (96)             144 B per particle
#   sort  key written + read, permutation written + read     16 B per particle
#   grid  (m, mv) written by P2G 16, read 16, velocity written 12 and read by
#         G2P 12, accumulator cleared 16                     72 B per active node
# (~270 B per particle-substep at 8 particles per cell.)  This design moves
# somewhat more (implementation_bytes): the stress is stored by G2P and read
# by P2G instead of F (24 + 24 B for 36 B), particle ids, the next substep's
# brick key and rank, and the permutation rewritten in cell order.

ALGO_PER_PARTICLE = {"sort": 16, "p2g": 96, "grid": 0, "g2p": 144}
ALGO_PER_NODE = {"sort": 0, "p2g": 0, "grid": 72, "g2p": 0}


def algorithmic_bytes(N, active_nodes):
    """Algorithmic bytes of each phase of one substep over N particles whose
    stencils touch `active_nodes` grid nodes (the table above)."""
    return {k: ALGO_PER_PARTICLE[k] * N + ALGO_PER_NODE[k] * active_nodes for k in ALGO_PER_PARTICLE}


def implementation_bytes(N, bricks, active_nodes, pp_mat=False):
    """Bytes this design's kernels move at least once per substep:
      sort  scan: brick count + node flag (8 B per brick of the grid); scatter:
            key, rank and the brick offset read, slot and its cell written (17 B
            per particle)
      p2g   perm 4 + cell 1 + x 12 + v 12 + C 36 + tau 24 read, perm 4 rewritten
            in cell order (93 B per particle) + one 16-B reduction per active node
      grid  (m, mv) read, (v, m) written, (m, mv) cleared: 48 B per active node
      g2p   perm 4 + x 12 + F 36 + id 4 read; x, v, C, F 96 + tau 24 + id 4 +
            key, rank 8 written (188 B per particle; + mu, lam 16 with
            per-particle materials) + the velocity window, 16 B per active node"""
    extra = 16 if pp_mat else 0
    return {
        "sort": 8 * bricks + 17 * N,
        "p2g": 93 * N + 16 * active_nodes,
        "grid": 48 * active_nodes,
        "g2p": (188 + extra) * N + 16 * active_nodes,
    }


def kernel_source_digest():
    """Digest of the CUDA sources, to tell whether a recorded ncu figure still
    describes the kernels that run.  Whole-line comments and blank lines are left
    out, so that editing documentation does not retire a capture; any change to
    a line of code does."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2502_18437_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            for line in fh:
                t = line.strip()
                if t and not t.startswith(b"//"):
                    h.update(line.rstrip() + b"\n")
    return h.hexdigest()[:16]


def recorded_profile(kernel):
    """Per-launch figures of `kernel`'s ncu summary under profiles/ (DRAM traffic,
    warp instructions), or {} when the summary is missing or the CUDA sources
    changed since the capture."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_tissue_block_1m.md")
    if not os.path.exists(path):
        return {}
    fields = {}
    keys = ("traffic_bytes_per_launch", "warp_instructions_per_launch", "source_digest")
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.split(":", 1)[0] in keys:
                k, v = line.split(":", 1)
                fields[k] = v.strip()
    if fields.pop("source_digest", None) != kernel_source_digest():
        return {}
    return {k: int(v) for k, v in fields.items()}


def recorded_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` from its ncu summary, or None."""
    return recorded_profile(kernel).get("traffic_bytes_per_launch")


def issue_roofline(kernel, launch_ms, sm_count, sm_mhz):
    """Instruction-issue roofline of `kernel`: its warp instructions per launch
    (ncu, impact phase) over its launch duration, against one warp instruction
    per cycle on each of the 4 schedulers of every SM at the sampled SM clock;
    None without a current ncu summary."""
    instr = recorded_profile(kernel).get("warp_instructions_per_launch")
    if not instr or not launch_ms or not sm_count or not sm_mhz:
        return None
    peak = sm_count * 4 * sm_mhz * 1e6 / 1e9  # G warp instructions / s
    achieved = instr / (launch_ms / 1e3) / 1e9
    return {"kernel": kernel, "warp_instructions": instr, "achieved": round(achieved, 1), "peak": round(peak, 1),
            "unit": "G warp instructions/s", "frac": round(achieved / peak, 4),
            "floor_ms": round(instr / (peak * 1e9) * 1e3, 5), "launch_ms": round(launch_ms, 5)}


def roofline_fields(N, bricks, active_nodes, per_launch_ms, substep_ms, peak, peak_kind, pp_mat=False):
    """The `roofline` object of the JSON line: the dominant kernel (largest share
    of the substep's device time), its algorithmic bytes per launch divided by its
    mean launch duration, against the measured HBM copy peak; the whole substep's
    algorithmic bytes over the substep time beside it.  `implementation_bytes`
    reports what this design's kernels move, for comparison."""
    ab = algorithmic_bytes(N, active_nodes)
    ib = implementation_bytes(N, bricks, active_nodes, pp_mat)
    tot = sum(per_launch_ms.values())
    dom = max(per_launch_ms, key=per_launch_ms.get)
    achieved = ab[dom] / (per_launch_ms[dom] / 1e3) / 1e9
    step = sum(ab.values())
    return {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_source": peak_kind, "traffic": recorded_traffic(dom),
            "algorithmic_bytes_per_launch": ab[dom], "launch_ms": round(per_launch_ms[dom], 5),
            "algorithmic_bytes_per_particle": {k: ALGO_PER_PARTICLE[k] for k in ab},
            "algorithmic_bytes_per_active_node": {k: ALGO_PER_NODE[k] for k in ab},
            "share": {k: round(v / tot, 4) for k, v in per_launch_ms.items()},
            "per_launch_ms": {k: round(v, 5) for k, v in per_launch_ms.items()},
            "kernel_frac": {k: round(ab[k] / (per_launch_ms[k] / 1e3) / 1e9 / peak, 4) for k in ab},
            "substep_algorithmic_bytes_per_particle": round(step / N, 1),
            "whole_substep_frac": round(step / (substep_ms / 1e3) / 1e9 / peak, 4),
            "implementation_bytes_per_particle_substep": round(sum(ib.values()) / N, 1),
            "implementation_bytes_per_launch": ib[dom],
            "active_nodes": active_nodes}


# ----------------------------------------------------------- our arm

class Trajectory:
    """The block's trajectory replayed from its initial state: `step()` runs one
    bench step (SUBSTEPS_PER_STEP substeps) and restarts from the initial state
    (device-to-device state writes) after every TRAJECTORY_STEPS steps."""

    def __init__(self, sim, dt, x0, v0, C0, F0):
        self.sim, self.dt = sim, dt
        self.init = dict(x=x0, v=v0, C=C0, F=F0)
        self.k = 0

    def restart(self):
        self.sim.write_state(0, **self.init)
        self.k = 0

    def step(self):
        if self.k == TRAJECTORY_STEPS:
            self.restart()
        self.sim.substep(self.dt, SUBSTEPS_PER_STEP)
        self.k += 1


def phase_windows(sim, traj, dt):
    """Per-phase device time over the whole trajectory with CUDA events around
    every phase (direct launches), split into the falling window (substeps
    1..FALL_SUBSTEPS) and the impact / plastic-flow window after it."""
    traj.restart()
    sim.set_option("phase_timing", 1)
    sim.phase_stats(reset=True)
    total = TRAJECTORY_STEPS * SUBSTEPS_PER_STEP
    out = {}
    for name, k in (("fall", FALL_SUBSTEPS), ("impact", total - FALL_SUBSTEPS)):
        sim.substep(dt, k)
        out[name] = sim.phase_stats(reset=True)
    sim.set_option("phase_timing", 0)
    return out


def run_ours(args):
    import torch

    from paper_2502_18437_gb300 import build as libbuild
    from paper_2502_18437_gb300 import mpm, workloads

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        libbuild.build()
    if dist:
        dist.barrier()
    mpm.lib()

    if args.profile_batched_substeps:
        # the command of the batched ncu summary under profiles/: direct launches, no timing
        bstream = torch.cuda.Stream()
        bsim = mpm.from_scenes(workloads.batched_scenes(), stream=bstream.cuda_stream)
        for k, v in (("use_graphs", 0), ("p2g_chunk", 576), ("g2p_threads", 128), ("g2p_regs64", 1)):
            bsim.set_option(k, v)
        bsim.substep(1e-4, args.profile_batched_substeps)
        errs = [bsim.error_bits(s) for s in range(256)]
        bsim.close()
        if rank == 0:
            print(json.dumps({"profile_batched_substeps": args.profile_batched_substeps, "errors": sum(errs)}),
                  flush=True)
        return
    sc = workloads.tissue_block(N=args.particles)
    N, n, dt = len(sc["x"]), sc["n"], sc["dt"]
    stream = torch.cuda.Stream()
    sim = mpm.from_workload(sc, stream=stream.cuda_stream)
    if args.profile_substeps:
        # the command the ncu summaries under profiles/ capture: direct launches, no timing
        sim.set_option("use_graphs", 0)
        sim.substep(dt, args.profile_substeps)
        sim.read_state(0, ("x",))
        sim.close()
        if rank == 0:
            print(json.dumps({"profile_substeps": args.profile_substeps, "particles": N}), flush=True)
        if dist:
            dist.barrier()
            dist.destroy_process_group()
        return
    init = sim.read_state(0, device=True)
    traj = Trajectory(sim, dt, init["x"], init["v"], init["C"], init["F"])
    tuned = None
    if args.autotune:
        sim.autotune(dt, 5)
        tuned = {k: sim.get_option(k) for k in ("p2g_chunk", "g2p_threads", "g2p_regs64", "ctas_per_sm")}

    reps = Replicas(dist, device="cuda", sync=torch.cuda.synchronize)
    barrier, max_over_ranks = reps.barrier, reps.max_over_ranks

    # ---- device-resident timed region: the trajectory from its initial state ----
    for _ in range(args.warmup):
        traj.step()
    traj.restart()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        traj.step()
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if sim.error_bits(0):
        raise RuntimeError(f"device error bits {sim.error_bits(0)} during the timed trajectory")
    ms = max_over_ranks(ms)
    total_substeps = args.steps * SUBSTEPS_PER_STEP
    value = whole_job_rate(world, N * total_substeps, ms)
    ms_per_step = ms / args.steps
    restarts = max(0, (args.steps - 1) // TRAJECTORY_STEPS)

    # ---- per-kernel durations over the same trajectory (CUDA events per phase) ----
    win = phase_windows(sim, traj, dt)
    names = ["sort", "p2g", "grid", "g2p"]
    sub = sum(w["substeps"] for w in win.values())
    per_launch_ms = {k: sum(w["ms"][i] for w in win.values()) / sub for i, k in enumerate(names)}
    active_nodes = win["impact"]["active_nbricks"] * 64
    peak, peak_kind = measured_peaks()
    roofline = roofline_fields(N, (n // 4) ** 3, active_nodes, per_launch_ms, ms / total_substeps, peak, peak_kind)
    roofline["windows"] = {
        name: {"substeps": w["substeps"],
               "per_launch_ms": {k: round(w["ms"][i] / w["substeps"], 5) for i, k in enumerate(names)},
               "kernel_frac": {k: round(algorithmic_bytes(N, w["active_nbricks"] * 64)[k] /
                                        (w["ms"][i] / w["substeps"] / 1e3) / 1e9 / peak, 4)
                               for i, k in enumerate(names)},
               "active_nodes": w["active_nbricks"] * 64}
        for name, w in win.items()}
    roofline["timing"] = ("per-phase CUDA events on the context's stream over the whole 500-substep "
                          "trajectory (direct launches); the headline value is graph replay")
    # the kernels move their algorithmic bytes at a fraction of the HBM peak; the issue
    # rate of their instructions (ncu counts of the impact-phase launch against the
    # impact window's mean launch duration) is the bound beside it
    props = torch.cuda.get_device_properties(local)
    roofline["issue"] = {k: issue_roofline(k, win["impact"]["ms"][names.index(k)] / win["impact"]["substeps"],
                                           props.multi_processor_count, clk.get("sm_mhz"))
                         for k in ("g2p", "p2g")}

    chunk = sim.get_option("graph_chunk")
    graphs = -(-SUBSTEPS_PER_STEP // chunk)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded tissue block, 1 replica per GPU)",
            "config": {"workload": f"tissue_block_{N}p_256^3_fixed_corotated_von_mises",
                       "particles_per_gpu": N, "grid": f"{n}^3", "substeps_per_step": SUBSTEPS_PER_STEP,
                       "dt": dt, "parallelism": f"replicas x{world}",
                       "window": (f"substeps 1..{min(total_substeps, TRAJECTORY_STEPS * SUBSTEPS_PER_STEP)} of the "
                                  f"{TRAJECTORY_STEPS * SUBSTEPS_PER_STEP}-substep trajectory from its initial "
                                  f"state (fall, impact, plastic flow); {restarts} restart(s) inside the timed region"),
                       "l2": "working set > 129 MB L2 between iterations (no flush)",
                       "launch": (f"per step: mpm_substep(dt, {SUBSTEPS_PER_STEP}) = {graphs} CUDA graph replay(s) "
                                  f"of up to {chunk} substeps, {KERNELS_PER_SUBSTEP} kernels per substep"
                                  + "; the first substep runs directly after the key kernel of the initial "
                                  "state" + ("" if restarts == 0 else "; each restart adds 4 state-write kernels "
                                             "and the key kernel"))},
            "gpu_launches": KERNELS_PER_SUBSTEP * total_substeps + 1 + restarts * (4 + 1), "clocks": clk,
            "roofline": roofline}
    if tuned:
        line["config"]["autotuned"] = tuned

    if not args.no_extras:
        # ---- end to end through the C ABI with pinned HOST buffers -------------
        traj.restart()
        pin = {f: torch.empty(s, dtype=torch.float32).pin_memory().numpy()
               for f, s in (("x", (N, 3)), ("v", (N, 3)), ("C", (N, 3, 3)), ("F", (N, 3, 3)))}
        st = sim.read_state(0)
        for f in pin:
            pin[f][...] = st[f]
        ptrs = [pin[f].ctypes.data for f in ("x", "v", "C", "F")]

        def e2e_step():
            mpm.mpm_write_state(sim.h, 0, 15, ptrs, mpm.MEM_HOST)
            sim.substep(dt, SUBSTEPS_PER_STEP)
            s = mpm.mpm_read_state(sim.h, 0, 15, ptrs, mpm.MEM_HOST)
            if s != 0:
                raise mpm.MPMError(s, "e2e read")

        for _ in range(args.warmup):
            e2e_step()
        for f in pin:  # the e2e trajectory also starts from the initial state
            pin[f][...] = st[f]
        barrier()
        t0 = time.perf_counter()
        for k in range(args.steps):
            if k and k % TRAJECTORY_STEPS == 0:
                for f in pin:
                    pin[f][...] = st[f]
            e2e_step()
        barrier()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3)
        line["e2e"] = {"value": whole_job_rate(world, N * total_substeps, e2e_ms), "unit": UNIT,
                       "h2d_bytes_per_step": 96 * N, "d2h_bytes_per_step": 96 * N,
                       "ms_per_step": e2e_ms / args.steps,
                       "what": (f"mpm_write_state(x,v,C,F from pinned host) + {SUBSTEPS_PER_STEP} substeps + "
                                "mpm_read_state(x,v,C,F to pinned host), wall clock")}
    sim.close()

    if not args.no_extras and rank == 0:
        line["batched"] = run_batched(args, stream)
        line["scale_sweep"] = run_scale_sweep(stream)
        line["paper_timing_scene"] = run_paper_timing(stream)
        line["cpu_baseline"] = run_cpu_baseline(sc)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def time_substeps(sim, stream, dt, k):
    """Device time (ms) of k substeps on the context's stream, CUDA events."""
    import torch

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.substep(dt, k)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def run_batched(args, stream):
    """256 scenes, 2k-32k particles each: env-substeps/s with one launch per
    phase over all scenes (graph replay, launch shapes from mpm_autotune on this
    workload) vs a per-scene launch loop (direct, and captured in graphs), each
    timed with CUDA events over 200 substeps after 20 of warm-up."""
    from paper_2502_18437_gb300 import mpm, workloads

    scenes = workloads.batched_scenes()
    out = {"scenes": len(scenes), "particles": int(sum(len(s["x"]) for s in scenes)), "substeps_timed": 200}
    dt = 1e-4
    shapes = None
    for name, opts in (("batched_graph", {"launch_mode": 0, "use_graphs": 1}),
                       ("looped_direct", {"launch_mode": 1, "use_graphs": 0}),
                       ("looped_graph", {"launch_mode": 1, "use_graphs": 1})):
        sim = mpm.from_scenes(scenes, stream=stream.cuda_stream)
        for k, v in opts.items():
            sim.set_option(k, v)
        if name == "batched_graph":
            out["autotune_best_ms_per_substep"] = sim.autotune(dt, 10)
            shapes = {k: sim.get_option(k) for k in ("p2g_chunk", "g2p_threads", "g2p_regs64", "ctas_per_sm")}
        elif shapes:
            for k, v in shapes.items():
                sim.set_option(k, v)
        sim.substep(dt, 20)
        ms = time_substeps(sim, stream, dt, 200)
        if sim.error_bits(0):
            raise RuntimeError(f"batched {name}: device error bits {sim.error_bits(0)}")
        out[name] = len(scenes) * 200 / (ms / 1e3)
        sim.close()
    out["autotuned_shapes"] = shapes
    out["unit"] = "env-substeps/s"
    out["speedup_vs_looped_direct"] = out["batched_graph"] / out["looped_direct"]
    out["speedup_vs_looped_graph"] = out["batched_graph"] / out["looped_graph"]
    return out


def run_scale_sweep(stream):
    """The scale-sweep tissue blocks (64k, 256k, 1M, 4M particles): particle-substeps/s
    in graph replay over substeps 31..130 (CUDA events), and per kernel the
    algorithmic GB/s from phase events over 20 more substeps."""
    from paper_2502_18437_gb300 import mpm, workloads

    peak, _ = measured_peaks()
    out = {}
    for N in sorted(workloads.SCALE_POINTS):
        sc = workloads.tissue_block(N=N)
        n, dt = sc["n"], sc["dt"]
        sim = mpm.from_workload(sc, stream=stream.cuda_stream)
        sim.substep(dt, 30)
        ms = time_substeps(sim, stream, dt, 100) / 100
        sim.set_option("phase_timing", 1)
        sim.phase_stats(reset=True)
        sim.substep(dt, 20)
        ps = sim.phase_stats(reset=True)
        sim.close()
        ab = algorithmic_bytes(N, ps["active_nbricks"] * 64)
        per = {k: ps["ms"][i] / ps["substeps"] for i, k in enumerate(["sort", "p2g", "grid", "g2p"])}
        out[str(N)] = {"grid": f"{n}^3", "value": N / (ms / 1e3), "ms_per_substep": round(ms, 5),
                       "kernel_gbs": {k: round(ab[k] / (per[k] / 1e3) / 1e9, 1) for k in per},
                       "kernel_frac": {k: round(ab[k] / (per[k] / 1e3) / 1e9 / peak, 3) for k in per},
                       "whole_substep_frac": round(sum(ab.values()) / (ms / 1e3) / 1e9 / peak, 3),
                       "active_pbricks": ps["active_pbricks"], "active_nbricks": ps["active_nbricks"]}
    return {"unit": "particle-substeps/s", "points": out}


def run_paper_timing(stream):
    """The paper's timing scene (Sec. III-D): a cube falling on the fixed 56^3
    grid, each step advancing 0.02 s; MLS-MPM and standard MPM take 10 substeps
    of 0.002 s per step, PB-MPM one step of 0.02 s with 10 or 20 cycles.  For
    each particle count and solver: 12 steps timed with CUDA events after 1
    step of warm-up, graph replay; the cube falls freely over those 0.26 s
    (PB-MPM with 10 cycles at 0.02 s steps does not hold a 22-cell cube up on
    the floor, in the oracle as in the kernels, so the window ends before the
    impact)."""
    from paper_2502_18437_gb300 import mpm, workloads

    per = workloads.PAPER_TIMING_SUBSTEPS_PER_STEP
    solvers = (("mls", {}, per), ("standard", {}, per), ("pb10", {"solver": "pb", "pb_iterations": 10}, 1),
               ("pb20", {"solver": "pb", "pb_iterations": 20}, 1))
    out = {}
    for N in workloads.PAPER_TIMING_POINTS:
        sc = workloads.paper_timing_cube(N=N)
        row = {}
        for name, kw, substeps in solvers:
            kw = dict(kw)
            if name == "standard":
                kw["solver"] = "standard"
            sim = mpm.from_workload(sc, stream=stream.cuda_stream, **kw)
            dt = sc["dt"] * per / substeps
            sim.substep(dt, substeps)
            ms = time_substeps(sim, stream, dt, 12 * substeps)
            bits = sim.error_bits(0)
            sim.close()
            row[name] = {"steps_per_s": 12 / (ms / 1e3), "ms_per_step": ms / 12,
                         "particle_steps_per_s": N * 12 / (ms / 1e3), "error_bits": bits}
        out[str(N)] = row
    return {"grid": "56^3", "step": "0.02 s: 10 substeps of 0.002 s (mls, standard) or one PB-MPM step "
            "of 0.02 s with 10 / 20 cycles", "points": out,
            "paper": "figure only (absent from the text): no number to compare"}


def cpu_info():
    """Host CPU model, logical CPUs, and the threads the oracle uses (it is serial)."""
    model = None
    try:
        r = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10)
        for l in r.stdout.splitlines():
            if l.lower().startswith("model name"):
                model = l.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            with open("/proc/cpuinfo") as f:
                for l in f:
                    if l.lower().startswith(("model name", "cpu part")):
                        model = l.split(":", 1)[1].strip()
                        break
        except OSError:
            pass
    return {"cpu": model, "nproc": os.cpu_count(), "threads_used": 1}


def run_cpu_baseline(sc):
    import oracle

    N = len(sc["x"])
    st = oracle.state_from_workload(sc)
    cfg = oracle.config_from_workload(sc)
    t0 = time.perf_counter()
    oracle.run(cfg, st, sc["dt"], 1)
    dt_s = time.perf_counter() - t0
    info = cpu_info()
    return {"value": N / dt_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 substep of the full {N}-particle block (FP64, serial C, dense 256^3 grid)",
            "seconds": dt_s, **info}


# ------------------------------------------------------- reference arm

def run_reference(args):
    """FP64 CPU oracle, as it stands, on host cores: each step is one substep
    of a bounded sample (the first 262,144 particles) of the 1M block."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle

    from paper_2502_18437_gb300 import workloads

    sc = workloads.tissue_block(N=args.particles)
    keep = min(262144, len(sc["x"]))
    sample = workloads.scaled_copy(sc, keep)
    cfg = oracle.config_from_workload(sample)
    st = oracle.state_from_workload(sample)
    for _ in range(args.warmup):
        oracle.run(cfg, st, sample["dt"], 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.run(cfg, st, sample["dt"], 1)
    sec = time.perf_counter() - t0
    value = keep * args.steps / sec
    info = cpu_info()
    note = ("the oracle sweeps its dense 256^3 grid (16.8 M nodes) every substep whatever the particle count, "
            "so its rate per particle on this 262,144-particle sample is below the full 1M block's "
            "(cpu_baseline of the GPU arm's line)")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"tissue_block_{len(sc['x'])}p_256^3_fixed_corotated_von_mises",
                       "sample": f"first {keep} particles, 1 substep per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {keep} particles of the block, 1 substep per step",
                             "note": note, **info},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
