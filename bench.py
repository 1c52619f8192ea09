"""Benchmark of the MLS-MPM substep library on GB300.

Headline: particle-substeps/s on the 1,048,576-particle elastoplastic tissue
block (256^3 grid, fixed-corotated + von Mises, dt = 5e-5), FP32.  One bench
step = 10 substeps (one 0.02 s-style frame of the paper's timing scene is 10
substeps).  Inputs are synthetic and seeded.  The particle state (~110 MB read
+ written per substep) and the grid exceed the 129 MB L2 between timed
iterations, so no separate L2 flush is done (stated in ``config``).

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
SUBSTEPS_PER_STEP = 10


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
# Per-launch algorithmic bytes of each phase (FP32 SoA, each field moved once
# per phase in which the algorithm needs it):
#   sort : scan 4 B per brick of the grid; scatter 16 B per particle
#          (key + rank read, brick offset read, permutation write)
#   P2G  : 4 (perm) + 96 (x, v, C, F) [+ 8 mu, lam] B per particle
#          + 16 B per active node (the (m, mv) it produces)
#   grid : 48 B per active node (read (m, mv), write (v, m), clear the accumulator)
#   G2P  : 4 (perm) + 48 (x, F) + 4 (id) [+ 8] read, 96 (x, v, C, F) + 4 (id)
#          + 8 (key, rank) [+ 8] written per particle + 16 B per active node (halo)

def kernel_source_digest():
    """Digest of the CUDA sources, to tell whether a recorded ncu figure still
    describes the kernels that run."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2502_18437_gb300", "csrc")
    for f in sorted(glob.glob(os.path.join(csrc, "*.cu")) + glob.glob(os.path.join(csrc, "*.cuh"))):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes (read + write) per launch of `kernel` from its ncu summary under
    profiles/, or None when the summary is missing or the sources changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_tissue_block_1m.md")
    if not os.path.exists(path):
        return None
    fields = {}
    with open(path) as fh:
        for line in fh:
            if ":" in line and line.split(":", 1)[0] in ("traffic_bytes_per_launch", "source_digest"):
                k, v = line.split(":", 1)
                fields[k] = v.strip()
    if fields.get("source_digest") != kernel_source_digest() or "traffic_bytes_per_launch" not in fields:
        return None
    return int(fields["traffic_bytes_per_launch"])


def algorithmic_bytes(N, bricks, active_nodes, pp_mat=False):
    """Bytes each phase must move at least once per substep (the table of the
    kernels and their bounds):
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


# ----------------------------------------------------------- our arm

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
    if args.autotune:
        sim.autotune(dt, 5)

    reps = Replicas(dist, device="cuda", sync=torch.cuda.synchronize)
    barrier, max_over_ranks = reps.barrier, reps.max_over_ranks

    # ---- device-resident timed region (graph replay) -------------------
    for _ in range(args.warmup):
        sim.substep(dt, SUBSTEPS_PER_STEP)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    for _ in range(args.steps):
        sim.substep(dt, SUBSTEPS_PER_STEP)
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = max_over_ranks(ms)
    total_substeps = args.steps * SUBSTEPS_PER_STEP
    value = whole_job_rate(world, N * total_substeps, ms)
    ms_per_step = ms / args.steps

    # ---- per-kernel durations (CUDA events around each phase) ---------------
    sim.set_option("phase_timing", 1)
    sim.phase_stats(reset=True)
    sim.substep(dt, SUBSTEPS_PER_STEP)
    sim.phase_stats(reset=True)
    sim.substep(dt, args.steps * SUBSTEPS_PER_STEP // 2 or 1)
    ps = sim.phase_stats(reset=True)
    sim.set_option("phase_timing", 0)
    nb = (n // 4) ** 3
    active_nodes = ps["active_nbricks"] * 64
    ab = algorithmic_bytes(N, nb, active_nodes)
    per_launch_ms = {k: ps["ms"][i] / ps["substeps"] for i, k in enumerate(["sort", "p2g", "grid", "g2p"])}
    tot = sum(per_launch_ms.values())
    dom = max(per_launch_ms, key=per_launch_ms.get)
    peak, peak_kind = measured_peaks()
    achieved = ab[dom] / (per_launch_ms[dom] / 1e3) / 1e9
    step_bytes = sum(ab.values())
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind, "traffic": recorded_traffic(dom),
                "algorithmic_bytes_per_launch": ab[dom], "launch_ms": round(per_launch_ms[dom], 5),
                "share": {k: round(v / tot, 4) for k, v in per_launch_ms.items()},
                "per_launch_ms": {k: round(v, 5) for k, v in per_launch_ms.items()},
                "step_bytes_per_particle_substep": round(step_bytes / N, 1),
                "whole_substep_frac": round(step_bytes / (ms / total_substeps / 1e3) / 1e9 / peak, 4),
                "active_pbricks": ps["active_pbricks"], "active_nbricks": ps["active_nbricks"]}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded tissue block, 1 replica per GPU)",
            "config": {"workload": f"tissue_block_{N}p_256^3_fixed_corotated_von_mises",
                       "particles_per_gpu": N, "grid": f"{n}^3", "substeps_per_step": SUBSTEPS_PER_STEP,
                       "dt": dt, "parallelism": f"replicas x{world}",
                       "l2": "working set > 129 MB L2 between iterations (no flush)",
                       "launch": "CUDA graph replay, 5 kernels per substep"},
            "gpu_launches": 5 * total_substeps, "clocks": clk, "roofline": roofline}

    if not args.no_extras:
        # ---- end to end through the C ABI with pinned HOST buffers -------------
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
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        barrier()
        e2e_ms = max_over_ranks((time.perf_counter() - t0) * 1e3)
        line["e2e"] = {"value": whole_job_rate(world, N * total_substeps, e2e_ms), "unit": UNIT,
                       "h2d_bytes_per_step": 96 * N, "d2h_bytes_per_step": 96 * N,
                       "ms_per_step": e2e_ms / args.steps,
                       "what": "mpm_write_state(x,v,C,F from pinned host) + 10 substeps + mpm_read_state(x,v,C,F to pinned host)"}
    sim.close()

    if not args.no_extras and rank == 0:
        line["batched"] = run_batched(args, stream)
        line["scale_sweep"] = run_scale_sweep(stream)
        line["cpu_baseline"] = run_cpu_baseline(sc)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def run_batched(args, stream):
    """256 scenes, 2k-32k particles each: env-substeps/s, one launch per phase
    over all scenes (graph) vs a per-scene launch loop (direct and in a graph)."""
    import torch

    from paper_2502_18437_gb300 import mpm, workloads

    scenes = workloads.batched_scenes()
    out = {"scenes": len(scenes), "particles": int(sum(len(s["x"]) for s in scenes))}
    K = 20
    for name, opts in (("batched_graph", {"launch_mode": 0, "use_graphs": 1}),
                       ("looped_direct", {"launch_mode": 1, "use_graphs": 0}),
                       ("looped_graph", {"launch_mode": 1, "use_graphs": 1})):
        sim = mpm.from_scenes(scenes, stream=stream.cuda_stream)
        for k, v in opts.items():
            sim.set_option(k, v)
        sim.substep(1e-4, 4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.substep(1e-4, K)
        sim.error_bits(0)  # waits for the stream
        dt_s = time.perf_counter() - t0
        out[name] = len(scenes) * K / dt_s
        sim.close()
    out["unit"] = "env-substeps/s"
    out["speedup_vs_looped_direct"] = out["batched_graph"] / out["looped_direct"]
    out["speedup_vs_looped_graph"] = out["batched_graph"] / out["looped_graph"]
    return out


def run_scale_sweep(stream):
    """The scale-sweep tissue blocks (64k, 256k, 1M, 4M particles): particle-substeps/s
    in graph replay over 100 substeps after 30 of warm-up, and per kernel the
    algorithmic GB/s from phase events over 20 more substeps."""
    import torch

    from paper_2502_18437_gb300 import mpm, workloads

    peak, _ = measured_peaks()
    out = {}
    for N in sorted(workloads.SCALE_POINTS):
        sc = workloads.tissue_block(N=N)
        n, dt = sc["n"], sc["dt"]
        sim = mpm.from_workload(sc, stream=stream.cuda_stream)
        sim.substep(dt, 30)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sim.substep(dt, 100)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 100
        sim.set_option("phase_timing", 1)
        sim.phase_stats(reset=True)
        sim.substep(dt, 20)
        ps = sim.phase_stats(reset=True)
        sim.close()
        ab = algorithmic_bytes(N, (n // 4) ** 3, ps["active_nbricks"] * 64)
        per = {k: ps["ms"][i] / ps["substeps"] for i, k in enumerate(["sort", "p2g", "grid", "g2p"])}
        out[str(N)] = {"grid": f"{n}^3", "value": N / (ms / 1e3), "ms_per_substep": round(ms, 5),
                       "kernel_gbs": {k: round(ab[k] / (per[k] / 1e3) / 1e9, 1) for k in per},
                       "kernel_frac": {k: round(ab[k] / (per[k] / 1e3) / 1e9 / peak, 3) for k in per},
                       "active_pbricks": ps["active_pbricks"], "active_nbricks": ps["active_nbricks"]}
    return {"unit": "particle-substeps/s", "points": out}


def run_cpu_baseline(sc):
    import oracle

    N = len(sc["x"])
    st = oracle.state_from_workload(sc)
    cfg = oracle.config_from_workload(sc)
    t0 = time.perf_counter()
    oracle.run(cfg, st, sc["dt"], 1)
    dt_s = time.perf_counter() - t0
    return {"value": N / dt_s, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"1 substep of the full {N}-particle block (FP64, serial C)",
            "seconds": dt_s, "cpu": _cpu_name()}


def _cpu_name():
    try:
        with open("/proc/cpuinfo") as f:
            for l in f:
                if l.lower().startswith(("model name", "cpu part")):
                    return l.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


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
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"tissue_block_{len(sc['x'])}p_256^3_fixed_corotated_von_mises",
                       "sample": f"first {keep} particles, 1 substep per step"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"first {keep} particles of the block, 1 substep per step"},
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
