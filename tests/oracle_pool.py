"""Parallel evaluations of the FP64 oracle for finite differences (test
infrastructure).  Worker processes are started with the spawn method, so they
inherit no CUDA state from a test process that already used the GPU; each
worker rebuilds the seeded workload itself, so a task is only a few numbers."""
import multiprocessing as mp
import os

import numpy as np

import oracle
from paper_2502_18437_gb300 import workloads as W


def diff_cube_loss(task):
    """Loss of the differentiable workload after `steps` substeps, with the
    perturbations `pert` = [(kind, particle, coordinate, delta)] applied to the
    inputs: kind "E" scales E by (1 + delta), "nu" and "v0" add delta."""
    wl_kwargs, steps, pert = task
    sc = W.diff_cube(**wl_kwargs)
    E, nu, v0 = sc["E"].astype(np.float64), sc["nu"].astype(np.float64), sc["v"].astype(np.float64)
    for kind, i, d, delta in pert:
        if kind == "E":
            E[i] *= 1.0 + delta
        elif kind == "nu":
            nu[i] += delta
        else:
            v0[i, d] += delta
    mu, lam = oracle.lame_arrays(E, nu)
    st = oracle.State(sc["x"], v0, mu=mu, lam=lam)
    err = oracle.run(oracle.config_from_workload(sc), st, sc["dt"], steps)
    if err:
        raise RuntimeError(f"oracle error bits {err}")
    return oracle.loss(st.x, st.v, sc["target"])


def map_tasks(fn, tasks, workers=None):
    oracle.lib()  # build once in the parent, before the workers load it
    n = workers or max(1, min(16, os.cpu_count() or 1, len(tasks)))
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(fn, tasks)
