"""The full-size workload configurations on the GPU.

- the tissue slab at full size (256k particles on 128^3, Neo-Hookean with per-particle
  E, the slicer moving down through it and the capsule-chain thread sliding along its
  axis) for its full 1,000 substeps: no error flag, every particle finite and inside
  the domain, mass conserved on the grid, the blade receiving an impulse and the
  tissue under it pushed down;
- the largest scale-sweep block (4M particles on 256^3): one substep from perturbed
  state against the FP64 oracle, every particle;
- the smallest scale-sweep block (64k on 64^3) after 200 substeps against the oracle
  run from the same state.
"""
import numpy as np
import pytest

import oracle
from paper_2502_18437_gb300 import mpm, workloads as W
from tests.parity_util import Scales, oracle_cfg, oracle_state, perturbed
from tests.test_gpu_parity import check_fields, gpu_one_step, oracle_one_step

pytestmark = pytest.mark.gpu


def test_full_tissue_slab_1000_substeps():
    sc = W.tissue_slab()
    N, n = len(sc["x"]), sc["n"]
    assert N == 262144 and n == 128 and sc["substeps"] == 1000
    m_p = sc["rho"] * sc["V0"]
    with mpm.from_workload(sc) as sim:
        sim.impulse(0)
        sim.substep(sc["dt"], sc["substeps"])
        assert sim.error_bits(0) == 0
        st = sim.read_state(0)
        grid = sim.read_grid(0)
        imp = sim.impulse(0)
    x = st["x"].astype(np.float64)
    assert np.all(np.isfinite(x)) and np.all(np.isfinite(st["F"]))
    # every 3-node stencil still on the grid (the walls act on grid velocities; the
    # sticky floor lets the slab sink into its band)
    assert x.min() >= 1.5 / n and x.max() <= 1.0 - 2.5 / n
    # mass on the grid equals the particle mass (P2G conserves it)
    assert abs(grid[..., 3].astype(np.float64).sum() - N * m_p) <= 1e-5 * N * m_p
    # the blade pushed into the tissue: it received an upward reaction, and the
    # material under its edge moved down
    assert imp[0, 1] > 0.0
    # (the blade's plane is x = cx, its edge runs along z; over the run it moves 0.01
    # down from 0.01 below the slab's top)
    blade = sc["rigids"][0]
    cx, cz, half_edge = blade["center"][0], blade["center"][2], blade["half"][0]
    top = 0.03 + 0.1
    x0 = sc["x"].astype(np.float64)
    under = (np.abs(x0[:, 0] - cx) < 1.5 / n) & (np.abs(x0[:, 2] - cz) < 0.5 * half_edge) & (x0[:, 1] > top - 0.02)
    assert under.sum() > 100
    assert np.mean(x[under, 1] - x0[under, 1]) < 0.0


def test_full_size_4m_block_one_substep():
    sc = W.tissue_block(N=4194304)
    assert sc["n"] == 256
    v, C, F = perturbed(sc, seed=17, f_amp=0.03, c_amp=5.0)
    x, v, C, F, out = gpu_one_step(sc, v, C, F)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    assert abs(out["grid"][..., 3].astype(np.float64).sum() - gm.sum()) <= 1e-6 * gm.sum()


def test_small_block_200_substeps_tracks_oracle():
    # The 64k block falling onto the sticky floor (plastic flow at impact): after 200
    # substeps from the same state the positions agree to a small fraction of a cell.
    sc = W.tissue_block(N=65536)
    n = sc["n"]
    with mpm.from_workload(sc) as sim:
        sim.substep(sc["dt"], 200)
        assert sim.error_bits(0) == 0
        out = sim.read_state(0)
    st = oracle_state(sc)
    assert oracle.run(oracle_cfg(sc), st, sc["dt"], 200) == 0
    err = np.max(np.abs(out["x"].astype(np.float64) - st.x))
    print(f"64k block, 200 substeps: max |x - x_oracle| = {err:.3e} (dx = {1 / n:.3e})")
    assert err <= 1e-3 / n, err
    assert np.max(np.abs(st.x - sc["x"])) > 10 * err
