"""The paper's other two solvers (Sec. III) on the GPU against the FP64 oracle,
through the C ABI: standard MPM (Sec. III-A, Eq. 1-6) and PB-MPM (Sec. III-C).
One step from perturbed states, element by element, and a short trajectory."""
import numpy as np
import pytest

import oracle
from paper_2502_18437_gb300 import mpm, workloads as W
from tests.parity_util import EPS32, Scales, assert_close, oracle_cfg, oracle_rigids, oracle_state, perturbed

pytestmark = pytest.mark.gpu


def gpu_step(sc, v, C, F, solver, steps_before=0, **kw):
    with mpm.from_workload(sc, solver=solver, **kw) as sim:
        sim.write_state(0, v=v, C=C, F=F)
        if steps_before:
            sim.substep(sc["dt"], steps_before)
        st = sim.read_state(0)
        sim.impulse(0)
        sim.substep(sc["dt"], 1)
        out = sim.read_state(0)
        out["impulse"] = sim.impulse(0)
        assert sim.error_bits(0) == 0
    return st, out


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
@pytest.mark.parametrize("steps_before", [0, 10])
def test_standard_mpm_one_substep_matches_oracle(model, steps_before):
    sc = W.elastic_cube(model=model)
    sc["rigids"] = [W.sphere((0.5 + 0.013, 0.36, 0.5 - 0.007), 0.05, vel=(0.0, -0.2, 0.0), margin=1 / 32)]
    v, C, F = perturbed(sc, seed=51, f_amp=0.01, c_amp=0.0)
    st, out = gpu_step(sc, v, C, F, "standard", steps_before)
    ost = oracle_state(sc, st["x"], st["v"], st["C"], st["F"])
    rig, nr = oracle_rigids(sc, steps_before)
    assert oracle.run_solver(oracle_cfg(sc), ost, sc["dt"], 1, "standard", rig, nr) == 0
    err = Scales(sc, st["F"])
    assert_close("x", out["x"], ost.x)
    assert_close("v", out["v"], ost.v, atol_floor=err.atol_v(ost.v))
    # L = n sum v_I dW: the same cancellation as the APIC C, without the factor 4
    assert_close("L", out["C"], ost.C, atol_floor=err.atol_C(ost.v))
    assert_close("F", out["F"], ost.F)
    assert_close("impulse", out["impulse"][0], oracle.rigid_impulse(rig[0]), rtol=1e-4, rel_scale=1e-4)


def test_standard_mpm_trajectory():
    # The elastic cube falling onto the sticky floor for 100 substeps: the
    # whole-run criterion of the MLS-MPM parity tests (1e-3 dx).
    sc = W.elastic_cube()
    with mpm.from_workload(sc, solver="standard") as sim:
        sim.substep(sc["dt"], sc["substeps"])
        got = sim.read_state(0, ("x",))
    st = oracle_state(sc)
    assert oracle.run_solver(oracle_cfg(sc), st, sc["dt"], sc["substeps"], "standard") == 0
    err = np.max(np.abs(got["x"] - st.x))
    assert err <= 1e-3 / sc["n"], err
    assert np.max(np.abs(st.x - sc["x"])) > 10 * err


def pb_scene(N=6000, seed=53):
    sc = W.paper_timing_cube(N=N, steps=1)
    sc["dt"] = 0.02  # PB-MPM takes the whole 0.02 s step at once (Sec. III-D)
    return sc


@pytest.mark.parametrize("iters,beta", [(1, 1.0), (10, 1.0), (20, 0.6)])
def test_pb_mpm_one_step_matches_oracle(iters, beta):
    sc = pb_scene()
    sc["rigids"] = [W.box((0.5 + 0.21 / 56, 0.62 - 0.13 / 56, 0.5 + 0.07 / 56), (0.08, 0.05, 0.1),
                          quat=(0.96, 0.1, 0.2, 0.15), vel=(0.0, -0.5, 0.1), mu_k=0.3, margin=0.5 / 56)]
    v, C, F = perturbed(sc, seed=54, f_amp=0.01, c_amp=0.5, v_amp=0.05)
    st, out = gpu_step(sc, v, C, F, "pb", pb_iterations=iters, pb_beta=beta)
    ost = oracle_state(sc, st["x"], st["v"], st["C"], st["F"])
    rig, nr = oracle_rigids(sc)
    assert oracle.run_solver(oracle_cfg(sc), ost, sc["dt"], 1, "pb", rig, nr, iters=iters, beta=beta) == 0
    # The constraint divides by dt: its FP32 rounding of F* (a few units of
    # 2^-24 of |F|) becomes up to ~8 eps / dt in C per cycle, carried into v
    # by the APIC transfer (|C| dx) and into F by dt C.
    c_floor = 8 * EPS32 / sc["dt"] * iters
    assert_close("x", out["x"], ost.x)
    assert_close("v", out["v"], ost.v, atol_floor=c_floor / sc["n"] + 2e-5 * np.abs(ost.v).max())
    assert_close("C", out["C"], ost.C, atol_floor=4 * c_floor + 27 * 4 * sc["n"] * EPS32 * np.abs(ost.v).max())
    assert_close("F", out["F"], ost.F, atol_floor=c_floor * sc["dt"])
    assert_close("impulse", out["impulse"][0], oracle.rigid_impulse(rig[0]), rtol=1e-3, rel_scale=1e-3)


def test_pb_mpm_falling_cube_steps():
    # Five 0.02 s steps of the falling cube with 10 cycles each: positions track
    # the oracle to a small fraction of a cell.
    sc = pb_scene(N=4000, seed=55)
    with mpm.from_workload(sc, solver="pb", pb_iterations=10, pb_beta=0.9) as sim:
        sim.substep(sc["dt"], 5)
        got = sim.read_state(0, ("x", "v"))
    st = oracle_state(sc)
    assert oracle.run_solver(oracle_cfg(sc), st, sc["dt"], 5, "pb", iters=10, beta=0.9) == 0
    err = np.max(np.abs(got["x"] - st.x))
    assert err <= 1e-3 / sc["n"], err
    assert np.max(np.abs(st.x - sc["x"])) > 10 * err


def test_solver_options_are_checked():
    with pytest.raises(mpm.MPMError):
        mpm.Simulation(32, 10, solver=3)
    with pytest.raises(mpm.MPMError):
        mpm.Simulation(32, 10, solver="pb", pb_beta=1.5)
    with pytest.raises(mpm.MPMError):
        mpm.Simulation(32, 10, solver="pb", plasticity=True, yield_stress=10.0)
    with mpm.Simulation(32, 10, solver="standard") as sim:
        with pytest.raises(mpm.MPMError):
            sim.set_option("fused", 1)
