"""GPU (CUDA, through the C ABI) vs FP64 oracle parity of the MLS-MPM substep.

Element-by-element comparison of every particle field after one substep from
identical FP32 inputs, at sizes the oracle finishes in seconds that still span
many bricks and ragged (partially filled) bricks, plus the whole-run criterion
on the elastic-cube workload and sampled checks at the full 1M-particle size.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2502_18437_gb300 import mpm, workloads as W
from tests.parity_util import Scales, assert_close, oracle_cfg, oracle_rigids, oracle_state, perturbed

pytestmark = pytest.mark.gpu


def gpu_one_step(sc, v, C, F, steps_before=0, **opts):
    """Write (v, C, F), run steps_before substeps, read the state, run one more
    substep; returns the state before that substep and the GPU result."""
    with mpm.from_workload(sc) as sim:
        for k, val in opts.items():
            sim.set_option(k, val)
        sim.write_state(0, v=v, C=C, F=F)
        if steps_before:
            sim.substep(sc["dt"], steps_before)
        st = sim.read_state(0)
        sim.impulse(0)  # reset the accumulated impulse
        sim.substep(sc["dt"], 1)
        out = sim.read_state(0)
        out["grid"] = sim.read_grid(0)
        out["impulse"] = sim.impulse(0)
    return st["x"], st["v"], st["C"], st["F"], out


def oracle_one_step(sc, x, v, C, F, steps_before=0):
    cfg = oracle_cfg(sc)
    st = oracle_state(sc, x, v, C, F)
    rig, nr = oracle_rigids(sc, steps_before)
    gm, gv, err = oracle.substep(cfg, st, sc["dt"], rig, nr)
    imp = np.array([oracle.rigid_impulse(rig[i]) for i in range(nr)]) if nr else np.zeros((0, 6))
    return st, gm, gv, err, imp


def check_fields(sc, out, st, sc_err):
    assert_close("x", out["x"], st.x)
    assert_close("v", out["v"], st.v, atol_floor=sc_err.atol_v(st.v))
    assert_close("C", out["C"], st.C, atol_floor=sc_err.atol_C(st.v))
    assert_close("F", out["F"], st.F)


def check_grid(sc, out, gm, gv, sc_err):
    n = sc["n"]
    g = out["grid"].reshape(-1, 4).astype(np.float64)
    # grid mass and momentum sums within 1e-6 relative; per node within FP32 tolerance
    assert abs(g[:, 3].sum() - gm.sum()) <= 1e-6 * gm.sum()
    mom_g = (g[:, :3] * g[:, 3:4]).sum(0)
    mom_o = (gv * gm[:, None]).sum(0)
    assert np.max(np.abs(mom_g - mom_o)) <= 1e-6 * np.abs(gv * gm[:, None]).sum(0).max() + 1e-12
    assert_close("grid m", g[:, 3], gm)
    assert_close("grid v", g[:, :3], gv, atol_floor=sc_err.atol_v(gv))
    assert g.shape[0] == n ** 3


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
def test_cube_one_substep_all_fields(model):
    sc = W.elastic_cube(model=model)
    v, C, F = perturbed(sc, seed=11)
    x, v, C, F, out = gpu_one_step(sc, v, C, F)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    check_grid(sc, out, gm, gv, Scales(sc, F))


def test_cube_100_substeps_position_error():
    # Whole-run criterion: max particle position error <= 1e-3 dx after 100 substeps.
    sc = W.elastic_cube()
    with mpm.from_workload(sc) as sim:
        sim.substep(sc["dt"], sc["substeps"])
        got = sim.read_state(0, ("x", "v"))
    st = oracle_state(sc)
    assert oracle.run(oracle_cfg(sc), st, sc["dt"], sc["substeps"]) == 0
    dx = 1.0 / sc["n"]
    err = np.max(np.abs(got["x"] - st.x))
    assert err <= 1e-3 * dx, err
    assert np.max(np.abs(st.x - sc["x"])) > 10 * err  # the cube did move


@pytest.mark.parametrize("steps_before", [0, 12, 40])
def test_slab_with_blade_and_thread(steps_before):
    # Tissue slab (Neo-Hookean, per-particle E) cut by the slicer and pushed by
    # the capsule-chain thread; one substep from the same state at several
    # points of the trajectory, including the impulse given to each rigid.
    sc = W.tissue_slab(cells=(40, 8, 40), lo=(0.25, 0.15, 0.25), size=(0.5, 0.1, 0.5), n=64, substeps=50)
    # blade edge already 0.03 deep in the tissue; its mid-plane lies between grid planes
    c = sc["rigids"][0]["center"]
    sc["rigids"][0]["center"] = (c[0], 0.15 + 0.1 - 0.03 + 0.04, c[2])
    N = len(sc["x"])
    g = np.random.default_rng(5)
    v0 = (0.05 * g.normal(size=(N, 3))).astype(np.float32)
    x, v, C, F, out = gpu_one_step(sc, v0, np.zeros((N, 3, 3), np.float32),
                                   np.tile(np.eye(3, dtype=np.float32), (N, 1, 1)), steps_before=steps_before)
    st, gm, gv, err, imp = oracle_one_step(sc, x, v, C, F, steps_before)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    check_grid(sc, out, gm, gv, Scales(sc, F))
    assert np.abs(imp[:, :3]).max() > 0  # there is contact
    for r in range(len(sc["rigids"])):
        assert_close(f"impulse[{r}]", out["impulse"][r], imp[r], rtol=1e-4, rel_scale=1e-4)


@pytest.mark.parametrize("steps_before", [0, 30])
def test_plastic_block(steps_before):
    sc = W.tissue_block(N=65536, n=64)
    v, C, F = perturbed(sc, seed=3, f_amp=0.03, c_amp=5.0)
    x, v, C, F, out = gpu_one_step(sc, v, C, F, steps_before=steps_before)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    check_grid(sc, out, gm, gv, Scales(sc, F))


def test_full_size_1m_block_one_substep():
    # Full-size scale-sweep case (1M particles, 256^3) in the launch shape the
    # benchmark times (graphs, default options): every particle checked.
    sc = W.tissue_block(N=1048576, n=256)
    v, C, F = perturbed(sc, seed=7, f_amp=0.03, c_amp=5.0)
    x, v, C, F, out = gpu_one_step(sc, v, C, F)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    assert abs(out["grid"][..., 3].sum() - gm.sum()) <= 1e-6 * gm.sum()


def test_sort_by_brick_order():
    # After a substep particles are stored sorted by the brick of their base
    # cell at the start of that substep: compare the key sequence and counts.
    sc = W.tissue_block(N=65536, n=64)
    with mpm.from_workload(sc) as sim:
        sim.substep(sc["dt"], 1)
        order = sim.read_state(0, ("order",))["order"]
    key, perm, count = oracle.sort_by_brick(sc["n"], sc["x"])
    assert np.array_equal(np.sort(order), np.arange(len(order)))
    assert np.array_equal(key[order], key[perm])  # identical key sequence (same bricks, same offsets)


def dense_bricks_scene():
    """Bricks far above the P2G pass size and single cells far above the mean:
    1,700 particles in one 4^3-cell brick, 400 in one cell, 100 scattered."""
    n = 32
    dx = 1.0 / n
    g = np.random.default_rng(41)
    brick = (4.5 + 4.0 * g.random((1700, 3))) * dx   # base cells 4..7: one brick
    cell = (10.5 + g.random((400, 3))) * dx          # base cell (10, 10, 10)
    sparse = (6.0 + 18.0 * g.random((100, 3))) * dx
    x = np.concatenate([brick, cell, sparse])
    return W._scene(n, x, np.zeros_like(x), 1e4, 0.3, rho=1.0, V0=(dx / 2) ** 3, model="fixed_corotated",
                    dt=1e-4, substeps=1, name="dense_bricks")


@pytest.mark.parametrize("chunk", [384, 576, 768])
def test_p2g_dense_bricks_and_heavy_cells(chunk):
    # several P2G passes per brick, items cut from a 400-particle cell
    sc = dense_bricks_scene()
    v, C, F = perturbed(sc, seed=12)
    x, v, C, F, out = gpu_one_step(sc, v, C, F, p2g_chunk=chunk)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    check_grid(sc, out, gm, gv, Scales(sc, F))


def test_graph_direct_and_looped_agree():
    sc = W.tissue_slab(cells=(32, 6, 32), lo=(0.3, 0.2, 0.3), size=(0.4, 0.08, 0.4), n=32, substeps=20)
    outs = []
    for opts in ({"use_graphs": 1}, {"use_graphs": 0}, {"launch_mode": 1}, {"fused": 0},
                 {"fused": 0, "p2g_chunk": 384}, {"fused": 0, "p2g_chunk": 768}):
        with mpm.from_workload(sc) as sim:
            for k, v in opts.items():
                sim.set_option(k, v)
            sim.substep(sc["dt"], 20)
            outs.append(sim.read_state(0))
    for o in outs[1:]:
        for f in ("x", "v", "F"):
            assert_close(f, o[f], outs[0][f], rtol=1e-4, rel_scale=1e-4)


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
@pytest.mark.parametrize("eps", [0.0, 1e-30, 1e-20, 1e-12, 1e-7, 1e-3])
def test_stress_near_identity_matches_oracle(model, eps):
    # F = I + eps N(0,1): from exact identity through perturbations that underflow
    # when squared inside the FP32 SVD, to ordinary strains.  One substep from
    # identical inputs; every field finite and within tolerance.
    sc = W.elastic_cube(model=model, n_side=12)
    N = len(sc["x"])
    g = np.random.default_rng(int(1e6 * eps) % 1000 + 1)
    F = (np.eye(3) + eps * g.normal(size=(N, 3, 3))).astype(np.float32)
    C = np.zeros((N, 3, 3), np.float32)
    v = sc["v"]
    x, v, C, F, out = gpu_one_step(sc, v, C, F)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    for f in ("x", "v", "C", "F"):
        assert np.all(np.isfinite(out[f])), f
    check_fields(sc, out, st, Scales(sc, F))


def test_degenerate_F_fixed_corotated():
    # Rank-deficient and inverted F (fixed-corotated handles both): finite and
    # equal to the oracle's rotation-variant SVD result.
    sc = W.elastic_cube(n_side=8)
    N = len(sc["x"])
    g = np.random.default_rng(9)
    base = [np.diag([1.0, 1.0, 0.0]), np.diag([1.2, 0.9, -0.8]), np.diag([1.0, 1.0, 1.0]) * 0.5,
            np.array([[1.0, 1.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])]
    F = np.stack([base[i % len(base)] + 1e-4 * g.normal(size=(3, 3)) for i in range(N)]).astype(np.float32)
    C = np.zeros((N, 3, 3), np.float32)
    x, v, C, F, out = gpu_one_step(sc, sc["v"], C, F)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))


def _rotation(g):
    q, r = np.linalg.qr(g.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
@pytest.mark.parametrize("plastic", [False, True])
def test_stress_exact_eigen_structures_matches_oracle(model, plastic):
    # F = R diag(s) Q^T with exactly repeated, symmetric and separated singular
    # values: the left stretch's eigenvalues are double (larger or smaller pair),
    # triple (isotropic, a scaled rotation), evenly spaced around their mean, or
    # generic, and one case is a pure rotation.  The closed-form eigen-decomposition
    # meets its special cases here (deviator zero, the cubic's cosine at +-1 and 0);
    # every field equals the oracle's one substep, with and without the von Mises
    # return map (yield low enough that the larger strains yield).
    sc = W.elastic_cube(model=model, n_side=10)
    if plastic:
        sc = dict(sc, plasticity=True, yield_stress=20.0)
    N = len(sc["x"])
    g = np.random.default_rng(31)
    sv = [(1.2, 1.2, 0.8), (1.2, 0.8, 0.8), (0.9, 0.9, 0.9), (0.9, 1.0, 1.1), (1.5, 1.0, 0.6),
          (1.0, 1.0, 1.0), (1.0, 1.0 + 1e-4, 1.0 + 1e-4)]
    if model == "fixed_corotated" and not plastic:
        sv.append((1.1, 0.9, -0.7))  # inverted
    F = np.stack([_rotation(g) @ np.diag(sv[i % len(sv)]) @ _rotation(g).T for i in range(N)]).astype(np.float32)
    C = np.zeros((N, 3, 3), np.float32)
    x, v, C, F, out = gpu_one_step(sc, sc["v"], C, F)
    st, gm, gv, err, _ = oracle_one_step(sc, x, v, C, F)
    assert err == 0
    for f in ("x", "v", "C", "F"):
        assert np.all(np.isfinite(out[f])), f
    check_fields(sc, out, st, Scales(sc, F))


@pytest.mark.parametrize("steps_before", [0, 15])
def test_box_contact_matches_oracle(steps_before):
    # A rotated box (Sec. IV-A, solid SDF, Eq. 11 friction) pressed down into a
    # soft cube while turning: inside-face, edge and corner normals all occur.
    # One substep from the same state at two points of the trajectory, the
    # box's impulse included.
    sc = W.elastic_cube(n=32, n_side=14, corner=(0.32, 0.1, 0.33), substeps=40)
    q = np.array([0.96, 0.12, 0.2, -0.15])
    q /= np.linalg.norm(q)
    sc["rigids"] = [W.box((0.43 + 0.21 / 32, 0.37 - 0.37 / 32, 0.43 - 0.13 / 32), (0.1, 0.06, 0.08),
                          quat=tuple(q), vel=(0.02, -0.3, 0.0), omega=(0.0, 1.5, 0.5), mu_k=0.4, c_d=0.9,
                          margin=0.5 / 32)]
    v, C, F = perturbed(sc, seed=21, f_amp=0.01, c_amp=1.0)
    x, v, C, F, out = gpu_one_step(sc, v, C, F, steps_before=steps_before)
    st, gm, gv, err, imp = oracle_one_step(sc, x, v, C, F, steps_before)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    check_grid(sc, out, gm, gv, Scales(sc, F))
    assert np.abs(imp[0, :3]).max() > 0  # in contact
    assert_close("box impulse", out["impulse"][0], imp[0], rtol=1e-4, rel_scale=1e-4)


@pytest.mark.parametrize("shape", ["sphere", "box"])
@pytest.mark.parametrize("steps_before", [0, 8])
def test_push_out_matches_oracle(shape, steps_before):
    # A solid rigid sweeping through a block of particles, many of which start
    # inside it: after each substep the particles left inside are pushed to its
    # surface at its pose at the end of the substep (Sec. IV-A particle
    # correction).  One substep from the same state at two points of the run.
    sc = W.elastic_cube(n=32, n_side=14, corner=(0.32, 0.3, 0.33), substeps=20)
    if shape == "sphere":
        rig = W.sphere((0.43 + 0.17 / 32, 0.42 - 0.23 / 32, 0.44 + 0.11 / 32), 0.07, vel=(0.3, -0.4, 0.1),
                       mu_k=0.2, margin=0.25 / 32)
    else:
        q = np.array([0.93, -0.2, 0.25, 0.18])
        rig = W.box((0.43 + 0.17 / 32, 0.42 - 0.23 / 32, 0.44 + 0.11 / 32), (0.06, 0.04, 0.07),
                    quat=tuple(q / np.linalg.norm(q)), vel=(-0.2, -0.3, 0.2), omega=(1.0, -2.0, 0.5), mu_k=0.2,
                    margin=0.25 / 32)
    sc["rigids"] = [rig]
    v, C, F = perturbed(sc, seed=41, f_amp=0.01, c_amp=1.0)
    x, v, C, F, out = gpu_one_step(sc, v, C, F, steps_before=steps_before)
    st, gm, gv, err, imp = oracle_one_step(sc, x, v, C, F, steps_before)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    check_grid(sc, out, gm, gv, Scales(sc, F))
    # nobody is left inside the rigid at its new pose
    r = oracle.make_rigid(rig)
    for _ in range(steps_before + 1):
        oracle.rigid_advance(r, sc["dt"])
    inside = [oracle.geometry(r, p)[3] for p in out["x"].astype(np.float64)]
    assert min(inside) > -1e-6
    assert np.sum(np.abs(inside) < 1e-6) > 20  # the pushed particles sit on the surface


def _suturing_scene():
    # Small tissue slab with a curved needle (Arc, Sec. IV-C) turning about its
    # own circle axis, i.e. sliding along its tangent as in an insertion, and
    # a curved blade given as a triangle mesh (TriangleMeshSlicer, Sec. IV-B)
    # moving down into the tissue with its spine up.
    n = 64
    sc = W.tissue_slab(cells=(40, 8, 40), lo=(0.25, 0.15, 0.25), size=(0.5, 0.1, 0.5), n=n, substeps=40,
                       with_tools=False)
    dx = 1.0 / n
    # needle: circle of radius 0.05 in a vertical plane, half of it below the top surface
    qn = (math.cos(0.2), 0.0, math.sin(0.2), 0.0)  # plane turned about world y
    needle = W.arc((0.37 + 0.31 * dx, 0.25 + 0.02 + 0.17 * dx, 0.41 - 0.23 * dx), qn, arc_radius=0.05, start=-2.6,
                   sweep=2.2, radius=0.002, omega=(0.0, 0.0, 0.0), mu_k=0.3, c_d=1.0, margin=dx)
    # its body z axis in world coordinates: turning about it moves the arc along its tangent
    w, x, y, z = qn
    axis = np.array([2 * (x * z + w * y), 2 * (y * z - w * x), 1 - 2 * (x * x + y * y)])
    needle["omega"] = tuple(4.0 * axis)
    pts, tris, spine = W.curved_blade_mesh(half_edge=0.07, depth=0.05, bend=0.015)
    # blade: edge (body +y) pointing down, normal along world x, slightly turned
    blade = W.mesh_slicer((0.62 + 0.37 * dx, 0.25 + 0.025 - 0.015 + 0.11 * dx, 0.58 + 0.21 * dx),
                          (0.0, math.sqrt(0.5), 0.05, math.sqrt(0.5)), pts, tris, spine, thickness=0.003,
                          spine_radius=0.002, vel=(0.0, -0.1, 0.02), mu_k=0.3, c_d=1.0, margin=dx)
    q = np.array(blade["quat"])
    blade["quat"] = tuple(q / np.linalg.norm(q))
    sc["rigids"] = [needle, blade]
    return sc


@pytest.mark.parametrize("steps_before", [0, 10])
def test_arc_needle_and_mesh_slicer_match_oracle(steps_before):
    sc = _suturing_scene()
    N = len(sc["x"])
    g = np.random.default_rng(61)
    v0 = (0.05 * g.normal(size=(N, 3))).astype(np.float32)
    x, v, C, F, out = gpu_one_step(sc, v0, np.zeros((N, 3, 3), np.float32),
                                   np.tile(np.eye(3, dtype=np.float32), (N, 1, 1)), steps_before=steps_before)
    st, gm, gv, err, imp = oracle_one_step(sc, x, v, C, F, steps_before)
    assert err == 0
    check_fields(sc, out, st, Scales(sc, F))
    check_grid(sc, out, gm, gv, Scales(sc, F))
    for r in range(2):
        assert np.abs(imp[r, :3]).max() > 0, r  # both tools are in contact
        assert_close(f"impulse[{r}]", out["impulse"][r], imp[r], rtol=1e-4, rel_scale=1e-4)
