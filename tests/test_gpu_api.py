"""GPU tests of the C ABI's behaviour: batching, ragged and empty scenes, error
reporting, state round trips, autotuning.  All through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2502_18437_gb300 import mpm, workloads as W
from tests.parity_util import assert_close, oracle_cfg, oracle_state

pytestmark = pytest.mark.gpu


def small_cube(N_side=6, corner=(0.4, 0.4, 0.4), n=32):
    sc = W.elastic_cube(n=n, n_side=N_side, corner=corner, substeps=10)
    return sc


def test_batched_scenes_match_oracle_per_scene():
    # Ragged batch in one context: an empty scene, one particle, a few, a full
    # cube with a rigid sphere, and a 64^3 scene.  One substep from perturbed
    # states; every scene must match the oracle run on that scene alone.
    from tests.parity_util import Scales, oracle_rigids, perturbed

    scenes = [small_cube(0), small_cube(1), small_cube(3, (0.2, 0.5, 0.6)), W.elastic_cube(), small_cube(7, n=64)]
    scenes[3]["rigids"] = [W.sphere((0.5 + 0.013, 0.12, 0.5 - 0.007), 0.05, margin=1 / 32)]
    pert = [perturbed(sc, seed=s) if len(sc["x"]) else None for s, sc in enumerate(scenes)]
    with mpm.from_scenes(scenes) as sim:
        for s, p in enumerate(pert):
            if p is not None:
                sim.write_state(s, v=p[0], C=p[1], F=p[2])
        sim.substep(1e-4, 1)
        batched = [sim.read_state(s) for s in range(len(scenes))]
    for s, sc in enumerate(scenes):
        assert len(batched[s]["x"]) == len(sc["x"])
        if len(sc["x"]) == 0:
            continue
        st = oracle_state(sc, sc["x"], *pert[s])
        rig, nr = oracle_rigids(sc)
        assert oracle.substep(oracle_cfg(sc), st, 1e-4, rig, nr)[2] == 0
        err = Scales(sc, pert[s][2], 1e-4)
        for f in ("x", "F"):
            assert_close(f"scene {s} {f}", batched[s][f], getattr(st, f))
        assert_close(f"scene {s} v", batched[s]["v"], st.v, atol_floor=err.atol_v(st.v))
        assert_close(f"scene {s} C", batched[s]["C"], st.C, atol_floor=err.atol_C(st.v))


def test_batched_multi_step_tracks_single_runs():
    # Many substeps: batched and single-scene runs stay close (they differ only
    # by the order of floating-point atomics).
    scenes = [small_cube(4, (0.3, 0.4, 0.3)), W.elastic_cube(n_side=8), small_cube(5, n=64)]
    with mpm.from_scenes(scenes) as sim:
        sim.substep(1e-4, 30)
        batched = [sim.read_state(s, ("x",)) for s in range(len(scenes))]
    for s, sc in enumerate(scenes):
        with mpm.from_workload(sc) as sim:
            sim.substep(1e-4, 30)
            alone = sim.read_state(0, ("x",))
        assert np.max(np.abs(batched[s]["x"] - alone["x"])) < 1e-4 / sc["n"]


def test_batched_looped_mode_matches():
    scenes = W.batched_scenes(n_scenes=6, substeps=10)
    res = []
    for mode in (0, 1):
        with mpm.from_scenes(scenes) as sim:
            sim.set_option("launch_mode", mode)
            sim.substep(1e-4, 10)
            res.append([sim.read_state(s, ("x",)) for s in range(len(scenes))])
    for s in range(len(scenes)):
        assert np.max(np.abs(res[1][s]["x"] - res[0][s]["x"])) < 1e-4 / scenes[s]["n"]


def test_single_particle_free_fall_matches_closed_form():
    # A lone particle of a soft material (explicit step well inside its CFL limit).
    sc = W.elastic_cube(n=32, n_side=1, corner=(0.5, 0.5, 0.5), E=10.0, substeps=10)
    with mpm.from_workload(sc) as sim:
        sim.substep(1e-3, 10)
        st = sim.read_state(0)
    g = -9.8
    assert abs(st["v"][0, 1] - 10 * 1e-3 * g) < 1e-5
    assert abs(st["x"][0, 1] - (sc["x"][0, 1] + 1e-6 * g * 55)) < 1e-6


def test_empty_context_substeps():
    with mpm.Simulation(32, 16) as sim:
        sim.substep(1e-4, 3)
        out = sim.read_state(0, ("x",))
        assert out["x"].shape == (0, 3)


def test_write_read_roundtrip_and_order():
    sc = W.elastic_cube(n_side=8)
    g = np.random.default_rng(0)
    N = len(sc["x"])
    with mpm.from_workload(sc) as sim:
        sim.substep(1e-4, 3)  # storage order is now the sorted order
        vals = {"x": sc["x"] + 0.001 * g.random((N, 3)).astype(np.float32),
                "v": g.normal(size=(N, 3)).astype(np.float32),
                "C": g.normal(size=(N, 3, 3)).astype(np.float32),
                "F": g.normal(size=(N, 3, 3)).astype(np.float32)}
        sim.write_state(0, **vals)
        out = sim.read_state(0)
        for f, a in vals.items():
            assert np.array_equal(out[f], a), f


def test_device_tensors_roundtrip():
    torch = pytest.importorskip("torch")
    sc = W.elastic_cube(n_side=8)
    with mpm.from_workload(sc) as sim:
        sim.substep(1e-4, 2)
        host = sim.read_state(0)
        dev = sim.read_state(0, device=True)
        for f in ("x", "v", "C", "F"):
            assert np.array_equal(dev[f].cpu().numpy(), host[f])
        sim.write_state(0, v=dev["v"] * 2)
        assert np.array_equal(sim.read_state(0, ("v",))["v"], 2 * host["v"])


@pytest.mark.parametrize("misalign", [False, True])
def test_pinned_host_state_io_matches_staged_path(misalign):
    # Pinned host arrays take the one-kernel path over the host link (state <->
    # id-ordered arrays through the id inverse); pageable ones the staged path.
    # Two scenes (the second starts at a nonzero slot), counts that are not
    # multiples of the kernel's 128-id blocks, storage permuted by the sort; with
    # misalign the arrays start 4 bytes into their allocation (no 16-byte words).
    torch = pytest.importorskip("torch")
    scenes = [W.elastic_cube(n_side=7), W.elastic_cube(n_side=9, corner=(0.3, 0.12, 0.3))]
    g = np.random.default_rng(5)
    shapes = {"x": (3,), "v": (3,), "C": (3, 3), "F": (3, 3)}
    masks = {"x": mpm.FIELD["x"], "v": mpm.FIELD["v"], "C": mpm.FIELD["C"], "F": mpm.FIELD["F"]}

    def pinned(n, shape):
        k = int(np.prod(shape))
        t = torch.empty(n * k + (1 if misalign else 0), dtype=torch.float32).pin_memory()
        a = t.numpy()[(1 if misalign else 0):].reshape((n,) + shape)
        return t, a

    with mpm.from_scenes(scenes) as sim:
        sim.substep(1e-4, 4)
        for scene, sc in enumerate(scenes):
            N = len(sc["x"])
            ref = sim.read_state(scene)  # pageable: staged path
            keep, arrs = [], {}
            for f, sh in shapes.items():
                t, a = pinned(N, sh)
                keep.append(t)
                arrs[f] = a
            st = mpm.mpm_read_state(sim.h, scene, 15, [arrs[f].ctypes.data for f in ("x", "v", "C", "F")],
                                    mpm.MEM_HOST)
            assert st == 0
            for f in shapes:
                assert np.array_equal(arrs[f], ref[f]), (scene, f)
            # write new values from pinned arrays, one field alone and then all four
            vals = {"x": (sc["x"] + 0.001 * g.random((N, 3))).astype(np.float32),
                    "v": (0.1 * g.normal(size=(N, 3))).astype(np.float32),
                    "C": (0.1 * g.normal(size=(N, 3, 3))).astype(np.float32),
                    "F": (np.eye(3) + 0.01 * g.normal(size=(N, 3, 3))).astype(np.float32)}
            arrs["v"][...] = vals["v"]
            assert mpm.mpm_write_state(sim.h, scene, masks["v"], [arrs["v"].ctypes.data], mpm.MEM_HOST) == 0
            assert np.array_equal(sim.read_state(scene, ("v",))["v"], vals["v"])
            for f in shapes:
                arrs[f][...] = vals[f]
            assert mpm.mpm_write_state(sim.h, scene, 15, [arrs[f].ctypes.data for f in ("x", "v", "C", "F")],
                                       mpm.MEM_HOST) == 0
            out = sim.read_state(scene)
            for f in shapes:
                assert np.array_equal(out[f], vals[f]), (scene, f)
        # the other scene is untouched by these writes; substeps still run
        sim.substep(1e-4, 2)
        assert sim.error_bits(0) == 0 and sim.error_bits(1) == 0


def test_out_of_domain_reported():
    sc = small_cube(2, (0.0, 0.5, 0.5))  # first layer's base cell is -1
    with mpm.from_workload(sc) as sim:
        sim.substep(1e-4, 1)
        out = sim.read_state(0, ("x",), check=False)
        assert out["status"] == -4
        assert sim.error_bits(0) & mpm.EBIT["out_of_domain"]


def test_nonfinite_reported():
    sc = small_cube(2)
    v = sc["v"].copy()
    v[0, 0] = np.nan
    with mpm.from_workload(sc) as sim:
        sim.write_state(0, v=v)
        sim.substep(1e-4, 1)
        assert sim.read_state(0, ("x",), check=False)["status"] == -5


def test_neo_hookean_inversion_reported():
    sc = small_cube(2)
    sc["model"] = "neo_hookean"
    N = len(sc["x"])
    F = np.tile(np.diag([1.0, 1.0, -1.0]).astype(np.float32), (N, 1, 1))
    with mpm.from_workload(sc) as sim:
        sim.write_state(0, F=F)
        sim.substep(1e-5, 1)
        assert sim.read_state(0, ("x",), check=False)["status"] == -6


def test_invalid_arguments():
    with pytest.raises(mpm.MPMError) as e:
        mpm.Simulation(30, 10)  # n not a multiple of 4
    assert e.value.status == -1
    with mpm.Simulation(32, 10) as sim:
        with pytest.raises(mpm.MPMError) as e:
            sim.add_particles(0, np.full((11, 3), 0.5, np.float32), E0=1e3, nu0=0.3, rho=1, V0=1e-6)
        assert e.value.status == -7  # capacity
        with pytest.raises(mpm.MPMError):
            sim.add_particles(1, np.full((1, 3), 0.5, np.float32), E0=1e3, nu0=0.3, rho=1, V0=1e-6)
        with pytest.raises(mpm.MPMError):
            sim.substep(-1.0, 1)
        with pytest.raises(mpm.MPMError):
            sim.set_option("p2g_threads", 100)
        with pytest.raises(mpm.MPMError):
            sim.set_option("p2g_chunk", 192)
        sim.set_option("g2p_threads", 512)
        assert sim.get_option("g2p_threads") == 512
        with pytest.raises(mpm.MPMError):
            sim.get_option(99)
        with pytest.raises(mpm.MPMError) as e:
            sim.backward()
        assert e.value.status in (-1, -9)


def test_autotune_restores_state():
    sc = W.tissue_block(N=65536, n=64)
    with mpm.from_workload(sc) as sim:
        sim.substep(sc["dt"], 5)
        before = sim.read_state(0)
        ms = sim.autotune(sc["dt"], 3)
        assert ms > 0
        # the chosen launch shape is one of the candidates
        assert sim.get_option("p2g_chunk") in (384, 576, 768)
        assert sim.get_option("g2p_threads") in (128, 256, 512)
        assert sim.get_option("g2p_regs64") in (0, 1) and sim.get_option("ctas_per_sm") in (0, 2)
        after = sim.read_state(0)
        for f in ("x", "v", "C", "F"):
            assert np.array_equal(before[f], after[f])
        sim.substep(sc["dt"], 5)
        tuned = sim.read_state(0)
    with mpm.from_workload(sc) as sim:
        sim.substep(sc["dt"], 10)
        ref = sim.read_state(0)
    for f in ("x", "v"):
        assert_close(f, tuned[f], ref[f], rtol=1e-5, rel_scale=1e-5)


def test_rigid_motion_follows_set_velocity():
    # A sphere moving at constant velocity into resting particles: the particles
    # it touches end up moving with it (grid-level coupling, Sec. IV-A).
    sc = W.elastic_cube(n=32, n_side=10, corner=(0.4, 0.3, 0.4), substeps=1)
    sc["gravity"] = (0.0, 0.0, 0.0)
    sc["rigids"] = [W.sphere((0.5, 0.25, 0.5), 0.06, vel=(0.0, 0.5, 0.0), mu_k=0.0, margin=0.0)]
    with mpm.from_workload(sc) as sim:
        sim.substep(1e-4, 400)
        st = sim.read_state(0)
        imp = sim.impulse(0)
    assert st["v"][:, 1].max() > 0.2
    assert imp[0, 1] < 0  # the soft body pushes back on the rigid


def test_bounded_wait_times_out_on_a_host_stall():
    # A host function enqueued on the context's stream blocks it for longer than
    # the context's timeout (only the host waits; no GPU work stalls).  The
    # blocking read must give up with TIMEOUT instead of waiting it out, and the
    # next read succeeds once the stream has drained.
    import ctypes
    import threading
    import time

    torch = pytest.importorskip("torch")
    cuda = ctypes.CDLL("libcuda.so.1")
    hostfn_t = ctypes.CFUNCTYPE(None, ctypes.c_void_p)
    release = threading.Event()
    cb = hostfn_t(lambda _: release.wait(10.0))  # bounded even if the test failed to release it
    cuda.cuLaunchHostFunc.argtypes = [ctypes.c_void_p, hostfn_t, ctypes.c_void_p]
    cuda.cuLaunchHostFunc.restype = ctypes.c_int
    stream = torch.cuda.Stream()
    sc = small_cube(4)
    with mpm.from_workload(sc, stream=stream.cuda_stream, timeout_ms=200) as sim:
        sim.substep(1e-4, 2)
        assert cuda.cuLaunchHostFunc(stream.cuda_stream, cb, None) == 0
        try:
            t0 = time.perf_counter()
            out = sim.read_state(0, ("x",), check=False)
            waited = time.perf_counter() - t0
            assert out["status"] == -8, mpm.STATUS.get(out["status"])
            assert 0.15 < waited < 3.0, waited
            with pytest.raises(mpm.MPMError) as e:
                sim.error_bits(0)
            assert e.value.status == -8
        finally:
            release.set()
        stream.synchronize()
        out = sim.read_state(0, ("x", "v"))
        assert np.all(np.isfinite(out["x"])) and sim.error_bits(0) == 0


def test_batched_slicers_match_oracle_per_scene():
    # Scenes of the batched workload (ragged counts, 32^3 and 64^3 grids, one
    # yawed QuadSlicer each), with every blade lowered into its block so that
    # its faces and edge touch tissue: one substep from perturbed
    # states in one batched launch per phase, every scene against the oracle run
    # on that scene alone, the blades' impulses included.
    from tests.parity_util import Scales, oracle_rigids, perturbed

    scenes = W.batched_scenes(n_scenes=8, substeps=1)
    for sc in scenes:
        b = sc["rigids"][0]
        top = float(sc["x"][:, 1].max())
        b["center"] = (b["center"][0], top - 0.02 + b["half"][1], b["center"][2])
    pert = [perturbed(sc, seed=100 + s, f_amp=0.02, c_amp=2.0) for s, sc in enumerate(scenes)]
    with mpm.from_scenes(scenes) as sim:
        for s, p in enumerate(pert):
            sim.write_state(s, v=p[0], C=p[1], F=p[2])
        for s in range(len(scenes)):
            sim.impulse(s)
        sim.substep(1e-4, 1)
        got = [sim.read_state(s, ("x", "v", "C", "F", "impulse")) for s in range(len(scenes))]
    touched = 0
    for s, sc in enumerate(scenes):
        st = oracle_state(sc, sc["x"], *pert[s])
        rig, nr = oracle_rigids(sc)
        assert oracle.substep(oracle_cfg(sc), st, 1e-4, rig, nr)[2] == 0
        err = Scales(sc, pert[s][2], 1e-4)
        for f in ("x", "F"):
            assert_close(f"scene {s} {f}", got[s][f], getattr(st, f))
        assert_close(f"scene {s} v", got[s]["v"], st.v, atol_floor=err.atol_v(st.v))
        assert_close(f"scene {s} C", got[s]["C"], st.C, atol_floor=err.atol_C(st.v))
        imp = oracle.rigid_impulse(rig[0])
        assert_close(f"scene {s} impulse", got[s]["impulse"][0], imp, rtol=1e-4, rel_scale=1e-4)
        touched += np.abs(imp[:3]).max() > 0
    assert touched == len(scenes)
