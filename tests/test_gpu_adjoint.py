"""Gradients of a trajectory loss from the hand-written adjoint kernels (through
the C ABI and the torch.autograd.Function) against central finite differences
of the FP64 oracle, h = 1e-6 (relative for E, absolute for nu and v0)."""
import numpy as np
import pytest

import oracle
from paper_2502_18437_gb300 import mpm, workloads as W

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

H = 1e-6
TOL = 1e-3


def oracle_loss(sc, E, nu, v0, steps):
    mu, lam = oracle.lame_arrays(E, nu)
    st = oracle.State(sc["x"], v0, mu=mu, lam=lam)
    assert oracle.run(oracle.config_from_workload(sc), st, sc["dt"], steps) == 0
    return oracle.loss(st.x, st.v, sc["target"])


def gpu_grads(sc, steps, checkpoint_every):
    from paper_2502_18437_gb300.autograd import trajectory

    dev = "cuda"
    E = torch.tensor(sc["E"], device=dev, requires_grad=True)
    nu = torch.tensor(sc["nu"], device=dev, requires_grad=True)
    v0 = torch.tensor(sc["v"], device=dev, requires_grad=True)
    x0 = torch.tensor(sc["x"], device=dev)
    x, v = trajectory(E, nu, v0, x0, n=sc["n"], substeps=steps, dt=sc["dt"], rho=sc["rho"], V0=sc["V0"],
                      model=sc["model"], checkpoint_every=checkpoint_every)
    target = torch.tensor(sc["target"], device=dev, dtype=torch.float32)
    N = x.shape[0]
    L = ((x.mean(0) - target) ** 2).sum() + (v * v).sum() / N
    L.backward()
    return float(L), E.grad.cpu().numpy().astype(np.float64), nu.grad.cpu().numpy().astype(np.float64), \
        v0.grad.cpu().numpy().astype(np.float64)


def fd_direction(sc, steps, kind, u):
    E, nu, v0 = sc["E"].astype(np.float64), sc["nu"].astype(np.float64), sc["v"].astype(np.float64)
    args = {"E": E, "nu": nu, "v0": v0}
    plus, minus = dict(args), dict(args)
    if kind == "E":
        plus["E"], minus["E"] = E * (1 + H * u), E * (1 - H * u)
    else:
        plus[kind], minus[kind] = args[kind] + H * u, args[kind] - H * u
    return (oracle_loss(sc, plus["E"], plus["nu"], plus["v0"], steps) -
            oracle_loss(sc, minus["E"], minus["nu"], minus["v0"], steps)) / (2 * H)


def check(sc, steps, checkpoint_every, n_dirs, seed, coords=True):
    L, gE, gnu, gv0 = gpu_grads(sc, steps, checkpoint_every)
    Lo = oracle_loss(sc, sc["E"].astype(np.float64), sc["nu"].astype(np.float64), sc["v"].astype(np.float64), steps)
    assert abs(L - Lo) <= 1e-5 * abs(Lo)
    g = np.random.default_rng(seed)
    N = len(sc["x"])
    for _ in range(n_dirs):
        for kind, grad in (("E", gE * sc["E"]), ("nu", gnu), ("v0", gv0)):
            u = g.normal(size=grad.shape)
            fd = fd_direction(sc, steps, kind, u)
            got = float(np.sum(grad * u))
            assert abs(got - fd) <= TOL * abs(fd), (kind, got, fd)
    # single initial-velocity coordinates
    for i in (g.integers(0, N, 2) if coords else ()):
        for d in range(3):
            u = np.zeros((N, 3))
            u[i, d] = 1.0
            fd = fd_direction(sc, steps, "v0", u)
            assert abs(gv0[i, d] - fd) <= TOL * abs(fd) + 1e-6 * np.abs(gv0).max(), (i, d, gv0[i, d], fd)


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
def test_adjoint_small_cube(model):
    # 1,728 particles, 40 substeps, a checkpoint every 7 (ragged last segment).
    sc = W.diff_cube(n=32, n_side=12, substeps=40, model=model)
    check(sc, 40, 7, n_dirs=2, seed=1)


def test_adjoint_differentiable_workload():
    # The differentiable workload at full size: 32,768 particles on 64^3,
    # 200 substeps, a checkpoint every 20.
    sc = W.diff_cube()
    check(sc, sc["substeps"], 20, n_dirs=1, seed=2, coords=False)


def test_adjoint_checkpoint_interval_invariance():
    # Recomputing from one checkpoint or keeping every state gives the same
    # gradients up to the order of floating-point atomics in the recompute.
    sc = W.diff_cube(n=32, n_side=10, substeps=30)
    a = gpu_grads(sc, 30, 1)
    b = gpu_grads(sc, 30, 30)
    for x, y in zip(a[1:], b[1:]):
        assert np.max(np.abs(x - y)) <= TOL * np.max(np.abs(y))


def test_adjoint_refuses_what_it_does_not_differentiate():
    sc = W.diff_cube(n=32, n_side=6, substeps=5)
    with mpm.Simulation(32, len(sc["x"]), tape_checkpoint_every=2, tape_max_substeps=5, plasticity=True,
                        yield_stress=50.0) as sim:
        sim.add_particles(0, sc["x"], sc["v"], sc["E"], sc["nu"], rho=sc["rho"], V0=sc["V0"])
        with pytest.raises(mpm.MPMError):
            sim.tape_begin()
    with mpm.Simulation(32, len(sc["x"]), tape_checkpoint_every=2, tape_max_substeps=5) as sim:
        sim.add_particles(0, sc["x"], sc["v"], sc["E"], sc["nu"], rho=sc["rho"], V0=sc["V0"])
        sim.set_rigid(0, 0, W.sphere((0.1, 0.9, 0.1), 0.01))
        sim.tape_begin()
        sim.substep(sc["dt"], 2)
        with pytest.raises(mpm.MPMError):
            sim.backward(np.zeros((len(sc["x"]), 3), np.float32))


# Step of the single-coordinate differences.  Perturbing one particle changes
# the 200-substep loss (~0.14) by only ~1e-8 h, while two FP64 runs whose
# inputs differ round differently by ~1e-14 in the loss: at h = 1e-6 that
# rounding is ~1 % of the difference (measured on the largest E coordinate:
# -1.5737e-8 at h = 1e-6, -1.5593e-8 at 1e-5, -1.5589e-8 at 1e-4, -1.5572e-8 at
# 1e-3, against -1.5571e-8 from the adjoint).  h = 1e-3 of each coordinate's
# own size keeps that rounding near 1e-4 and the O(h^2) truncation near 1e-6.
H_COORD = 1e-3


def test_adjoint_full_size_single_coordinates():
    # The differentiable workload at full size (32,768 particles, 64^3, 200
    # substeps, a checkpoint every 20): single coordinates of E, nu and the
    # three components of v0 on a seeded sample of particles plus the particle
    # of largest |E dL/dE|, each against its own FP64 central difference (the
    # oracle runs in spawned worker processes).
    from tests.oracle_pool import diff_cube_loss, map_tasks

    sc = W.diff_cube()
    steps = sc["substeps"]
    L, gE, gnu, gv0 = gpu_grads(sc, steps, 20)
    N = len(sc["x"])
    g = np.random.default_rng(11)
    idx = [int(i) for i in g.choice(N, 3, replace=False)] + [int(np.argmax(np.abs(gE * sc["E"])))]
    coords = [("E", 0), ("nu", 0), ("v0", 0), ("v0", 1), ("v0", 2)]

    def step(k, i, d):  # E: relative; nu, v0: absolute, scaled by the coordinate
        if k == "E":
            return H_COORD
        if k == "nu":
            return H_COORD * float(sc["nu"][i])
        return H_COORD * max(abs(float(sc["v"][i, d])), 0.1)

    tasks = [({}, steps, [(k, i, d, s * step(k, i, d))]) for i in idx for k, d in coords for s in (1, -1)]
    losses = np.array(map_tasks(diff_cube_loss, tasks)).reshape(len(idx), len(coords), 2)
    scale = {"E": np.abs(gE * sc["E"]).max(), "nu": np.abs(gnu).max(), "v0": np.abs(gv0).max()}
    for a, i in enumerate(idx):
        for b, (k, d) in enumerate(coords):
            fd = (losses[a, b, 0] - losses[a, b, 1]) / (2 * step(k, i, d))
            got = {"E": gE[i] * sc["E"][i], "nu": gnu[i], "v0": gv0[i, d]}[k]
            print(f"particle {i} {k}[{d}]: adjoint {got:.6e} fd {fd:.6e}")
            assert abs(got - fd) <= TOL * abs(fd) + 1e-6 * scale[k], (i, k, d, got, fd)


# ---------------------------------------------- dot-product tests per block
#
# For the substep map s_0 -> s_T (s = x, v, C, F per particle; mu, lambda as
# parameters) the adjoint must satisfy <J u, w> = <u, J^T w> for every input
# direction u and output weight w.  J u comes from FP64 central differences of
# the oracle, J^T w from the hand-written adjoint kernels (mpm_backward_state).
# Taking u and w inside one block each checks one path through the reverse
# kernels, e.g. (F -> v): the stress VJP of P2G^-1 (polar derivative for
# fixed-corotated), the grid^-1 normalisation and G2P^-1's gather; (C -> C):
# P2G^-1's affine term and G2P^-1's B-matrix; (x -> x): the weight-gradient
# terms of both transfers; (mu, lambda -> *): the material VJP.

IN_BLOCKS = ("x", "v", "C", "F", "mu", "lam")
OUT_BLOCKS = ("x", "v", "C", "F")


def _perturbed_state(sc, seed):
    g = np.random.default_rng(seed)
    N = len(sc["x"])
    v = (sc["v"] + 0.05 * g.normal(size=(N, 3))).astype(np.float32)
    C = (0.5 * g.normal(size=(N, 3, 3))).astype(np.float32)
    F = (np.eye(3) + 0.02 * g.normal(size=(N, 3, 3))).astype(np.float32)
    return v, C, F


def _oracle_out(sc, x, v, C, F, mu, lam, steps):
    st = oracle.State(x, v, C, F, mu=mu, lam=lam)
    assert oracle.run(oracle.config_from_workload(sc), st, sc["dt"], steps) == 0
    return {"x": st.x, "v": st.v, "C": st.C, "F": st.F}


@pytest.mark.parametrize("model,steps", [("fixed_corotated", 1), ("neo_hookean", 1), ("fixed_corotated", 6)])
def test_adjoint_dot_product_per_block(model, steps):
    sc = W.diff_cube(n=32, n_side=10, substeps=steps, model=model)
    N = len(sc["x"])
    v, C, F = _perturbed_state(sc, 5)
    x = sc["x"]
    mu, lam = oracle.lame_arrays(sc["E"], sc["nu"])
    g = np.random.default_rng(6)
    base = {"x": x.astype(np.float64), "v": v.astype(np.float64), "C": C.astype(np.float64),
            "F": F.astype(np.float64), "mu": mu, "lam": lam}
    # GPU: J^T w for one weight per output block
    with mpm.Simulation(32, N, model=model, tape_checkpoint_every=max(1, steps // 2),
                        tape_max_substeps=steps) as sim:
        sim.add_particles(0, x, sc["v"], sc["E"], sc["nu"], rho=sc["rho"], V0=sc["V0"])
        sim.write_state(0, v=v, C=C, F=F)
        sim.tape_begin()
        sim.substep(sc["dt"], steps)
        ws = {b: g.normal(size=base[b].shape) for b in OUT_BLOCKS}
        jt = {b: sim.backward_state({b: ws[b]}) for b in OUT_BLOCKS}
    # oracle: J u by central differences, one direction per input block (the
    # Lame parameters with a relative step of 1e-3: the x block of their
    # response is ~dt times smaller than the FP64 rounding of x / 1e-6)
    steps_h = {"x": 1e-6, "v": 1e-6, "C": 1e-5, "F": 1e-6, "mu": 1e-3, "lam": 1e-3}
    worst = 0.0
    for a in IN_BLOCKS:
        u = g.normal(size=base[a].shape)
        h = steps_h.get(a, 1e-6)
        args_p, args_m = dict(base), dict(base)
        if a in ("mu", "lam"):
            args_p[a], args_m[a] = base[a] * (1 + h * u), base[a] * (1 - h * u)
            u = u * base[a]  # the direction in mu / lambda itself
        else:
            args_p[a], args_m[a] = base[a] + h * u, base[a] - h * u
        op = _oracle_out(sc, args_p["x"], args_p["v"], args_p["C"], args_p["F"], args_p["mu"], args_p["lam"], steps)
        om = _oracle_out(sc, args_m["x"], args_m["v"], args_m["C"], args_m["F"], args_m["mu"], args_m["lam"], steps)
        ju = {b: (op[b] - om[b]) / (2 * h) for b in OUT_BLOCKS}
        for b in OUT_BLOCKS:
            fd = float(np.sum(ju[b] * ws[b]))
            got = float(np.sum(u * jt[b][a].astype(np.float64)))
            # the floor: FP32 rounding of the adjoint relative to the block's size
            floor = 1e-5 * float(np.linalg.norm(ju[b]) * np.linalg.norm(ws[b]))
            print(f"{model} T={steps} {a}->{b}: adjoint {got:.6e} fd {fd:.6e}")
            assert abs(got - fd) <= TOL * abs(fd) + floor, (a, b, got, fd)
            worst = max(worst, abs(got - fd) / max(abs(fd), 1e-300))
    print(f"worst relative difference {worst:.2e}")
