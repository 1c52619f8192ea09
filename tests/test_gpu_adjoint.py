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
