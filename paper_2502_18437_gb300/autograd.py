"""Differentiable trajectories: a torch.autograd.Function over the C ABI.

Forward records a tape (``mpm_tape_begin`` + ``mpm_substep``) and returns the
final positions and velocities; backward calls ``mpm_backward``, i.e. the
hand-written adjoint kernels of G2P, grid update and P2G (including the
polar-decomposition derivative), with checkpoint/recompute, and returns the
gradients with respect to the per-particle Young's modulus, Poisson ratio and
initial velocity.  All tensors live on the GPU; nothing is computed in PyTorch.
"""
import torch

from . import mpm


class MPMTrajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, E, nu, v0, x0, opts):
        N = x0.shape[0]
        sim = mpm.Simulation(opts["n"], N, model=opts.get("model", "fixed_corotated"),
                             gravity=opts.get("gravity", (0.0, -9.8, 0.0)), bound=opts.get("bound", 3),
                             floor_sticky=opts.get("floor_sticky", True),
                             tape_checkpoint_every=opts.get("checkpoint_every", 20),
                             tape_max_substeps=opts["substeps"], stream=torch.cuda.current_stream().cuda_stream)
        sim.add_particles(0, x0.detach().float().contiguous(), v0.detach().float().contiguous(),
                          E.detach().float().contiguous(), nu.detach().float().contiguous(),
                          rho=opts["rho"], V0=opts["V0"])
        sim.tape_begin()
        sim.substep(opts["dt"], opts["substeps"])
        st = sim.read_state(0, ("x", "v"), device=True)
        ctx.sim = sim
        return st["x"], st["v"]

    @staticmethod
    def backward(ctx, gx, gv):
        sim = ctx.sim
        dE, dnu, dv0 = sim.backward(gx.float().contiguous(), gv.float().contiguous(), device=True)
        sim.close()
        return dE, dnu, dv0, None, None


def trajectory(E, nu, v0, x0, **opts):
    """(x_T, v_T) after ``opts['substeps']`` substeps; differentiable in E, nu, v0."""
    return MPMTrajectory.apply(E, nu, v0, x0, opts)
