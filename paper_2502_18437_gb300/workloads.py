"""Seeded synthetic workloads shaped like the paper's scenes.

This module only draws inputs: particle positions, initial velocities, material
constants and rigid-body descriptions.  It holds none of the method's arithmetic,
so both the CUDA library and the FP64 oracle consume exactly the same FP32 input
values from it.

Every workload is a plain dict:
  n            grid nodes per dimension (dx = 1/n, domain [0,1)^3)
  x, v         float32 (N,3) positions and initial velocities
  E, nu        float32 (N,) Young's modulus and Poisson ratio per particle
  rho, V0      density and initial particle volume (mass = rho * V0)
  model        "fixed_corotated" | "neo_hookean"
  plasticity   bool (von Mises), yield_stress
  dt, substeps time step and number of substeps of the scene
  gravity      3-vector; bound boundary width in nodes; floor_sticky bool
  rigids       list of rigid descriptions (dicts), see ``quad_slicer`` etc.

The falling-cube shape follows the paper's timing scene (Sec. III-D: a cube
falling under gravity); the tissue slab, blade ("slicer", Sec. IV-B) and
capsule-chain thread ("connected line segments", Sec. IV-C) follow the cutting
and suturing scenes of Sec. VI.  The paper gives no tissue constants, sizes or
particle counts for those scenes, so the numbers below are proposed values.
"""
import math

import numpy as np

SEED_BASE = 2502_18437


def rng(tag: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(SEED_BASE + int(tag)))


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _scene(n, x, v, E, nu, *, rho, V0, model, dt, substeps, plasticity=False, yield_stress=0.0,
           rigids=(), gravity=(0.0, -9.8, 0.0), bound=3, floor_sticky=True, name=""):
    N = len(x)
    return dict(name=name, n=int(n), x=_f32(x).reshape(N, 3), v=_f32(v).reshape(N, 3),
                E=_f32(np.broadcast_to(E, (N,))), nu=_f32(np.broadcast_to(nu, (N,))),
                rho=float(rho), V0=float(np.float32(V0)), model=model, plasticity=bool(plasticity),
                yield_stress=float(yield_stress), dt=float(dt), substeps=int(substeps),
                gravity=tuple(float(g) for g in gravity), bound=int(bound),
                floor_sticky=bool(floor_sticky), rigids=list(rigids))


# ----------------------------------------------------------- rigid bodies

def quad_slicer(center, quat, *, half_edge, half_depth, thickness, vel=(0, 0, 0), omega=(0, 0, 0),
                mu_k=0.3, c_d=1.0, margin=0.0, spine_radius=None):
    """Blade: body x along the cutting edge, body y from the spine to the edge,
    body z the blade normal; half sizes half_edge (x) and half_depth (y)."""
    return dict(type="quad_slicer", center=tuple(center), quat=tuple(quat), vel=tuple(vel),
                omega=tuple(omega), mu_k=mu_k, c_d=c_d, margin=margin,
                half=(half_edge, half_depth, 0.0), thickness=thickness,
                spine_radius=0.5 * thickness if spine_radius is None else spine_radius)


def segments(center, quat, pts, *, radius, vel=(0, 0, 0), omega=(0, 0, 0), mu_k=0.3, c_d=1.0,
             margin=0.0):
    """Chain of connected capsules through ``pts`` (body frame)."""
    return dict(type="segments", center=tuple(center), quat=tuple(quat), pts=np.asarray(pts, float),
                radius=radius, vel=tuple(vel), omega=tuple(omega), mu_k=mu_k, c_d=c_d, margin=margin)


def arc(center, quat, *, arc_radius, start, sweep, radius, vel=(0, 0, 0), omega=(0, 0, 0), mu_k=0.3, c_d=1.0,
        margin=0.0):
    """Curved suture needle (Sec. IV-C): the circle of radius arc_radius about
    the body origin in the body x-y plane, from angle ``start`` over ``sweep``
    radians, with wire radius ``radius``."""
    return dict(type="arc", center=tuple(center), quat=tuple(quat), half=(arc_radius, start, sweep), radius=radius,
                vel=tuple(vel), omega=tuple(omega), mu_k=mu_k, c_d=c_d, margin=margin)


def mesh_slicer(center, quat, pts, tris, spine, *, thickness, spine_radius=None, vel=(0, 0, 0), omega=(0, 0, 0),
                mu_k=0.3, c_d=1.0, margin=0.0):
    """Blade given as an open triangle mesh (Sec. IV-B, TriangleMeshSlicer):
    vertices ``pts`` (body frame), triangles ``tris`` (vertex indices), the
    spine as a polyline of vertex indices ``spine``, blade thickness."""
    return dict(type="mesh_slicer", center=tuple(center), quat=tuple(quat), pts=np.asarray(pts, float),
                tris=np.asarray(tris, int), spine=np.asarray(spine, int), thickness=thickness,
                spine_radius=0.5 * thickness if spine_radius is None else spine_radius, vel=tuple(vel),
                omega=tuple(omega), mu_k=mu_k, c_d=c_d, margin=margin)


def curved_blade_mesh(half_edge=0.08, depth=0.06, bend=0.02, nu=8, nv=4, seed=6, jitter=0.1):
    """A seeded curved scalpel blade: a (nu+1) x (nv+1) vertex grid over body
    x in [-half_edge, half_edge] (along the edge) and body y in [-depth/2, depth/2]
    (spine at -depth/2, cutting edge at +depth/2), bent out of the x-y plane by
    z = bend (x / half_edge)^2 and jittered inside the grid; two triangles per
    cell.  Returns (pts, tris, spine)."""
    g = rng(seed)
    xs = np.linspace(-half_edge, half_edge, nu + 1)
    ys = np.linspace(-depth / 2, depth / 2, nv + 1)
    X, Y = np.meshgrid(xs, ys, indexing="ij")
    dxg, dyg = xs[1] - xs[0], ys[1] - ys[0]
    X = X + jitter * dxg * g.uniform(-1, 1, X.shape) * (np.abs(X) < half_edge - 1e-12)
    Y = Y + jitter * dyg * g.uniform(-1, 1, Y.shape) * (np.abs(Y) < depth / 2 - 1e-12)
    Z = bend * (X / half_edge) ** 2
    pts = np.stack([X, Y, Z], -1).reshape(-1, 3)
    idx = lambda i, j: i * (nv + 1) + j
    tris = []
    for i in range(nu):
        for j in range(nv):
            tris.append((idx(i, j), idx(i + 1, j), idx(i + 1, j + 1)))
            tris.append((idx(i, j), idx(i + 1, j + 1), idx(i, j + 1)))
    spine = [idx(i, 0) for i in range(nu + 1)]
    return pts, np.array(tris), np.array(spine)


def sphere(center, radius, *, vel=(0, 0, 0), omega=(0, 0, 0), mu_k=0.3, c_d=1.0, margin=0.0,
           quat=(1, 0, 0, 0)):
    return dict(type="sphere", center=tuple(center), quat=tuple(quat), radius=radius, vel=tuple(vel),
                omega=tuple(omega), mu_k=mu_k, c_d=c_d, margin=margin)


def box(center, half, *, quat=(1, 0, 0, 0), vel=(0, 0, 0), omega=(0, 0, 0), mu_k=0.3, c_d=1.0,
        margin=0.0):
    return dict(type="box", center=tuple(center), quat=tuple(quat), half=tuple(half), vel=tuple(vel),
                omega=tuple(omega), mu_k=mu_k, c_d=c_d, margin=margin)


# Blade orientation with the edge along world z, the edge pointing down (-y)
# and the blade normal along world x: a half turn about (1,0,1)/sqrt(2).
BLADE_EDGE_Z_DOWN = (0.0, math.sqrt(0.5), 0.0, math.sqrt(0.5))


def _yaw_blade_quat(yaw):
    """Blade edge down, rotated by ``yaw`` about world y."""
    qy = np.array([math.cos(yaw / 2), 0.0, math.sin(yaw / 2), 0.0])
    qb = np.array(BLADE_EDGE_Z_DOWN)
    w1, x1, y1, z1 = qy
    w2, x2, y2, z2 = qb
    return (w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
            w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2)


# -------------------------------------------------------------- workloads

def lattice_cube(n_side, spacing, corner):
    i = (np.arange(n_side) + 0.5) * spacing
    g = np.stack(np.meshgrid(i, i, i, indexing="ij"), -1).reshape(-1, 3)
    return g + np.asarray(corner, float)


def elastic_cube(n=32, n_side=16, corner=(0.375, 0.1, 0.375), substeps=100, v0=(0.0, 0.0, 0.0),
                 E=1e4, nu=0.3, rho=1.0, dt=1e-4, gravity=(0.0, -9.8, 0.0), model="fixed_corotated"):
    """Falling elastic cube: 16^3 lattice at spacing dx/2 (8 particles per cell)
    on a 32^3 grid, fixed-corotated E=1e4 nu=0.3 rho=1, dt=1e-4, sticky floor."""
    dx = 1.0 / n
    x = lattice_cube(n_side, dx / 2, corner)
    V0 = (dx / 2) ** 3
    v = np.broadcast_to(np.asarray(v0, float), x.shape)
    return _scene(n, x, v, E, nu, rho=rho, V0=V0, model=model, dt=dt, substeps=substeps,
                  gravity=gravity, name=f"elastic_cube_{len(x)}p_n{n}")


def tissue_slab(cells=(128, 16, 128), lo=(0.25, 0.03, 0.25), size=(0.5, 0.1, 0.5), n=128, seed=1,
                substeps=1000, with_tools=True, dt=1e-4):
    """Tissue slab for cutting/suturing: one uniform point per jitter cell in a
    0.5 x 0.1 x 0.5 box, Neo-Hookean, E ~ U[5e3, 2e4], nu = 0.4, rho = 1000,
    driven by a thin blade (0.002 thick, 0.1 m/s down) and a 32-capsule thread
    (radius 0.003) sliding along its own axis at 0.05 m/s."""
    g = rng(seed)
    cells = np.asarray(cells)
    N = int(np.prod(cells))
    idx = np.stack(np.meshgrid(*[np.arange(c) for c in cells], indexing="ij"), -1).reshape(-1, 3)
    h = np.asarray(size) / cells
    x = np.asarray(lo) + (idx + g.random((N, 3))) * h
    E = g.uniform(5e3, 2e4, N)
    V0 = float(np.prod(size)) / N
    dx = 1.0 / n
    rigids = []
    if with_tools:
        # centre line offset by a fraction of a cell so that no grid plane holds
        # the blade's mid-plane or the thread's axis (contact decisions there are
        # ties of the normal's sign)
        cx, cz = lo[0] + size[0] / 2 + 0.37 * dx, lo[2] + size[2] / 2 + 0.21 * dx
        top = lo[1] + size[1]
        half_edge, half_depth = 0.3 * size[2], 0.04
        edge_y = top - 0.01
        rigids.append(quad_slicer((cx, edge_y + half_depth, cz), BLADE_EDGE_Z_DOWN, half_edge=half_edge,
                                  half_depth=half_depth, thickness=0.002, vel=(0.0, -0.1, 0.0),
                                  mu_k=0.3, c_d=1.0, margin=dx))
        L = 0.8 * size[0]
        pts = np.stack([np.linspace(-L / 2, L / 2, 33), np.zeros(33), np.zeros(33)], -1)
        rigids.append(segments((cx, lo[1] + 0.5 * size[1] + 0.29 * dx, cz), (1, 0, 0, 0), pts, radius=0.003,
                               vel=(0.05, 0.0, 0.0), mu_k=0.3, c_d=1.0, margin=dx))
    return _scene(n, x, np.zeros((N, 3)), E, 0.4, rho=1000.0, V0=V0, model="neo_hookean", dt=dt,
                  substeps=substeps, rigids=rigids, name=f"tissue_slab_{N}p_n{n}")


# The paper's timing scene (Sec. III-D): a cube falling under gravity on a grid
# fixed at 175,616 nodes (56^3); one rendered step is 0.02 s = 10 substeps of
# dt = 0.002.  The paper states neither the particle counts, the cube's size nor
# its material, so those are proposed: a cube of side 0.4 centred in x and z
# with its bottom at y = ``bottom`` (0.54: it falls 13 steps, 0.26 s, before it
# nears the floor), N uniform random points, Neo-Hookean (the law the paper
# writes out, Eq. 6), E = 3e3, nu = 0.3, rho = 1000 (CFL dt c / dx = 0.22).
PAPER_TIMING_GRID = 56
PAPER_TIMING_DT = 0.002
PAPER_TIMING_SUBSTEPS_PER_STEP = 10
PAPER_TIMING_POINTS = (16384, 131072, 1048576)


def paper_timing_cube(N=131072, seed=5, steps=10, model="neo_hookean", bottom=0.54):
    """The falling cube of the paper's speed comparison on the fixed 56^3 grid,
    10 substeps of dt = 0.002 per 0.02 s step (``substeps`` = steps x 10)."""
    n = PAPER_TIMING_GRID
    side = 0.4
    g = rng(seed + 7 * (N % 1009))
    lo = np.array([0.5 - side / 2, bottom, 0.5 - side / 2])
    x = lo + g.random((N, 3)) * side
    return _scene(n, x, np.zeros((N, 3)), 3e3, 0.3, rho=1000.0, V0=side ** 3 / N, model=model,
                  dt=PAPER_TIMING_DT, substeps=steps * PAPER_TIMING_SUBSTEPS_PER_STEP,
                  name=f"paper_timing_cube_{N}p_n{n}")


SCALE_POINTS = {65536: 64, 262144: 128, 1048576: 256, 4194304: 256}


def tissue_block(N=1048576, n=None, seed=2, substeps=500, dt=5e-5, plasticity=True):
    """Scale-sweep block: N uniform points (8 per cell on average) in an
    axis-aligned cube of side (N/8)^(1/3) dx, centred in x and z with its bottom
    at y = 0.03 (or 4 dx on coarse grids, to start clear of the wall), falling at 2 m/s onto the sticky floor; fixed-corotated
    E = 1e4, nu = 0.3, rho = 1000, von Mises yield 50."""
    if n is None:
        n = SCALE_POINTS.get(N, 256)
    dx = 1.0 / n
    side = (N / 8.0) ** (1.0 / 3.0) * dx
    g = rng(seed + 1000 * (N % 997))
    lo = np.array([0.5 - side / 2, max(0.03, 4.0 * dx), 0.5 - side / 2])  # clear of the 3-node wall
    x = lo + g.random((N, 3)) * side
    V0 = side ** 3 / N
    v = np.broadcast_to(np.array([0.0, -2.0, 0.0]), (N, 3))
    return _scene(n, x, v, 1e4, 0.3, rho=1000.0, V0=V0, model="fixed_corotated", dt=dt,
                  substeps=substeps, plasticity=plasticity, yield_stress=50.0,
                  name=f"tissue_block_{N}p_n{n}")


def diff_cube(n=64, n_side=32, seed=3, substeps=200, model="fixed_corotated", dt=1e-4):
    """Differentiable workload: 32^3 lattice at 8 particles per cell on a 64^3
    grid (cube side 0.25, centred), rho = 1000, E ~ U[5e3, 2e4], nu ~ U[0.25, 0.4],
    v0 = a + B (x - c) + N(0, 0.01^2) with seeded a, B (|B| ~ 1/s); no rigids and
    no wall contact.  Also returns the loss target (centre + seeded offset)."""
    g = rng(seed)
    dx = 1.0 / n
    side = n_side * dx / 2
    c = np.array([0.5, 0.5, 0.5])
    x = lattice_cube(n_side, dx / 2, c - side / 2)
    N = len(x)
    E = g.uniform(5e3, 2e4, N)
    nu = g.uniform(0.25, 0.4, N)
    a = g.normal(0, 0.1, 3)
    B = g.normal(0, 1.0 / math.sqrt(3.0), (3, 3))
    v = a + (x - c) @ B.T + g.normal(0, 0.01, (N, 3))
    sc = _scene(n, x, v, E, nu, rho=1000.0, V0=(dx / 2) ** 3, model=model, dt=dt, substeps=substeps,
                name=f"diff_cube_{N}p_n{n}")
    sc["target"] = tuple(float(t) for t in (c + g.normal(0, 0.01, 3)))
    return sc


def batched_scenes(n_scenes=256, seed=4, lo_count=2048, hi_count=32768, substeps=1000, dt=1e-4):
    """Batched workload: scenes with particle counts log-uniform in [2k, 32k],
    grid 64^3 when the count exceeds 16k and otherwise a coin flip between
    32^3 and 64^3; a tissue block at 8 particles per cell resting above the
    sticky floor and one blade per scene with seeded yaw in [0, pi), position
    within 0.05 of the block centre and downward speed U[0.05, 0.2] m/s;
    fixed-corotated E = 1e4, nu = 0.3, rho = 1000, dt = 1e-4."""
    g = rng(seed)
    scenes = []
    for s in range(n_scenes):
        N = int(round(math.exp(g.uniform(math.log(lo_count), math.log(hi_count)))))
        n = 64 if N > 16384 else int(g.choice([32, 64]))
        dx = 1.0 / n
        side = (N / 8.0 / 0.5) ** (1.0 / 3.0) * dx  # block side x side/2 x side
        size = np.array([side, side / 2, side])
        lo = np.array([0.5 - side / 2, 4.0 * dx, 0.5 - side / 2])
        x = lo + g.random((N, 3)) * size
        yaw = g.uniform(0.0, math.pi)
        off = g.uniform(-0.05, 0.05, 2)
        speed = g.uniform(0.05, 0.2)
        top = lo[1] + size[1]
        half_depth = 0.05
        blade = quad_slicer((0.5 + off[0], top + 0.005 + half_depth, 0.5 + off[1]), _yaw_blade_quat(yaw),
                            half_edge=0.3 * side, half_depth=half_depth, thickness=0.002,
                            vel=(0.0, -speed, 0.0), mu_k=0.3, c_d=1.0, margin=dx)
        scenes.append(_scene(n, x, np.zeros((N, 3)), 1e4, 0.3, rho=1000.0, V0=float(np.prod(size)) / N,
                             model="fixed_corotated", dt=dt, substeps=substeps, rigids=[blade],
                             name=f"batched_{s}"))
    return scenes


def scaled_copy(sc, keep):
    """The first ``keep`` particles of a scene (a bounded sample of it)."""
    out = dict(sc)
    for k in ("x", "v", "E", "nu"):
        out[k] = np.ascontiguousarray(sc[k][:keep])
    out["name"] = sc["name"] + f"_sample{keep}"
    return out
