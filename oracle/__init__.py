"""FP64 CPU oracle of the MLS-MPM substep (arXiv 2502.18437, Algorithm 1).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``; the library in
``paper_2502_18437_gb300`` never imports it.  The arithmetic lives in
``mpm_oracle.c`` (plain C, double precision, serial); this module only marshals
numpy arrays through ctypes.

State layout used here: ``x, v`` (N,3); ``C, F`` (N,3,3) row-major; ``mu, lam``
(N,) Lame parameters per particle.  Rigid bodies are described by plain dicts
(see ``paper_2502_18437_gb300.workloads``), converted here into the oracle's own
struct.

Parity status: every function is pinned by ``tests/test_oracle_pins.py`` against
closed forms, invariants, brute force or LAPACK, except the full multi-substep
trajectory, which has no published value (the paper's only performance figure is
absent from its text): "parity unpinned" beyond the invariants the whole step
must satisfy (momentum and angular-momentum conservation, free fall, affine and
rigid-rotation reproduction).
"""
import ctypes as ct
import os

import numpy as np

from . import build as _build

MAX_PTS = 64
MAX_TRIS = 64
MAX_SPINE = 16
ERR_OUT_OF_DOMAIN, ERR_NONFINITE, ERR_INVERTED = 1, 2, 4
MODELS = {"fixed_corotated": 0, "neo_hookean": 1}
RIGID_TYPES = {"sphere": 0, "box": 1, "quad_slicer": 2, "segments": 3, "arc": 4, "mesh_slicer": 5}
REGION = {0: "none", 1: "regular", 2: "oned", 3: "sticky"}


class Config(ct.Structure):
    _fields_ = [
        ("n", ct.c_int), ("bound", ct.c_int), ("floor_sticky", ct.c_int), ("model", ct.c_int),
        ("plasticity", ct.c_int), ("pad_", ct.c_int), ("yield_stress", ct.c_double),
        ("gravity", ct.c_double * 3), ("m_p", ct.c_double), ("V0", ct.c_double),
    ]


class Rigid(ct.Structure):
    _fields_ = [
        ("type", ct.c_int), ("n_pts", ct.c_int), ("c", ct.c_double * 3), ("R", ct.c_double * 9),
        ("vel", ct.c_double * 3), ("omega", ct.c_double * 3), ("mu_k", ct.c_double),
        ("c_d", ct.c_double), ("margin", ct.c_double), ("radius", ct.c_double),
        ("half", ct.c_double * 3), ("thickness", ct.c_double), ("spine_radius", ct.c_double),
        ("pts", ct.c_double * (MAX_PTS * 3)), ("impulse", ct.c_double * 6),
        ("n_tris", ct.c_int), ("n_spine", ct.c_int), ("tris", ct.c_int * (MAX_TRIS * 3)),
        ("spine", ct.c_int * MAX_SPINE),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ct.CDLL(path)
        D = ct.POINTER(ct.c_double)
        I = ct.POINTER(ct.c_int)
        F32 = ct.POINTER(ct.c_float)
        L.orc_bspline_N.restype = ct.c_double
        L.orc_bspline_N.argtypes = [ct.c_double]
        L.orc_bspline_weights.argtypes = [ct.c_double, D]
        L.orc_svd3.argtypes = [D, D, D, D]
        L.orc_polar_R.argtypes = [D, D]
        L.orc_kirchhoff.restype = ct.c_int
        L.orc_kirchhoff.argtypes = [ct.c_int, D, ct.c_double, ct.c_double, D]
        L.orc_lame.argtypes = [ct.c_double, ct.c_double, D, D]
        L.orc_kirchhoff_all.restype = ct.c_int
        L.orc_kirchhoff_all.argtypes = [ct.c_int, ct.c_int, D, D, D, D]
        L.orc_von_mises.restype = ct.c_int
        L.orc_von_mises.argtypes = [D, ct.c_double, ct.c_double]
        L.orc_rigid_set_quat.argtypes = [ct.POINTER(Rigid), D]
        L.orc_rigid_advance.argtypes = [ct.POINTER(Rigid), ct.c_double]
        L.orc_geometry.restype = ct.c_int
        L.orc_geometry.argtypes = [ct.POINTER(Rigid), D, D, D, D]
        L.orc_contact_node.argtypes = [ct.POINTER(Rigid), D, ct.c_double, D]
        L.orc_push_out.restype = ct.c_int
        L.orc_push_out.argtypes = [ct.POINTER(Rigid), D]
        L.orc_p2g.restype = ct.c_int
        L.orc_p2g.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D, D, D, ct.c_double, D, D]
        L.orc_grid_update.restype = ct.c_int
        L.orc_grid_update.argtypes = [ct.POINTER(Config), D, D, ct.c_int, ct.POINTER(Rigid), ct.c_double]
        L.orc_g2p.restype = ct.c_int
        L.orc_g2p.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D, D, ct.c_double, D]
        L.orc_substep.restype = ct.c_int
        L.orc_substep.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D, D, D, ct.c_int,
                                  ct.POINTER(Rigid), ct.c_double, D]
        L.orc_run.restype = ct.c_int
        L.orc_run.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D, D, D, ct.c_int,
                              ct.POINTER(Rigid), ct.c_double, ct.c_int]
        L.orc_bspline_dN.restype = ct.c_double
        L.orc_bspline_dN.argtypes = [ct.c_double]
        L.orc_p2g_standard.restype = ct.c_int
        L.orc_p2g_standard.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D, D, ct.c_double, D, D]
        L.orc_g2p_standard.restype = ct.c_int
        L.orc_g2p_standard.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D, D, ct.c_double, D]
        L.orc_pb_constraint.argtypes = [D, D, ct.c_double, ct.c_double, D]
        L.orc_p2g_apic.restype = ct.c_int
        L.orc_p2g_apic.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D, D]
        L.orc_g2p_vc.restype = ct.c_int
        L.orc_g2p_vc.argtypes = [ct.POINTER(Config), ct.c_int, D, D, D, D]
        L.orc_run_solver.restype = ct.c_int
        L.orc_run_solver.argtypes = [ct.POINTER(Config), ct.c_int, ct.c_int, D, D, D, D, D, D, ct.c_int,
                                     ct.POINTER(Rigid), ct.c_double, ct.c_int, ct.c_int, ct.c_double]
        L.orc_sort_by_brick.argtypes = [ct.c_int, ct.c_int, F32, I, I, I]
        L.orc_loss.restype = ct.c_double
        L.orc_loss.argtypes = [ct.c_int, D, D, D]
        _lib = L
    return _lib


def _dp(a):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(ct.POINTER(ct.c_double))


def _arr(a, shape=None):
    out = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        out = out.reshape(shape)
    return out


# ------------------------------------------------------------------ config

def make_config(n, m_p, V0, *, bound=3, floor_sticky=True, model="fixed_corotated",
                plasticity=False, yield_stress=0.0, gravity=(0.0, -9.8, 0.0)):
    c = Config()
    c.n, c.bound, c.floor_sticky = int(n), int(bound), int(bool(floor_sticky))
    c.model = MODELS[model] if isinstance(model, str) else int(model)
    c.plasticity, c.yield_stress = int(bool(plasticity)), float(yield_stress)
    for i in range(3):
        c.gravity[i] = float(gravity[i])
    c.m_p, c.V0 = float(m_p), float(V0)
    return c


def make_rigid(desc):
    """Oracle rigid struct from a plain description dict."""
    r = Rigid()
    r.type = RIGID_TYPES[desc["type"]]
    for i in range(3):
        r.c[i] = float(desc["center"][i])
        r.vel[i] = float(desc.get("vel", (0, 0, 0))[i])
        r.omega[i] = float(desc.get("omega", (0, 0, 0))[i])
        r.half[i] = float(desc.get("half", (0, 0, 0))[i])
    q = _arr(desc.get("quat", (1.0, 0.0, 0.0, 0.0)))
    lib().orc_rigid_set_quat(ct.byref(r), _dp(q))
    r.mu_k = float(desc.get("mu_k", 0.0))
    r.c_d = float(desc.get("c_d", 1.0))
    r.margin = float(desc.get("margin", 0.0))
    r.radius = float(desc.get("radius", 0.0))
    r.thickness = float(desc.get("thickness", 0.0))
    r.spine_radius = float(desc.get("spine_radius", 0.5 * r.thickness))
    pts = np.asarray(desc.get("pts", np.zeros((0, 3))), dtype=np.float64).reshape(-1, 3)
    assert len(pts) <= MAX_PTS
    r.n_pts = len(pts)
    for i, v in enumerate(pts.reshape(-1)):
        r.pts[i] = float(v)
    tris = np.asarray(desc.get("tris", np.zeros((0, 3))), dtype=np.int64).reshape(-1, 3)
    spine = np.asarray(desc.get("spine", []), dtype=np.int64).reshape(-1)
    assert len(tris) <= MAX_TRIS and len(spine) <= MAX_SPINE
    r.n_tris, r.n_spine = len(tris), len(spine)
    for i, v in enumerate(tris.reshape(-1)):
        r.tris[i] = int(v)
    for i, v in enumerate(spine):
        r.spine[i] = int(v)
    return r


def rigid_array(descs):
    arr = (Rigid * max(1, len(descs)))()
    for i, d in enumerate(descs):
        arr[i] = make_rigid(d)
    return arr


def rigid_pose(r):
    return np.array(r.c[:]), np.array(r.R[:]).reshape(3, 3)


def rigid_impulse(r):
    return np.array(r.impulse[:])


# --------------------------------------------------------------- functions

def bspline_N(r):
    return lib().orc_bspline_N(float(r))


def bspline_weights(f):
    w = np.zeros(3)
    lib().orc_bspline_weights(float(f), _dp(w))
    return w


def svd3(A):
    A = _arr(A, (3, 3))
    U, S, V = np.zeros((3, 3)), np.zeros(3), np.zeros((3, 3))
    lib().orc_svd3(_dp(A), _dp(U), _dp(S), _dp(V))
    return U, S, V


def polar_R(A):
    A = _arr(A, (3, 3))
    R = np.zeros((3, 3))
    lib().orc_polar_R(_dp(A), _dp(R))
    return R


def kirchhoff(model, F, mu, lam):
    F = _arr(F, (3, 3))
    tau = np.zeros((3, 3))
    m = MODELS[model] if isinstance(model, str) else int(model)
    err = lib().orc_kirchhoff(m, _dp(F), float(mu), float(lam), _dp(tau))
    return tau, err


def kirchhoff_all(model, F, mu, lam):
    """Kirchhoff stress of every particle: F (N,3,3) -> tau (N,3,3), error bits."""
    F = _arr(F).reshape(-1, 3, 3)
    N = len(F)
    mu = np.broadcast_to(_arr(mu), (N,)).copy()
    lam = np.broadcast_to(_arr(lam), (N,)).copy()
    tau = np.zeros((N, 3, 3))
    m = MODELS[model] if isinstance(model, str) else int(model)
    err = lib().orc_kirchhoff_all(m, N, _dp(np.ascontiguousarray(F)), _dp(mu), _dp(lam), _dp(tau))
    return tau, err


def lame(E, nu):
    mu, lam = ct.c_double(), ct.c_double()
    lib().orc_lame(float(E), float(nu), ct.byref(mu), ct.byref(lam))
    return mu.value, lam.value


def von_mises(F, mu, yield_stress):
    F = _arr(F, (3, 3)).copy()
    err = lib().orc_von_mises(_dp(F), float(mu), float(yield_stress))
    return F, err


def geometry(rigid, x):
    x = _arr(x, (3,))
    n, t, d = np.zeros(3), np.zeros(3), ct.c_double()
    code = lib().orc_geometry(ct.byref(rigid), _dp(x), _dp(n), _dp(t), ct.byref(d))
    return REGION[code], n, t, d.value


def contact_node(rigid, x, m, v):
    x = _arr(x, (3,))
    v = _arr(v, (3,)).copy()
    lib().orc_contact_node(ct.byref(rigid), _dp(x), float(m), _dp(v))
    return v


def push_out(rigid, x):
    """(x after the push-out against one rigid, whether it moved)."""
    x = _arr(x, (3,)).copy()
    moved = lib().orc_push_out(ct.byref(rigid), _dp(x))
    return x, bool(moved)


def rigid_advance(rigid, dt):
    lib().orc_rigid_advance(ct.byref(rigid), float(dt))


class State:
    """Particle state in FP64: x, v (N,3); C, F (N,3,3); mu, lam (N,)."""

    def __init__(self, x, v=None, C=None, F=None, mu=None, lam=None):
        x = _arr(x).reshape(-1, 3)
        N = len(x)
        self.x = x.copy()
        self.v = np.zeros((N, 3)) if v is None else _arr(v, (N, 3)).copy()
        self.C = np.zeros((N, 3, 3)) if C is None else _arr(C, (N, 3, 3)).copy()
        self.F = np.tile(np.eye(3), (N, 1, 1)) if F is None else _arr(F, (N, 3, 3)).copy()
        self.mu = np.zeros(N) if mu is None else np.broadcast_to(_arr(mu), (N,)).copy()
        self.lam = np.zeros(N) if lam is None else np.broadcast_to(_arr(lam), (N,)).copy()

    @property
    def N(self):
        return len(self.x)

    def copy(self):
        return State(self.x, self.v, self.C, self.F, self.mu, self.lam)

    def ptrs(self):
        return [_dp(a) for a in (self.x, self.v, self.C, self.F, self.mu, self.lam)]


def p2g(cfg, st, dt):
    nn = cfg.n ** 3
    gm, gmv = np.zeros(nn), np.zeros((nn, 3))
    x, v, C, F, mu, lam = st.ptrs()
    err = lib().orc_p2g(ct.byref(cfg), st.N, x, v, C, F, mu, lam, float(dt), _dp(gm), _dp(gmv))
    return gm, gmv, err


def grid_update(cfg, gm, gmv, dt, rigids=None, n_rigid=0):
    """Node loop; gmv momentum (n^3,3) in, velocity out.  Rigids advance not."""
    gmv = _arr(gmv).copy()
    gm = _arr(gm)
    if rigids is None:
        rigids, n_rigid = (Rigid * 1)(), 0
    err = lib().orc_grid_update(ct.byref(cfg), _dp(gm), _dp(gmv), int(n_rigid), rigids, float(dt))
    return gmv, err


def g2p(cfg, st, gv, dt):
    gv = _arr(gv)
    x, v, C, F, mu, lam = st.ptrs()
    return lib().orc_g2p(ct.byref(cfg), st.N, x, v, C, F, mu, float(dt), _dp(gv))


def substep(cfg, st, dt, rigids=None, n_rigid=0):
    """One substep in place; returns (grid_m (n^3,), grid_v (n^3,3), err)."""
    nn = cfg.n ** 3
    grid = np.zeros(4 * nn)
    if rigids is None:
        rigids, n_rigid = (Rigid * 1)(), 0
    x, v, C, F, mu, lam = st.ptrs()
    err = lib().orc_substep(ct.byref(cfg), st.N, x, v, C, F, mu, lam, int(n_rigid), rigids,
                            float(dt), _dp(grid))
    return grid[:nn].copy(), grid[nn:].reshape(nn, 3).copy(), err


def run(cfg, st, dt, n_steps, rigids=None, n_rigid=0):
    """n_steps substeps in place; returns the error bits."""
    if rigids is None:
        rigids, n_rigid = (Rigid * 1)(), 0
    x, v, C, F, mu, lam = st.ptrs()
    return lib().orc_run(ct.byref(cfg), st.N, x, v, C, F, mu, lam, int(n_rigid), rigids,
                         float(dt), int(n_steps))


SOLVERS = {"mls": 0, "standard": 1, "pb": 2}


def bspline_dN(r):
    return lib().orc_bspline_dN(float(r))


def p2g_standard(cfg, st, dt):
    nn = cfg.n ** 3
    gm, gmv = np.zeros(nn), np.zeros((nn, 3))
    x, v, C, F, mu, lam = st.ptrs()
    err = lib().orc_p2g_standard(ct.byref(cfg), st.N, x, v, F, mu, lam, float(dt), _dp(gm), _dp(gmv))
    return gm, gmv, err


def g2p_standard(cfg, st, gv, dt):
    gv = _arr(gv)
    x, v, C, F, mu, lam = st.ptrs()
    return lib().orc_g2p_standard(ct.byref(cfg), st.N, x, v, C, F, mu, float(dt), _dp(gv))


def pb_constraint(C, F, dt, beta):
    C, F = _arr(C, (3, 3)), _arr(F, (3, 3))
    out = np.zeros((3, 3))
    lib().orc_pb_constraint(_dp(C), _dp(F), float(dt), float(beta), _dp(out))
    return out


def run_solver(cfg, st, dt, n_steps, solver="mls", rigids=None, n_rigid=0, iters=1, beta=1.0):
    """n_steps steps of a solver ("mls", "standard", "pb") in place; returns the error bits."""
    if rigids is None:
        rigids, n_rigid = (Rigid * 1)(), 0
    x, v, C, F, mu, lam = st.ptrs()
    return lib().orc_run_solver(ct.byref(cfg), SOLVERS[solver], st.N, x, v, C, F, mu, lam, int(n_rigid), rigids,
                                float(dt), int(n_steps), int(iters), float(beta))


def sort_by_brick(n, x32):
    x32 = np.ascontiguousarray(np.asarray(x32, dtype=np.float32).reshape(-1, 3))
    N = len(x32)
    nb = n // 4
    key = np.zeros(N, dtype=np.int32)
    perm = np.zeros(N, dtype=np.int32)
    count = np.zeros(nb ** 3, dtype=np.int32)
    ip = lambda a: a.ctypes.data_as(ct.POINTER(ct.c_int))
    lib().orc_sort_by_brick(int(n), N, x32.ctypes.data_as(ct.POINTER(ct.c_float)), ip(key), ip(perm),
                            ip(count))
    return key, perm, count


def loss(x, v, target):
    x, v, t = _arr(x).reshape(-1, 3), _arr(v).reshape(-1, 3), _arr(target, (3,))
    return lib().orc_loss(len(x), _dp(x), _dp(v), _dp(t))


# ------------------------------------------------- workload marshalling

def lame_arrays(E, nu):
    """Lame parameters of per-particle (E, nu), the textbook formula of orc_lame."""
    E = np.asarray(E, dtype=np.float64)
    nu = np.asarray(nu, dtype=np.float64)
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def config_from_workload(sc):
    """Oracle config of a workload dict (mass = rho * V0 rounded as in FP32 inputs)."""
    m_p = float(np.float32(sc["rho"]) * np.float32(sc["V0"]))
    return make_config(sc["n"], m_p, sc["V0"], bound=sc["bound"], floor_sticky=sc["floor_sticky"],
                       model=sc["model"], plasticity=sc["plasticity"], yield_stress=sc["yield_stress"],
                       gravity=sc["gravity"])


def state_from_workload(sc, x=None, v=None, C=None, F=None):
    mu, lam = lame_arrays(sc["E"], sc["nu"])
    return State(sc["x"] if x is None else x, sc["v"] if v is None else v, C, F, mu, lam)
