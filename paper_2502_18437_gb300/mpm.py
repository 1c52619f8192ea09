"""Thin Python binding of the C ABI in include/mpm.h (ctypes).

Functions named ``mpm_*`` mirror the C entry points one to one and only
marshal arguments; every step of the substep runs in the CUDA kernels of
libmpm_gb300.so.  ``Simulation`` wraps a context for convenience: it accepts
numpy arrays (host memory) or CUDA torch tensors (device memory, passed by
data_ptr) and returns numpy arrays or torch tensors.

There is no fallback: if the library has not been built, or no CUDA device is
present, every call raises.
"""
import ctypes as ct
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_lib", "libmpm_gb300.so")

MPM_OK = 0
STATUS = {
    -1: "INVALID_ARGUMENT", -2: "OUT_OF_MEMORY", -3: "CUDA", -4: "OUT_OF_DOMAIN", -5: "NONFINITE",
    -6: "INVERTED", -7: "CAPACITY", -8: "TIMEOUT", -9: "STATE", -10: "INTERNAL",
}
MEM_HOST, MEM_DEVICE = 0, 1
MODELS = {"fixed_corotated": 0, "neo_hookean": 1}
SOLVERS = {"mls": 0, "standard": 1, "pb": 2}
RIGID_TYPES = {"sphere": 0, "box": 1, "quad_slicer": 2, "segments": 3, "arc": 4, "mesh_slicer": 5, "none": -1}
FIELD = {"x": 1, "v": 2, "C": 4, "F": 8, "order": 16, "impulse": 32}
FIELD_SHAPE = {"x": (3,), "v": (3,), "C": (3, 3), "F": (3, 3), "order": ()}
OPT = {"use_graphs": 1, "launch_mode": 2, "p2g_threads": 3, "g2p_threads": 4, "ctas_per_sm": 5, "graph_chunk": 6,
       "phase_timing": 7, "p2g_chunk": 8, "fused": 9, "g2p_regs64": 10}
MAX_PTS = 64
MAX_TRIS = 64
MAX_SPINE = 16
MAX_RIGIDS = 8
EBIT = {"out_of_domain": 1, "nonfinite": 2, "inverted": 4, "timeout": 8, "internal": 16}


class MPMError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status})")


class mpm_config(ct.Structure):
    _fields_ = [
        ("n_scenes", ct.c_int32), ("grid_n", ct.c_int32), ("scene_grid_n", ct.POINTER(ct.c_int32)),
        ("max_particles", ct.c_int64), ("model", ct.c_int32), ("plasticity", ct.c_int32),
        ("yield_stress", ct.c_float), ("gravity", ct.c_float * 3), ("bound", ct.c_int32),
        ("floor_sticky", ct.c_int32), ("timeout_ms", ct.c_int32), ("tape_checkpoint_every", ct.c_int32),
        ("tape_max_substeps", ct.c_int32), ("solver", ct.c_int32), ("pb_iterations", ct.c_int32),
        ("pb_beta", ct.c_float), ("reserved", ct.c_int32 * 4),
    ]


class mpm_rigid(ct.Structure):
    _fields_ = [
        ("type", ct.c_int32), ("n_points", ct.c_int32), ("center", ct.c_float * 3), ("quat", ct.c_float * 4),
        ("vel", ct.c_float * 3), ("omega", ct.c_float * 3), ("mu_k", ct.c_float), ("c_d", ct.c_float),
        ("margin", ct.c_float), ("radius", ct.c_float), ("half", ct.c_float * 3), ("thickness", ct.c_float),
        ("spine_radius", ct.c_float), ("points", (ct.c_float * 3) * MAX_PTS),
        ("n_triangles", ct.c_int32), ("n_spine", ct.c_int32), ("triangles", (ct.c_int32 * 3) * MAX_TRIS),
        ("spine", ct.c_int32 * MAX_SPINE),
    ]


_lib = None

_P = ct.c_void_p
_SIGS = {
    "mpm_create": (ct.c_int, [ct.POINTER(mpm_config), _P, ct.POINTER(_P)]),
    "mpm_destroy": (ct.c_int, [_P]),
    "mpm_status_string": (ct.c_char_p, [ct.c_int]),
    "mpm_set_option": (ct.c_int, [_P, ct.c_int, ct.c_int64]),
    "mpm_get_option": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int64)]),
    "mpm_add_particles": (ct.c_int, [_P, ct.c_int, ct.c_int64, _P, _P, _P, _P, ct.c_float, ct.c_float, ct.c_float,
                                     ct.c_float, ct.c_int, ct.POINTER(ct.c_int64)]),
    "mpm_set_rigid": (ct.c_int, [_P, ct.c_int, ct.c_int, ct.POINTER(mpm_rigid)]),
    "mpm_substep": (ct.c_int, [_P, ct.c_float, ct.c_int]),
    "mpm_read_state": (ct.c_int, [_P, ct.c_int, ct.c_uint32, ct.POINTER(_P), ct.c_int]),
    "mpm_write_state": (ct.c_int, [_P, ct.c_int, ct.c_uint32, ct.POINTER(_P), ct.c_int]),
    "mpm_read_grid": (ct.c_int, [_P, ct.c_int, _P, ct.c_int]),
    "mpm_get_error": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_uint32)]),
    "mpm_scene_count": (ct.c_int, [_P, ct.c_int, ct.POINTER(ct.c_int64)]),
    "mpm_tape_begin": (ct.c_int, [_P]),
    "mpm_backward": (ct.c_int, [_P, _P, _P, _P, _P, _P, ct.c_int]),
    "mpm_backward_state": (ct.c_int, [_P, ct.POINTER(_P), ct.POINTER(_P), _P, _P, ct.c_int]),
    "mpm_autotune": (ct.c_int, [_P, ct.c_float, ct.c_int, ct.POINTER(ct.c_float)]),
    "mpm_phase_stats": (ct.c_int, [_P, ct.POINTER(ct.c_double), ct.POINTER(ct.c_int64), ct.POINTER(ct.c_int64),
                                   ct.c_int]),
    "mpm_sort_bricks_noalloc": (ct.c_int, [ct.c_int, ct.c_int64, _P, _P, _P, _P]),
}


def lib():
    """Load libmpm_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2502_18437_gb300.build.build()")
        L = ct.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _check(status, where):
    if status != MPM_OK:
        raise MPMError(status, where)
    return status


# ------------------------------------------------------------ raw mirrors

def mpm_create(cfg, stream=0):
    h = _P()
    _check(lib().mpm_create(ct.byref(cfg), _P(stream or 0), ct.byref(h)), "mpm_create")
    return h


def mpm_destroy(h):
    return lib().mpm_destroy(h)


def mpm_status_string(status):
    return lib().mpm_status_string(status).decode()


def mpm_set_option(h, option, value):
    opt = OPT[option] if isinstance(option, str) else int(option)
    return _check(lib().mpm_set_option(h, opt, int(value)), "mpm_set_option")


def mpm_get_option(h, option):
    opt = OPT[option] if isinstance(option, str) else int(option)
    v = ct.c_int64()
    _check(lib().mpm_get_option(h, opt, ct.byref(v)), "mpm_get_option")
    return v.value


def mpm_add_particles(h, scene, n, x, v, E, nu, E0, nu0, rho, V0, mem):
    first = ct.c_int64()
    _check(lib().mpm_add_particles(h, scene, n, x, v, E, nu, E0, nu0, rho, V0, mem, ct.byref(first)),
           "mpm_add_particles")
    return first.value


def mpm_set_rigid(h, scene, rigid_id, rigid):
    return _check(lib().mpm_set_rigid(h, scene, rigid_id, ct.byref(rigid)), "mpm_set_rigid")


def mpm_substep(h, dt, n_substeps):
    return _check(lib().mpm_substep(h, float(dt), int(n_substeps)), "mpm_substep")


def mpm_read_state(h, scene, fields, ptrs, mem):
    arr = (_P * len(ptrs))(*ptrs)
    return lib().mpm_read_state(h, scene, fields, arr, mem)


def mpm_write_state(h, scene, fields, ptrs, mem):
    arr = (_P * len(ptrs))(*ptrs)
    return _check(lib().mpm_write_state(h, scene, fields, arr, mem), "mpm_write_state")


def mpm_read_grid(h, scene, ptr, mem):
    return _check(lib().mpm_read_grid(h, scene, ptr, mem), "mpm_read_grid")


def mpm_get_error(h, scene):
    bits = ct.c_uint32()
    _check(lib().mpm_get_error(h, scene, ct.byref(bits)), "mpm_get_error")
    return bits.value


def mpm_scene_count(h, scene):
    n = ct.c_int64()
    _check(lib().mpm_scene_count(h, scene, ct.byref(n)), "mpm_scene_count")
    return n.value


def mpm_tape_begin(h):
    return _check(lib().mpm_tape_begin(h), "mpm_tape_begin")


def mpm_backward(h, dx, dv, dE, dnu, dv0, mem):
    return _check(lib().mpm_backward(h, dx, dv, dE, dnu, dv0, mem), "mpm_backward")


def mpm_backward_state(h, bar_in, bar_out, dmu, dlam, mem):
    ins = (_P * 4)(*[p or None for p in bar_in]) if bar_in is not None else None
    outs = (_P * 4)(*[p or None for p in bar_out]) if bar_out is not None else None
    return _check(lib().mpm_backward_state(h, ins, outs, dmu, dlam, mem), "mpm_backward_state")


def mpm_autotune(h, dt, trial_substeps):
    best = ct.c_float()
    _check(lib().mpm_autotune(h, float(dt), int(trial_substeps), ct.byref(best)), "mpm_autotune")
    return best.value


def mpm_phase_stats(h, reset=True):
    ms = (ct.c_double * 4)()
    n = ct.c_int64()
    act = (ct.c_int64 * 2)()
    _check(lib().mpm_phase_stats(h, ms, ct.byref(n), act, int(reset)), "mpm_phase_stats")
    return {"ms": list(ms), "substeps": n.value, "active_pbricks": act[0], "active_nbricks": act[1]}


def mpm_sort_bricks_noalloc(n, N, x_ptr, perm_ptr, brick_start_ptr=None, stream=0):
    """Allocation-free brick sort (device pointers); returns the status code."""
    return lib().mpm_sort_bricks_noalloc(int(n), int(N), x_ptr, perm_ptr, brick_start_ptr, _P(stream or 0))


# ------------------------------------------------------------- marshalling

def make_rigid(desc):
    """mpm_rigid from a plain description dict (see workloads)."""
    r = mpm_rigid()
    r.type = RIGID_TYPES[desc["type"]]
    q = desc.get("quat", (1.0, 0.0, 0.0, 0.0))
    for i in range(3):
        r.center[i] = desc["center"][i]
        r.vel[i] = desc.get("vel", (0, 0, 0))[i]
        r.omega[i] = desc.get("omega", (0, 0, 0))[i]
        r.half[i] = desc.get("half", (0, 0, 0))[i]
    for i in range(4):
        r.quat[i] = q[i]
    r.mu_k = desc.get("mu_k", 0.0)
    r.c_d = desc.get("c_d", 1.0)
    r.margin = desc.get("margin", 0.0)
    r.radius = desc.get("radius", 0.0)
    r.thickness = desc.get("thickness", 0.0)
    r.spine_radius = desc.get("spine_radius", 0.5 * r.thickness)
    pts = np.asarray(desc.get("pts", np.zeros((0, 3))), dtype=np.float32).reshape(-1, 3)
    if len(pts) > MAX_PTS:
        raise ValueError("too many segment points")
    r.n_points = len(pts)
    for i, p in enumerate(pts):
        for d in range(3):
            r.points[i][d] = float(p[d])
    tris = np.asarray(desc.get("tris", np.zeros((0, 3))), dtype=np.int32).reshape(-1, 3)
    spine = np.asarray(desc.get("spine", []), dtype=np.int32).reshape(-1)
    if len(tris) > MAX_TRIS or len(spine) > MAX_SPINE:
        raise ValueError("too many mesh triangles or spine points")
    r.n_triangles, r.n_spine = len(tris), len(spine)
    for i, t in enumerate(tris):
        for d in range(3):
            r.triangles[i][d] = int(t[d])
    for i, v in enumerate(spine):
        r.spine[i] = int(v)
    return r


def _torch():
    try:
        import torch
        return torch
    except ImportError:
        return None


def _is_cuda_tensor(a):
    t = _torch()
    return t is not None and isinstance(a, t.Tensor) and a.is_cuda


def _ptr(a, dtype=np.float32):
    """(pointer, mem, keepalive) of a numpy array or CUDA tensor, or None."""
    if a is None:
        return None, MEM_HOST, None
    if _is_cuda_tensor(a):
        t = _torch()
        want = t.float32 if dtype == np.float32 else t.int32
        if a.dtype != want or not a.is_contiguous():
            a = a.to(want).contiguous()
        return a.data_ptr(), MEM_DEVICE, a
    arr = np.ascontiguousarray(np.asarray(a, dtype=dtype))
    return arr.ctypes.data, MEM_HOST, arr


def _default_stream():
    t = _torch()
    if t is not None and t.cuda.is_available() and t.cuda.is_initialized():
        return t.cuda.current_stream().cuda_stream
    return 0


class Simulation:
    """A context of one or more scenes (batched) sharing one CUDA stream."""

    def __init__(self, grid_n=64, max_particles=1 << 20, *, n_scenes=1, scene_grid_n=None,
                 model="fixed_corotated", plasticity=False, yield_stress=0.0, gravity=(0.0, -9.8, 0.0),
                 bound=3, floor_sticky=True, timeout_ms=20000, tape_checkpoint_every=0, tape_max_substeps=0,
                 solver="mls", pb_iterations=10, pb_beta=1.0, stream=None):
        cfg = mpm_config()
        cfg.n_scenes = int(n_scenes)
        cfg.grid_n = int(grid_n)
        self._scene_n = None
        if scene_grid_n is not None:
            self._scene_n = (ct.c_int32 * n_scenes)(*[int(v) for v in scene_grid_n])
            cfg.scene_grid_n = ct.cast(self._scene_n, ct.POINTER(ct.c_int32))
        cfg.max_particles = int(max_particles)
        cfg.model = MODELS[model] if isinstance(model, str) else int(model)
        cfg.plasticity = int(bool(plasticity))
        cfg.yield_stress = float(yield_stress)
        for i in range(3):
            cfg.gravity[i] = float(gravity[i])
        cfg.bound = int(bound)
        cfg.floor_sticky = int(bool(floor_sticky))
        cfg.timeout_ms = int(timeout_ms)
        cfg.tape_checkpoint_every = int(tape_checkpoint_every)
        cfg.tape_max_substeps = int(tape_max_substeps)
        cfg.solver = SOLVERS[solver] if isinstance(solver, str) else int(solver)
        cfg.pb_iterations = int(pb_iterations)
        cfg.pb_beta = float(pb_beta)
        self.n_scenes = n_scenes
        self.grid_n = list(scene_grid_n) if scene_grid_n is not None else [grid_n] * n_scenes
        self.stream = _default_stream() if stream is None else stream
        self.h = mpm_create(cfg, self.stream)

    # lifecycle
    def close(self):
        if getattr(self, "h", None):
            mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_option(self, name, value):
        mpm_set_option(self.h, name, value)

    def get_option(self, name):
        return mpm_get_option(self.h, name)

    # factory
    def add_particles(self, scene, x, v=None, E=None, nu=None, *, E0=0.0, nu0=0.0, rho=1.0, V0=1.0):
        px, mem, kx = _ptr(x)
        n = (kx.numel() if _is_cuda_tensor(kx) else kx.size) // 3
        keep = [kx]
        ptrs = []
        for a in (v, E, nu):
            p, m, k = _ptr(a)
            if a is not None and m != mem:
                raise ValueError("all inputs of one call must live in the same memory")
            keep.append(k)
            ptrs.append(p)
        return mpm_add_particles(self.h, scene, n, px, ptrs[0], ptrs[1], ptrs[2], float(E0), float(nu0),
                                 float(rho), float(V0), mem)

    def set_rigid(self, scene, rigid_id, desc):
        mpm_set_rigid(self.h, scene, rigid_id, make_rigid(desc))

    def remove_rigid(self, scene, rigid_id):
        r = mpm_rigid()
        r.type = -1
        mpm_set_rigid(self.h, scene, rigid_id, r)

    # simulation
    def substep(self, dt, n=1):
        mpm_substep(self.h, dt, n)

    def count(self, scene=0):
        return mpm_scene_count(self.h, scene)

    def read_state(self, scene=0, fields=("x", "v", "C", "F"), device=False, check=True):
        n = self.count(scene)
        t = _torch()
        out, ptrs, mask = {}, [], 0
        for f in sorted(fields, key=lambda f: FIELD[f]):
            mask |= FIELD[f]
        for f in sorted(fields, key=lambda f: FIELD[f]):
            if f == "impulse":
                shape, dt_np = (MAX_RIGIDS, 6), np.float64
            else:
                shape, dt_np = (n,) + FIELD_SHAPE[f], (np.int32 if f == "order" else np.float32)
            if device:
                tt = {np.float32: t.float32, np.int32: t.int32, np.float64: t.float64}[dt_np]
                a = t.empty(shape, dtype=tt, device="cuda")
                ptrs.append(a.data_ptr())
            else:
                a = np.empty(shape, dtype=dt_np)
                ptrs.append(a.ctypes.data)
            out[f] = a
        status = mpm_read_state(self.h, scene, mask, ptrs, MEM_DEVICE if device else MEM_HOST)
        if check:
            _check(status, "mpm_read_state")
        else:
            out["status"] = status
        return out

    def write_state(self, scene=0, **fields):
        mask, ptrs, keep, mem = 0, [], [], None
        for f in sorted(fields, key=lambda f: FIELD[f]):
            p, m, k = _ptr(fields[f])
            if mem is not None and m != mem:
                raise ValueError("all inputs of one call must live in the same memory")
            mem = m
            mask |= FIELD[f]
            ptrs.append(p)
            keep.append(k)
        mpm_write_state(self.h, scene, mask, ptrs, mem)

    def read_grid(self, scene=0):
        n = self.grid_n[scene]
        g = np.empty((n, n, n, 4), dtype=np.float32)
        mpm_read_grid(self.h, scene, g.ctypes.data, MEM_HOST)
        return g

    def error_bits(self, scene=0):
        return mpm_get_error(self.h, scene)

    def impulse(self, scene=0):
        return self.read_state(scene, ("impulse",))["impulse"]

    def tape_begin(self):
        mpm_tape_begin(self.h)

    def backward(self, dL_dx=None, dL_dv=None, *, device=False):
        """Gradients (dE, dnu, dv0) over all particles, scene-major id order."""
        n = sum(self.count(s) for s in range(self.n_scenes))
        t = _torch()
        if device:
            outs = [t.zeros(n, device="cuda"), t.zeros(n, device="cuda"), t.zeros((n, 3), device="cuda")]
            ptr = lambda a: a.data_ptr()
            mem = MEM_DEVICE
        else:
            outs = [np.zeros(n, np.float32), np.zeros(n, np.float32), np.zeros((n, 3), np.float32)]
            ptr = lambda a: a.ctypes.data
            mem = MEM_HOST
        ins = []
        for a in (dL_dx, dL_dv):
            p, m, k = _ptr(a)
            if a is not None and m != mem:
                raise ValueError("gradient inputs must live where the outputs are requested")
            ins.append((p, k))
        mpm_backward(self.h, ins[0][0], ins[1][0], ptr(outs[0]), ptr(outs[1]), ptr(outs[2]), mem)
        return outs

    def backward_state(self, bar=None, *, want=("x", "v", "C", "F")):
        """Adjoint of the state at tape_begin from the adjoint of the final state.
        ``bar``: dict field -> (N,3) / (N,3,3) float32 numpy array (missing = 0).
        Returns a dict with the wanted fields' adjoints and "mu", "lam"."""
        n = sum(self.count(s) for s in range(self.n_scenes))
        bar = bar or {}
        shapes = {"x": (n, 3), "v": (n, 3), "C": (n, 3, 3), "F": (n, 3, 3)}
        keep, ins = [], []
        for f in ("x", "v", "C", "F"):
            if f in bar:
                a = np.ascontiguousarray(np.asarray(bar[f], dtype=np.float32).reshape(shapes[f]))
                keep.append(a)
                ins.append(a.ctypes.data)
            else:
                ins.append(None)
        out = {f: np.zeros(shapes[f], np.float32) for f in want}
        outs = [out[f].ctypes.data if f in out else None for f in ("x", "v", "C", "F")]
        out["mu"], out["lam"] = np.zeros(n, np.float32), np.zeros(n, np.float32)
        mpm_backward_state(self.h, ins, outs, out["mu"].ctypes.data, out["lam"].ctypes.data, MEM_HOST)
        return out

    def autotune(self, dt, trial_substeps=5):
        return mpm_autotune(self.h, dt, trial_substeps)

    def phase_stats(self, reset=True):
        return mpm_phase_stats(self.h, reset)


def from_workload(sc, *, max_particles=None, **kw):
    """Simulation holding one workload dict (see workloads) in scene 0."""
    sim = Simulation(sc["n"], max_particles or len(sc["x"]), model=sc["model"], plasticity=sc["plasticity"],
                     yield_stress=sc["yield_stress"], gravity=sc["gravity"], bound=sc["bound"],
                     floor_sticky=sc["floor_sticky"], **kw)
    _add_workload(sim, 0, sc)
    return sim


def _add_workload(sim, scene, sc):
    E, nu = sc["E"], sc["nu"]
    if len(E) and np.all(E == E[0]) and np.all(nu == nu[0]):
        # uniform material: no per-particle arrays on the device
        sim.add_particles(scene, sc["x"], sc["v"], E0=float(E[0]), nu0=float(nu[0]), rho=sc["rho"], V0=sc["V0"])
    else:
        sim.add_particles(scene, sc["x"], sc["v"], E, nu, rho=sc["rho"], V0=sc["V0"])
    for i, r in enumerate(sc["rigids"]):
        sim.set_rigid(scene, i, r)


def from_scenes(scenes, **kw):
    """Batched Simulation: scene s of the context holds scenes[s]."""
    s0 = scenes[0]
    sim = Simulation(s0["n"], sum(len(s["x"]) for s in scenes), n_scenes=len(scenes),
                     scene_grid_n=[s["n"] for s in scenes], model=s0["model"], plasticity=s0["plasticity"],
                     yield_stress=s0["yield_stress"], gravity=s0["gravity"], bound=s0["bound"],
                     floor_sticky=s0["floor_sticky"], **kw)
    for i, s in enumerate(scenes):
        _add_workload(sim, i, s)
    return sim
