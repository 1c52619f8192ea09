"""Helpers shared by the GPU parity tests: build oracle inputs from a workload or
from a state read back from the GPU, and compare fields with stated tolerances.

Tolerance model (FP32 kernel vs FP64 oracle from identical FP32 inputs): every
field of one substep is compared element by element as
    |gpu - oracle| <= atol + rtol * |oracle|,   atol = rel_scale * max|oracle field|
with rtol = 2e-5 and rel_scale = 2e-5 per field, i.e. ~340 FP32 units of roundoff
(2^-24) relative to the field's scale.  The budget covers the rounding of the
27-node sums, of the FP32 Jacobi SVD/polar decomposition in the stress (relative
error ~1e-6 of |F|, amplified by 2 mu / |tau| where stresses are small) and of
single-precision atomics in an arbitrary order.

Two fields carry cancellation, so their absolute tolerances scale with the
terms that cancel rather than with the result:
 - v: the stress part of a node's momentum, dt V0 (4/dx^2) tau (x_I - x_p),
   contributes velocities of order s_v = 4 dt n |tau| / rho per node that
   largely cancel over the stencil.  The FP32 stress itself has an absolute
   floor: a strain below the unit roundoff of F ~ I is not representable, so
   tau carries an error up to tau_0 = 4 (2 mu + 3 lambda) 2^-24 whatever its
   size.  atol_v = 2e-5 (max|v| + s_v) + 4 dt n tau_0 / rho.
 - C = (4/dx) sum_I N_I v_I ((x_I - x_p)/dx)^T is a velocity gradient: an error
   delta in the node velocities becomes up to 4n delta in C, and the cancellation
   of the bulk velocity (sum_I N_I (x_I - x_p) = 0) leaves up to 2^-24 |v_I| per
   term: atol_C = 4n (2e-5 s_v + 4 dt n tau_0 / rho) + 27 * 4n * 2^-24 (max|v| + s_v).
"""
import numpy as np

import oracle

RTOL = 2e-5
REL_SCALE = 2e-5


def oracle_cfg(sc):
    return oracle.config_from_workload(sc)


def oracle_state(sc, x=None, v=None, C=None, F=None):
    return oracle.state_from_workload(sc, x, v, C, F)


def oracle_rigids(sc, advanced_substeps=0):
    rig = oracle.rigid_array(sc["rigids"])
    for _ in range(advanced_substeps):
        for i in range(len(sc["rigids"])):
            oracle.rigid_advance(rig[i], sc["dt"])
    return rig, len(sc["rigids"])


def assert_close(name, got, ref, rtol=RTOL, rel_scale=REL_SCALE, atol_floor=0.0):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert got.shape == ref.shape, (name, got.shape, ref.shape)
    scale = float(np.max(np.abs(ref))) if ref.size else 0.0
    atol = max(rel_scale * scale, atol_floor)
    err = np.abs(got - ref)
    bad = err > atol + rtol * np.abs(ref)
    if np.any(bad):
        i = np.unravel_index(np.argmax(err - atol - rtol * np.abs(ref)), err.shape)
        raise AssertionError(f"{name}: {int(bad.sum())}/{bad.size} elements out of tolerance; worst at {i}: "
                             f"gpu={got[i]!r} oracle={ref[i]!r} |err|={err[i]:.3e} atol={atol:.3e} "
                             f"(field scale {scale:.3e})")
    return float(err.max()) if err.size else 0.0


EPS32 = 2.0 ** -24


class Scales:
    """Error scales of one substep from a given state (see module docstring)."""

    def __init__(self, sc, F_before, dt=None):
        dt = dt or sc["dt"]
        n, rho = sc["n"], sc["rho"]
        mu, lam = oracle.lame_arrays(sc["E"], sc["nu"])
        tau_max = 0.0
        if len(F_before):
            tau, _ = oracle.kirchhoff_all(sc["model"], F_before, mu, lam)
            tau_max = float(np.max(np.abs(tau)))
        tau0 = 4.0 * (2.0 * float(np.max(mu, initial=0.0)) + 3.0 * float(np.max(lam, initial=0.0))) * EPS32
        self.n = n
        self.s_v = 4.0 * dt * n * tau_max / rho
        self.v_floor = 4.0 * dt * n * tau0 / rho

    def atol_v(self, v):
        return REL_SCALE * (_amax(v) + self.s_v) + self.v_floor

    def atol_C(self, v):
        return 4 * self.n * (REL_SCALE * self.s_v + self.v_floor) + 27 * 4 * self.n * EPS32 * (_amax(v) + self.s_v)


def _amax(a):
    return float(np.max(np.abs(a))) if np.size(a) else 0.0


def perturbed(sc, seed, f_amp=0.01, c_amp=1.0, v_amp=0.1):
    """Random C, F = I + f_amp N(0,1), v += v_amp N(0,1): exercises every term."""
    g = np.random.default_rng(seed)
    N = len(sc["x"])
    F = (np.eye(3) + f_amp * g.normal(size=(N, 3, 3))).astype(np.float32)
    C = (c_amp * g.normal(size=(N, 3, 3))).astype(np.float32)
    v = (sc["v"] + v_amp * g.normal(size=(N, 3))).astype(np.float32)
    return v, C, F
