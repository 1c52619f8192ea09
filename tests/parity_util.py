"""Helpers shared by the GPU parity tests: build oracle inputs from a workload or
from a state read back from the GPU, and compare fields with stated tolerances.

Tolerance model (FP32 kernel vs FP64 oracle from identical FP32 inputs): every
field of one substep is compared element by element as
    |gpu - oracle| <= atol + rtol * |oracle|,   atol = rel_scale * max|oracle field|
with rtol = 2e-5 and rel_scale = 2e-5 per field, i.e. ~170 FP32 units of roundoff
(2^-24) relative to the field's scale.  The budget covers the rounding of the
27-node sums, of the FP32 Jacobi SVD/polar decomposition in the stress (relative
error ~1e-6 of |F|, amplified by 2 mu / |tau| where stresses are small) and of
single-precision atomics in an arbitrary order.
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


def perturbed(sc, seed, f_amp=0.01, c_amp=1.0, v_amp=0.1):
    """Random C, F = I + f_amp N(0,1), v += v_amp N(0,1): exercises every term."""
    g = np.random.default_rng(seed)
    N = len(sc["x"])
    F = (np.eye(3) + f_amp * g.normal(size=(N, 3, 3))).astype(np.float32)
    C = (c_amp * g.normal(size=(N, 3, 3))).astype(np.float32)
    v = (sc["v"] + v_amp * g.normal(size=(N, 3))).astype(np.float32)
    return v, C, F
