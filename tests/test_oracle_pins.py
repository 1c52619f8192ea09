"""Pins of the FP64 oracle against facts fixed outside it: closed forms,
conservation laws, LAPACK/scipy, brute-force sampling and hand-worked values.

Each test names the passage of arXiv 2502.18437 (or the textbook fact) it relies
on.  A plausible slip in the oracle (a dropped term, a wrong sign or index, a
transposed operand) breaks at least one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2502_18437_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
RNG = np.random.default_rng(12345)


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0.0]])


# --------------------------------------------------------------- B-spline

def test_bspline_golden_values():
    # Sec. III-A quadratic basis; hand-worked values in tests/golden.
    rows = np.loadtxt(os.path.join(GOLDEN, "bspline_weights.txt"))
    for f, w0, w1, w2 in rows:
        assert np.array_equal(oracle.bspline_weights(f), [w0, w1, w2])


def test_bspline_moments():
    # Partition of unity, zero first moment and second moment dx^2/4: the
    # D = dx^2/4 I of Eq. 9 for the quadratic basis.
    for f in RNG.uniform(0.5, 1.5, 200):
        w = oracle.bspline_weights(f)
        d = np.arange(3) - f
        assert abs(w.sum() - 1) < 1e-15
        assert abs((w * d).sum()) < 1e-15
        assert abs((w * d * d).sum() - 0.25) < 1e-15
        assert np.all(w >= 0)


# -------------------------------------------------------------------- SVD

def _svd_cases():
    cases = [np.eye(3), np.diag([2.0, 2.0, 1.0]), np.diag([1.0, 1.0, -1.0]), np.diag([3.0, 0.0, 0.0])]
    for _ in range(60):
        cases.append(RNG.normal(size=(3, 3)))
    for _ in range(20):
        cases.append(np.eye(3) + 1e-6 * RNG.normal(size=(3, 3)))
    for _ in range(10):  # repeated singular values
        Q1, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
        Q2, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
        cases.append(Q1 @ np.diag([1.5, 1.5, 0.7]) @ Q2)
    return cases


def test_svd_against_lapack():
    for A in _svd_cases():
        U, S, V = oracle.svd3(A)
        assert rel(U @ np.diag(S) @ V.T, A) < 1e-12 or np.max(np.abs(U @ np.diag(S) @ V.T - A)) < 1e-13
        assert np.max(np.abs(U.T @ U - np.eye(3))) < 1e-12
        assert np.max(np.abs(V.T @ V - np.eye(3))) < 1e-12
        assert abs(np.linalg.det(U) - 1) < 1e-12 and abs(np.linalg.det(V) - 1) < 1e-12
        ref = np.linalg.svd(A, compute_uv=False)
        assert np.max(np.abs(np.abs(S) - ref)) <= 1e-12 * max(ref[0], 1)
        d = np.linalg.det(A)
        if abs(d) > 1e-9:
            assert np.sign(S[2]) == np.sign(d)
            assert S[0] > 0 and S[1] > 0


def test_polar_against_scipy():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    for A in _svd_cases():
        if np.linalg.det(A) <= 1e-6:
            continue
        R = oracle.polar_R(A)
        Rs, _ = scipy_linalg.polar(A)
        assert np.max(np.abs(R - Rs)) < 1e-10


# ----------------------------------------------------------------- stress

def _energy(model, F, mu, lam):
    # Textbook energy densities whose first Piola stress P gives tau = P F^T.
    J = np.linalg.det(F)
    if model == "fixed_corotated":
        U, s, Vt = np.linalg.svd(F)
        R = U @ Vt
        if np.linalg.det(R) < 0:
            U[:, 2] *= -1
            R = U @ Vt
        return mu * np.sum((F - R) ** 2) + 0.5 * lam * (J - 1) ** 2
    return 0.5 * mu * (np.sum(F * F) - 3) - mu * math.log(J) + 0.5 * lam * math.log(J) ** 2


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
def test_stress_is_energy_derivative(model):
    # tau = (dPsi/dF) F^T, checked by central differences of the energy.
    mu, lam = 3.0, 5.0
    for _ in range(10):
        F = np.eye(3) + 0.2 * RNG.normal(size=(3, 3))
        tau, err = oracle.kirchhoff(model, F, mu, lam)
        assert err == 0
        h = 1e-6
        P = np.zeros((3, 3))
        for i in range(3):
            for j in range(3):
                E = np.zeros((3, 3))
                E[i, j] = h
                P[i, j] = (_energy(model, F + E, mu, lam) - _energy(model, F - E, mu, lam)) / (2 * h)
        assert rel(tau, P @ F.T) < 1e-7


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
def test_stress_rest_symmetry_equivariance(model):
    mu, lam = 7.0, 11.0
    tau, _ = oracle.kirchhoff(model, np.eye(3), mu, lam)
    assert np.max(np.abs(tau)) < 1e-14
    for _ in range(10):
        F = np.eye(3) + 0.3 * RNG.normal(size=(3, 3))
        if np.linalg.det(F) <= 0.1:
            continue
        Q, _ = np.linalg.qr(RNG.normal(size=(3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        t1, _ = oracle.kirchhoff(model, F, mu, lam)
        t2, _ = oracle.kirchhoff(model, Q @ F, mu, lam)
        assert np.max(np.abs(t1 - t1.T)) < 1e-12
        assert rel(t2, Q @ t1 @ Q.T) < 1e-12


def test_stress_diagonal_closed_form():
    # F = diag(a,b,c) > 0 is its own stretch (R = I).
    a, b, c = 1.1, 0.9, 1.05
    mu, lam = 2.0, 3.0
    J = a * b * c
    tau, _ = oracle.kirchhoff("fixed_corotated", np.diag([a, b, c]), mu, lam)
    expect = np.diag([2 * mu * (s - 1) * s + lam * (J - 1) * J for s in (a, b, c)])
    assert np.max(np.abs(tau - expect)) < 1e-14
    tau, _ = oracle.kirchhoff("neo_hookean", np.diag([a, b, c]), mu, lam)
    expect = np.diag([mu * (s * s - 1) + lam * math.log(J) for s in (a, b, c)])
    assert np.max(np.abs(tau - expect)) < 1e-14


def test_neo_hookean_inverted_flags():
    tau, err = oracle.kirchhoff("neo_hookean", np.diag([1.0, 1.0, -1.0]), 1.0, 1.0)
    assert err == oracle.ERR_INVERTED and np.all(tau == 0)


def test_lame_textbook():
    mu, lam = oracle.lame(1e4, 0.3)
    assert abs(mu - 1e4 / 2.6) < 1e-9 and abs(lam - 3000 / 0.52) < 1e-9


# ------------------------------------------------------------- plasticity

def test_von_mises_projection():
    mu, ty = 100.0, 50.0
    for _ in range(50):
        F = np.eye(3) + 0.5 * RNG.normal(size=(3, 3))
        if np.linalg.det(F) <= 0.05:
            continue
        Fp, err = oracle.von_mises(F, mu, ty)
        assert err == 0
        s0 = np.linalg.svd(F, compute_uv=False)
        s1 = np.linalg.svd(Fp, compute_uv=False)
        e0, e1 = np.log(s0), np.log(s1)
        dev0, dev1 = e0 - e0.mean(), e1 - e1.mean()
        # volume preserved, yield surface respected, deviator direction kept
        assert abs(e1.sum() - e0.sum()) < 1e-12
        assert 2 * mu * np.linalg.norm(dev1) <= ty * (1 + 1e-12)
        if 2 * mu * np.linalg.norm(dev0) > ty:
            assert abs(2 * mu * np.linalg.norm(dev1) - ty) < 1e-10
            assert np.max(np.abs(dev1 / np.linalg.norm(dev1) - dev0 / np.linalg.norm(dev0))) < 1e-10
            # same singular vectors: F_p F^T and F^T F_p symmetric
            assert np.max(np.abs(Fp @ F.T - (Fp @ F.T).T)) < 1e-12
            assert np.max(np.abs(F.T @ Fp - (F.T @ Fp).T)) < 1e-12
        else:
            assert np.max(np.abs(Fp - F)) < 1e-14


def test_von_mises_diagonal_closed_form():
    # F = diag(exp(e)) with tr e = 0: projection scales e to |e| = yield/(2 mu).
    e = np.array([0.3, -0.1, -0.2])
    mu, ty = 10.0, 2.0
    Fp, _ = oracle.von_mises(np.diag(np.exp(e)), mu, ty)
    target = e / np.linalg.norm(e) * ty / (2 * mu)
    assert np.max(np.abs(Fp - np.diag(np.exp(target)))) < 1e-13


# --------------------------------------------------------- contact + SDFs

def test_sphere_contact_closed_forms():
    # Sec. IV-A: normal part removed when approaching, Eq. 11 friction on the
    # tangential part, separating nodes untouched.
    r = oracle.make_rigid(W.sphere((0.5, 0.5, 0.5), 0.1, mu_k=0.0, c_d=1.0))
    x = np.array([0.5, 0.55, 0.5])  # inside, normal +y
    v = np.array([0.3, -1.0, 0.0])
    assert np.allclose(oracle.contact_node(r, x, 2.0, v), [0.3, 0.0, 0.0], atol=1e-15)
    assert np.allclose(oracle.rigid_impulse(r)[:3], [0.0, -2.0, 0.0])  # -m (v' - v)
    assert np.array_equal(oracle.contact_node(r, x, 1.0, [0.3, 1.0, 0.0]), [0.3, 1.0, 0.0])
    far = np.array([0.5, 0.8, 0.5])
    assert np.array_equal(oracle.contact_node(r, far, 1.0, v), v)
    # friction: |v_t|=0.3, |v_n|=1, mu_k = 0.2 -> factor 1 - 0.2/0.3
    r = oracle.make_rigid(W.sphere((0.5, 0.5, 0.5), 0.1, mu_k=0.2, c_d=0.5))
    out = oracle.contact_node(r, x, 1.0, v)
    assert np.allclose(out, [0.5 * (1 - 0.2 / 0.3) * 0.3, 0, 0], atol=1e-15)
    # static friction: mu_k large -> stick to the rigid
    r = oracle.make_rigid(W.sphere((0.5, 0.5, 0.5), 0.1, mu_k=10.0, vel=(0.1, 0.2, 0.3)))
    assert np.allclose(oracle.contact_node(r, x, 1.0, v), [0.1, 0.2, 0.3], atol=1e-15)


def test_rigid_velocity_field_and_angular_impulse():
    w = np.array([0.0, 0.0, 2.0])
    r = oracle.make_rigid(W.sphere((0.5, 0.5, 0.5), 0.1, mu_k=10.0, omega=w))
    x = np.array([0.55, 0.5, 0.5])
    vr = np.cross(w, x - 0.5)
    out = oracle.contact_node(r, x, 3.0, [0.0, 0.0, -1.0])  # approaching along -x? normal +x
    # v_rel = (0,0,-1) - vr; normal +x, v_n = 0 -> counts as separating (v_n >= 0)
    assert np.array_equal(out, [0.0, 0.0, -1.0])
    out = oracle.contact_node(r, x, 3.0, [-1.0, 0.0, 0.0])
    assert np.allclose(out, vr, atol=1e-15)
    imp = oracle.rigid_impulse(r)
    dp = 3.0 * (out - np.array([-1.0, 0, 0]))
    assert np.allclose(imp[:3], -dp) and np.allclose(imp[3:], -np.cross(x - 0.5, dp))


def _brute_min_dist(p, pts):
    return np.min(np.linalg.norm(pts - p, axis=1))


def test_box_sdf_brute_force():
    half = np.array([0.1, 0.05, 0.08])
    q = (math.cos(0.3), 0.0, math.sin(0.3), 0.0)
    r = oracle.make_rigid(W.box((0.5, 0.5, 0.5), half, quat=q, margin=1.0))
    c, R = oracle.rigid_pose(r)
    m = 161
    g = np.linspace(-1, 1, m)
    faces = []
    for ax in range(3):
        o = [i for i in range(3) if i != ax]
        A, B = np.meshgrid(g * half[o[0]], g * half[o[1]], indexing="ij")
        for s in (-1, 1):
            P = np.zeros((m * m, 3))
            P[:, ax] = s * half[ax]
            P[:, o[0]], P[:, o[1]] = A.ravel(), B.ravel()
            faces.append(P)
    surf = np.concatenate(faces) @ R.T + c
    for _ in range(200):
        p = c + RNG.uniform(-0.2, 0.2, 3)
        code, n, t, d = oracle.geometry(r, p)
        loc = R.T @ (p - c)
        inside = np.all(np.abs(loc) <= half)
        bd = _brute_min_dist(p, surf)
        assert abs(abs(d) - bd) < 2.5e-3
        assert (d < 0) == inside
        assert abs(np.linalg.norm(n) - 1) < 1e-12


def test_quad_slicer_sdf_brute_force_and_regions():
    a, b, h = 0.15, 0.04, 0.002
    r = oracle.make_rigid(W.quad_slicer((0.5, 0.16, 0.5), W.BLADE_EDGE_Z_DOWN, half_edge=a, half_depth=b,
                                        thickness=h, margin=0.01, spine_radius=0.001))
    c, R = oracle.rigid_pose(r)
    # body axes: edge direction world z, spine->edge world -y, normal world x
    assert np.allclose(R @ [1, 0, 0], [0, 0, 1]) and np.allclose(R @ [0, 1, 0], [0, -1, 0])
    assert np.allclose(R @ [0, 0, 1], [1, 0, 0])
    S, T = np.meshgrid(np.linspace(-a, a, 301), np.linspace(-b, b, 81), indexing="ij")
    quad = np.stack([S.ravel(), T.ravel(), np.zeros(S.size)], -1) @ R.T + c
    spine = np.stack([np.linspace(-a, a, 3001), -b * np.ones(3001), np.zeros(3001)], -1) @ R.T + c
    for _ in range(300):
        p = c + RNG.uniform([-0.03, -0.07, -0.2], [0.03, 0.07, 0.2])
        code, n, t, d = oracle.geometry(r, p)
        dsp = _brute_min_dist(p, spine)
        if dsp < 0.011 - 2e-4:
            assert code == "sticky"
            continue
        if dsp > 0.011 + 2e-4:
            bd = _brute_min_dist(p, quad)
            assert abs(d - bd) < 1e-3
            if bd < 0.011 - 1e-3:
                assert code == "regular"
                # on the faces the normal points to the node's side of the blade
                side = np.sign(np.dot(R[:, 2], p - c)) or 1.0
                if abs(R.T @ (p - c))[0] <= a and abs(R.T @ (p - c))[1] <= b:
                    assert np.allclose(n, side * R[:, 2])
            elif bd > 0.011 + 1e-3:
                assert code == "none"


def test_segments_sdf_and_oned_rule():
    pts = np.array([[-0.1, 0, 0], [0.0, 0.02, 0], [0.1, 0.0, 0.03]])
    r = oracle.make_rigid(W.segments((0.5, 0.5, 0.5), (1, 0, 0, 0), pts, radius=0.003, margin=0.01,
                                     mu_k=0.0, c_d=1.0))
    line = np.concatenate([np.linspace(pts[i], pts[i + 1], 4001) for i in range(2)]) + 0.5
    for _ in range(200):
        p = 0.5 + RNG.uniform(-0.12, 0.12, 3) * [1, 0.2, 0.3]
        code, n, t, d = oracle.geometry(r, p)
        assert abs(d - _brute_min_dist(p, line)) < 1e-4
        assert code == ("oned" if d < 0.013 else "none")
    # Sec. IV-C / Eq. 12: motion along the tangent leaves the node alone,
    # lateral motion drags it with the rigid.
    tan = (pts[1] - pts[0]) / np.linalg.norm(pts[1] - pts[0])
    nrm = np.cross(tan, [0, 0, 1.0])
    x = 0.5 + 0.5 * (pts[0] + pts[1]) + 0.005 * nrm
    along = oracle.make_rigid(W.segments((0.5, 0.5, 0.5), (1, 0, 0, 0), pts, radius=0.003, margin=0.01,
                                         mu_k=0.0, c_d=1.0, vel=tuple(0.3 * tan)))
    assert np.array_equal(oracle.contact_node(along, x, 1.0, np.zeros(3)), np.zeros(3))
    lateral = oracle.make_rigid(W.segments((0.5, 0.5, 0.5), (1, 0, 0, 0), pts, radius=0.003, margin=0.01,
                                           mu_k=0.0, c_d=1.0, vel=tuple(0.3 * nrm)))
    assert np.allclose(oracle.contact_node(lateral, x, 1.0, np.zeros(3)), 0.3 * nrm, atol=1e-15)


def test_slicer_spine_sticky():
    r = oracle.make_rigid(W.quad_slicer((0.5, 0.16, 0.5), W.BLADE_EDGE_Z_DOWN, half_edge=0.15,
                                        half_depth=0.04, thickness=0.002, vel=(0, -0.1, 0), margin=0.005))
    x = np.array([0.5, 0.2 + 0.003, 0.5])  # just above the spine (spine at y = 0.2)
    assert oracle.geometry(r, x)[0] == "sticky"
    assert np.allclose(oracle.contact_node(r, x, 1.0, [1.0, 2.0, 3.0]), [0, -0.1, 0])


def test_rigid_advance_matches_rotation_exponential():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    w = np.array([0.3, -1.2, 0.7])
    r = oracle.make_rigid(W.box((0.1, 0.2, 0.3), (0.1, 0.1, 0.1), vel=(1.0, 2.0, -1.0), omega=w))
    c0, R0 = oracle.rigid_pose(r)
    for _ in range(37):
        oracle.rigid_advance(r, 0.01)
    c, R = oracle.rigid_pose(r)
    assert np.allclose(c, c0 + 0.37 * np.array([1.0, 2.0, -1.0]), atol=1e-14)
    assert np.max(np.abs(R - Rot.from_rotvec(0.37 * w).as_matrix() @ R0)) < 1e-13


# --------------------------------------------------------- transfers/step

def _cloud(N, n, lo=0.35, hi=0.65, seed=0):
    g = np.random.default_rng(seed)
    return lo + (hi - lo) * g.random((N, 3))


def test_p2g_conservation():
    # Eq. 1 and Eq. 8: mass and linear momentum are conserved exactly; the
    # angular momentum of the grid equals the APIC particle angular momentum
    # sum x_p x m v_p + m dx^2/4 eps:C_p^T (stress term vanishes for symmetric tau).
    n, N, m = 32, 500, 0.7
    cfg = oracle.make_config(n, m, 1e-4, model="fixed_corotated")
    g = np.random.default_rng(1)
    st = oracle.State(_cloud(N, n), g.normal(size=(N, 3)), g.normal(size=(N, 3, 3)),
                      np.eye(3) + 0.1 * g.normal(size=(N, 3, 3)), 3.0, 5.0)
    gm, gmv, err = oracle.p2g(cfg, st, 1e-3)
    assert err == 0
    assert abs(gm.sum() - N * m) < 1e-12 * N * m
    assert rel(gmv.sum(0), m * st.v.sum(0)) < 1e-12
    dx = 1.0 / n
    I = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) * dx
    Lg = np.cross(I, gmv).sum(0)
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    Lp = (np.cross(st.x, m * st.v) + m * dx * dx / 4 * np.einsum("ijk,pkj->pi", eps, st.C)).sum(0)
    assert rel(Lg, Lp) < 1e-12


def test_free_fall_closed_form():
    # Uniform velocity, F = I, C = 0, away from walls: the step reduces to
    # v_k = v0 + k dt g and x_k = x0 + k dt v0 + dt^2 g k(k+1)/2 (Eq. 3, 4).
    n, N, dt, k = 32, 300, 1e-3, 25
    cfg = oracle.make_config(n, 1.0, 1e-5)
    v0 = np.array([0.2, 0.1, -0.3])
    st = oracle.State(_cloud(N, n, 0.4, 0.6), np.tile(v0, (N, 1)), mu=10.0, lam=10.0)
    x0 = st.x.copy()
    assert oracle.run(cfg, st, dt, k) == 0
    g = np.array(cfg.gravity[:])
    assert np.max(np.abs(st.v - (v0 + k * dt * g))) < 1e-12
    assert np.max(np.abs(st.x - (x0 + k * dt * v0 + dt * dt * g * k * (k + 1) / 2))) < 1e-12
    assert np.max(np.abs(st.C)) < 1e-10 and np.max(np.abs(st.F - np.eye(3))) < 1e-12


def test_apic_reproduces_affine_fields():
    # APIC/MLS transfers (Eq. 8, 9) reproduce an affine velocity field exactly.
    n, N, dt = 32, 400, 1e-3
    cfg = oracle.make_config(n, 1.0, 1e-5, gravity=(0, 0, 0))
    g = np.random.default_rng(2)
    a, A = g.normal(size=3), g.normal(size=(3, 3))
    x = _cloud(N, n)
    st = oracle.State(x, a + x @ A.T, np.tile(A, (N, 1, 1)), mu=0.0, lam=0.0)
    assert oracle.run(cfg, st, dt, 1) == 0
    assert np.max(np.abs(st.v - (a + x @ A.T))) < 1e-12
    assert np.max(np.abs(st.C - A)) < 1e-10


def test_rigid_rotation_one_step():
    # A rotating field v = omega x (x - c) with C = [omega]x and no stress is
    # affine, so one step reproduces it on the grid and maps x - c to
    # (I + dt [omega]x)(x - c), with C unchanged and F = I + dt [omega]x
    # (Eq. 8-10).  (After that step v is no longer affine in the moved
    # positions with the same C, so the map is exact for one step only.)
    n, N, dt = 32, 200, 1e-3
    cfg = oracle.make_config(n, 1.0, 1e-5, gravity=(0, 0, 0))
    w = np.array([0.5, -1.0, 2.0])
    c = np.array([0.5, 0.5, 0.5])
    x = _cloud(N, n, 0.42, 0.58)
    st = oracle.State(x, np.cross(w, x - c), np.tile(skew(w), (N, 1, 1)), mu=0.0, lam=0.0)
    assert oracle.run(cfg, st, dt, 1) == 0
    M = np.eye(3) + dt * skew(w)
    assert np.max(np.abs(st.x - (c + (x - c) @ M.T))) < 1e-14
    assert np.max(np.abs(st.v - np.cross(w, x - c))) < 1e-13
    assert np.max(np.abs(st.C - skew(w))) < 1e-11
    assert np.max(np.abs(st.F - M)) < 1e-13


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
def test_step_conserves_momentum_and_angular_momentum(model):
    # With no gravity, walls or rigids the whole step (P2G, grid, G2P)
    # conserves linear and APIC angular momentum.
    n, N, dt, m = 32, 400, 2e-4, 0.3
    cfg = oracle.make_config(n, m, 1e-4, model=model, gravity=(0, 0, 0))
    g = np.random.default_rng(3)
    st = oracle.State(_cloud(N, n), g.normal(size=(N, 3)), 0.5 * g.normal(size=(N, 3, 3)),
                      np.eye(3) + 0.05 * g.normal(size=(N, 3, 3)), 40.0, 60.0)
    dx = 1.0 / n
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    L = lambda s: (np.cross(s.x, m * s.v) + m * dx * dx / 4 * np.einsum("ijk,pkj->pi", eps, s.C)).sum(0)
    P0, L0 = m * st.v.sum(0), L(st)
    assert oracle.run(cfg, st, dt, 3) == 0
    assert rel(m * st.v.sum(0), P0) < 1e-11
    assert rel(L(st), L0) < 1e-11


def test_contact_momentum_balance():
    # Two-way coupling bookkeeping (Sec. IV-A, Sec. V-C): the particles' momentum
    # change equals gravity's impulse minus the impulse given to the rigids,
    # linear and angular.
    sc = W.tissue_slab(cells=(24, 6, 24), lo=(0.3, 0.3, 0.3), size=(0.4, 0.1, 0.4), n=32, substeps=1)
    cfg = oracle.make_config(sc["n"], sc["rho"] * sc["V0"], sc["V0"], model=sc["model"])
    mu, lam = np.vectorize(oracle.lame)(sc["E"].astype(float), sc["nu"].astype(float))
    g = np.random.default_rng(4)
    st = oracle.State(sc["x"], 0.5 * g.normal(size=(len(sc["x"]), 3)), mu=mu, lam=lam)
    rig = oracle.rigid_array(sc["rigids"])
    m = cfg.m_p
    poses = [oracle.rigid_pose(rig[i])[0] for i in range(len(sc["rigids"]))]
    P0, L0 = m * st.v.sum(0), np.cross(st.x, m * st.v).sum(0)
    C0 = st.C.copy()
    gm, gv, err = oracle.substep(cfg, st, 1e-4, rig, len(sc["rigids"]))
    assert err == 0
    J = sum(oracle.rigid_impulse(rig[i])[:3] for i in range(len(sc["rigids"])))
    assert np.linalg.norm(J) > 0
    grav = 1e-4 * gm.sum() * np.array(cfg.gravity[:])
    assert rel(m * st.v.sum(0), P0 + grav - J) < 1e-10
    dx = 1.0 / cfg.n
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1
    n = cfg.n
    I = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) * dx
    Lnew = (np.cross(st.x, m * st.v) + m * dx * dx / 4 * np.einsum("ijk,pkj->pi", eps, st.C)).sum(0)
    Lold = L0 + (m * dx * dx / 4 * np.einsum("ijk,pkj->pi", eps, C0)).sum(0)
    Lgrav = np.cross(I, 1e-4 * gm[:, None] * np.array(cfg.gravity[:])).sum(0)
    Jang = sum(oracle.rigid_impulse(rig[i])[3:] + np.cross(poses[i], oracle.rigid_impulse(rig[i])[:3])
               for i in range(len(sc["rigids"])))
    assert rel(Lnew, Lold + Lgrav - Jang) < 1e-9


def test_grid_update_boundaries():
    # Domain walls (Eq. 3 "boundary conditions by altering the momentum"):
    # sticky floor zeroes the node, other walls remove the inward component only.
    n = 16
    cfg = oracle.make_config(n, 1.0, 1.0, gravity=(0, 0, 0))
    g = np.random.default_rng(5)
    gm = np.ones(n ** 3)
    gmv = g.normal(size=(n ** 3, 3))
    gv, _ = oracle.grid_update(cfg, gm, gmv, 0.0)
    idx = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3)
    floor = idx[:, 1] < 3
    assert np.all(gv[floor] == 0)
    inner = np.all((idx >= 3) & (idx <= n - 4), axis=1)
    assert np.array_equal(gv[inner], gmv[inner])
    for d in (0, 2):
        lo = (idx[:, d] < 3) & ~floor
        assert np.all(gv[lo, d] >= 0)
        side = lo & np.all((idx[:, [e for e in range(3) if e != d]] >= 3) & (idx[:, [e for e in range(3) if e != d]] <= n - 4), axis=1)
        assert np.array_equal(gv[side, d], np.maximum(gmv[side, d], 0))
        assert np.array_equal(gv[side][:, [e for e in range(3) if e != d]], gmv[side][:, [e for e in range(3) if e != d]])
    top = (idx[:, 1] > n - 4) & np.all((idx[:, [0, 2]] >= 3) & (idx[:, [0, 2]] <= n - 4), axis=1)
    assert np.array_equal(gv[top, 1], np.minimum(gmv[top, 1], 0))
    gm0 = gm.copy()
    gm0[::7] = 0
    gv0, _ = oracle.grid_update(cfg, gm0, gmv, 0.0)
    assert np.all(gv0[::7] == 0)


# ------------------------------------------------------------------- sort

def test_sort_by_brick_properties():
    n, N = 32, 5000
    x = np.random.default_rng(6).random((N, 3)).astype(np.float32) * 0.8 + 0.1
    key, perm, count = oracle.sort_by_brick(n, x)
    assert np.array_equal(np.sort(perm), np.arange(N))  # a permutation
    ks = key[perm]
    assert np.all(np.diff(ks) >= 0)  # sorted by key
    same = np.diff(ks) == 0
    assert np.all(np.diff(perm)[same] > 0)  # stable
    assert np.array_equal(count, np.bincount(key, minlength=(n // 4) ** 3))


def test_sort_key_closed_form_on_safe_points():
    # Points at (i + 1/4) dx have base cell i - 1 in exact arithmetic, far from
    # any rounding tie, so the brick is ((i-1)//4) per axis.
    n = 64
    g = np.random.default_rng(7)
    cells = g.integers(1, n - 2, size=(3000, 3))
    x = ((cells + 0.25) / n).astype(np.float32)
    key, _, _ = oracle.sort_by_brick(n, x)
    nb = n // 4
    b = (cells - 1) // 4
    assert np.array_equal(key, (b[:, 0] * nb + b[:, 1]) * nb + b[:, 2])


# ----------------------------------------------- plasticity inside the step

def _project_diagonal(eps, mu, ty):
    """Von Mises return map of a diagonal Hencky strain (the closed form of the
    reading used for plasticity): the deviator is scaled back to 2 mu |dev| = ty."""
    dev = eps - eps.mean()
    nrm = np.linalg.norm(dev)
    gamma = nrm - ty / (2 * mu)
    return eps - gamma * dev / nrm if gamma > 0 else eps


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
def test_plasticity_inside_step_uses_mu(model):
    # A whole substep with dt = 0, v = 0, C = 0 and no gravity moves no momentum
    # (Eq. 8 has no term left), so every node velocity is 0 and G2P leaves x, v,
    # C and F as they were, up to the plastic projection of F.  From a yielded
    # F = diag(exp(e)), tr e = 0, the step must return the diagonal closed form
    # with the particle's shear modulus: yield / (2 mu), not yield / (2 lambda).
    n, N = 32, 50
    mu, lam, ty = 10.0, 25.0, 2.0
    cfg = oracle.make_config(n, 1.0, 1e-5, model=model, plasticity=True, yield_stress=ty,
                             gravity=(0.0, 0.0, 0.0))
    e = np.array([0.3, -0.1, -0.2])
    st = oracle.State(_cloud(N, n, 0.4, 0.6), F=np.tile(np.diag(np.exp(e)), (N, 1, 1)), mu=mu, lam=lam)
    x0 = st.x.copy()
    assert oracle.run(cfg, st, 0.0, 1) == 0
    expect = np.diag(np.exp(_project_diagonal(e, mu, ty)))
    assert np.max(np.abs(st.F - expect)) < 1e-13
    assert np.max(np.abs(np.diag(np.exp(_project_diagonal(e, lam, ty))) - expect)) > 1e-2  # lambda would show
    assert np.array_equal(st.x, x0) and not st.v.any() and not st.C.any()


def test_plasticity_projects_the_updated_F():
    # V0 = 0 removes the stress force and g = 0, so the APIC transfers reproduce
    # the affine field v = a + A x, C = A exactly (Eq. 8, 9).  G2P then updates
    # F <- (I + dt C) F (Eq. 10) and projects that F.  With A and F diagonal the
    # whole step has a closed form; projecting before the update gives another F.
    n, N, dt = 32, 60, 1e-2
    mu, lam, ty = 10.0, 25.0, 2.0
    cfg = oracle.make_config(n, 1.0, 0.0, plasticity=True, yield_stress=ty, gravity=(0.0, 0.0, 0.0))
    a, Ad = np.array([0.1, -0.2, 0.05]), np.array([2.0, -3.0, 1.5])
    A = np.diag(Ad)
    e0 = np.array([0.3, -0.1, -0.2])
    x = _cloud(N, n, 0.45, 0.55)
    v = a + x @ A.T
    st = oracle.State(x, v, np.tile(A, (N, 1, 1)), np.tile(np.diag(np.exp(e0)), (N, 1, 1)), mu=mu, lam=lam)
    assert oracle.run(cfg, st, dt, 1) == 0
    expect = np.diag(np.exp(_project_diagonal(np.log(1 + dt * Ad) + e0, mu, ty)))
    assert np.max(np.abs(st.F - expect)) < 1e-10
    assert np.max(np.abs(st.v - v)) < 1e-12 and np.max(np.abs(st.C - A)) < 1e-10
    assert np.max(np.abs(st.x - (x + dt * v))) < 1e-13
    wrong_order = np.diag((1 + dt * Ad) * np.exp(_project_diagonal(e0, mu, ty)))
    assert np.max(np.abs(wrong_order - expect)) > 1e-3


# ------------------------------------------------------------------- loss

def test_loss_hand_worked():
    # Loss of the differentiable workload: squared distance of the particle
    # centroid to the target plus the mean squared particle speed, worked by
    # hand in binary fractions (tests/golden/loss_hand_worked.txt).
    parts, target, expect = [], None, None
    for line in open(os.path.join(GOLDEN, "loss_hand_worked.txt")):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "particle":
            parts.append([float(t) for t in f[1:]])
        elif f[0] == "target":
            target = [float(t) for t in f[1:]]
        elif f[0] == "loss":
            expect = float(f[1])
    parts = np.array(parts)
    assert oracle.loss(parts[:, :3], parts[:, 3:], target) == expect


# ------------------------------------------------------ paper's timing scene

def test_paper_timing_scene_constants():
    # Sec. III-D: 0.02 s per step, 10 substeps of dt = 0.002, 175,616 grid nodes
    # (tests/golden/paper_constants.txt); the workload of that scene uses them,
    # and its explicit step stays inside the CFL limit.
    kv = {}
    for line in open(os.path.join(GOLDEN, "paper_constants.txt")):
        f = line.split()
        if f and not f[0].startswith("#"):
            kv[f[0]] = float(f[1])
    sc = W.paper_timing_cube(N=4096, steps=1)
    assert sc["n"] ** 3 == kv["grid_nodes"] and sc["n"] == kv["grid_side"]
    assert sc["dt"] == kv["substep_dt"]
    assert sc["substeps"] == kv["substeps_per_step"]
    assert abs(sc["substeps"] * sc["dt"] - kv["step_seconds"]) < 1e-15
    mu, lam = oracle.lame(float(sc["E"][0]), float(sc["nu"][0]))
    c = math.sqrt((lam + 2 * mu) / sc["rho"])
    assert sc["dt"] * c * sc["n"] <= 0.3


# ----------------------------------------------------------- push-out

def test_push_out_sphere_closed_form():
    # Sec. IV-A particle correction: a point inside a sphere goes to the surface
    # point on the ray from the centre, c + R (x - c)/|x - c|; outside points stay.
    c, R = np.array([0.4, 0.5, 0.6]), 0.1
    r = oracle.make_rigid(W.sphere(tuple(c), R))
    g = np.random.default_rng(31)
    for _ in range(100):
        d = g.normal(size=3)
        d /= np.linalg.norm(d)
        rad = g.uniform(0.01, 0.2)
        x0 = c + rad * d
        x1, moved = oracle.push_out(r, x0)
        if rad < R:
            assert moved and np.max(np.abs(x1 - (c + R * d))) < 1e-15
        else:
            assert not moved and np.array_equal(x1, x0)


def test_push_out_box_nearest_face():
    # Inside a (rotated) box the nearest face is the one of largest q = |p| - h;
    # the point lands on that face: its body coordinate along the face normal
    # becomes +-h, the other two body coordinates are kept.
    q = np.array([0.9, 0.2, -0.3, 0.25])
    q /= np.linalg.norm(q)
    half = np.array([0.08, 0.05, 0.12])
    r = oracle.make_rigid(W.box((0.5, 0.45, 0.55), tuple(half), quat=tuple(q)))
    c, Rm = oracle.rigid_pose(r)
    g = np.random.default_rng(32)
    for _ in range(200):
        p = g.uniform(-1.3, 1.3, 3) * half
        x1, moved = oracle.push_out(r, c + Rm @ p)
        inside = np.all(np.abs(p) < half)
        assert moved == inside
        if inside:
            ax = int(np.argmax(np.abs(p) - half))
            p1 = Rm.T @ (x1 - c)
            expect = p.copy()
            expect[ax] = np.sign(p[ax]) * half[ax]
            assert np.max(np.abs(p1 - expect)) < 1e-13


def test_push_out_leaves_blades_and_segments():
    # Blades and line segments are crossed by the tissue by design (Sec. IV-B, IV-C).
    blade = oracle.make_rigid(W.quad_slicer((0.5, 0.5, 0.5), (1, 0, 0, 0), half_edge=0.1, half_depth=0.05,
                                            thickness=0.01))
    seg = oracle.make_rigid(W.segments((0.5, 0.5, 0.5), (1, 0, 0, 0), [[-0.1, 0, 0], [0.1, 0, 0]], radius=0.02))
    for r in (blade, seg):
        x1, moved = oracle.push_out(r, np.array([0.5, 0.5, 0.5]))
        assert not moved and np.array_equal(x1, [0.5, 0.5, 0.5])


def test_push_out_in_the_step_uses_the_moved_pose():
    # Particles resting inside a sphere that moves by dt * vel during the
    # substep end on the sphere's surface at its new centre (G2P, then the
    # kinematic advance, then the push-out); no node momentum changes for it.
    n, dt = 32, 1e-3
    cfg = oracle.make_config(n, 1.0, 1e-6, gravity=(0.0, 0.0, 0.0))
    c0, R, vel = np.array([0.5, 0.5, 0.5]), 0.08, np.array([0.3, -0.2, 0.1])
    rig = oracle.rigid_array([W.sphere(tuple(c0), R, vel=tuple(vel), mu_k=0.0, margin=0.0)])
    g = np.random.default_rng(33)
    d = g.normal(size=(40, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    x = c0 + d * g.uniform(0.02, 0.07, (40, 1))
    st = oracle.State(x, mu=0.0, lam=0.0)
    oracle.substep(cfg, st, dt, rig, 1)
    c1 = c0 + dt * vel
    assert np.max(np.abs(oracle.rigid_pose(rig[0])[0] - c1)) < 1e-15
    assert np.max(np.abs(np.linalg.norm(st.x - c1, axis=1) - R)) < 1e-13


# ------------------------------------------------------------ standard MPM

def test_bspline_derivative():
    # dN/dr of the quadratic basis (Sec. III-A: grad phi of Eq. 2 and Eq. 5)
    # against central differences of N; the basis is C1 (the difference is
    # O(h) only where the second derivative jumps, |r| = 0.5, 1.5).
    for r in np.linspace(-1.6, 1.6, 161):
        h = 1e-6
        fd = (oracle.bspline_N(r + h) - oracle.bspline_N(r - h)) / (2 * h)
        assert abs(oracle.bspline_dN(r) - fd) < 1e-6, r


def test_standard_g2p_affine_grid_field():
    # An affine grid velocity v_I = a + A x_I gives v_p = a + A x_p (Eq. 4) and
    # L = sum v_I grad phi^T = A (Eq. 5) at any particle position: partition of
    # unity and linear reproduction of the basis and of its gradient.
    n, N = 32, 300
    cfg = oracle.make_config(n, 1.0, 1e-5, gravity=(0.0, 0.0, 0.0))
    g = np.random.default_rng(41)
    a, A = g.normal(size=3), g.normal(size=(3, 3))
    I = np.stack(np.meshgrid(*[np.arange(n)] * 3, indexing="ij"), -1).reshape(-1, 3) / n
    gv = a + I @ A.T
    x = _cloud(N, n)
    st = oracle.State(x, mu=1.0, lam=1.0)
    assert oracle.g2p_standard(cfg, st, gv, 0.0) == 0
    assert np.max(np.abs(st.v - (a + x @ A.T))) < 1e-12
    assert np.max(np.abs(st.C - A)) < 1e-11


@pytest.mark.parametrize("model", ["fixed_corotated", "neo_hookean"])
def test_standard_force_is_the_energy_gradient(model):
    # The internal force of Eq. 2 is minus the gradient of the elastic energy
    # with respect to grid-node displacements: moving node I by delta_I deforms
    # each particle by F <- (I + sum delta_I grad phi_I^T) F (the F update of
    # Eq. 5 with v_I = delta_I / dt), and the P2G momentum of particles at rest
    # is dt f^int.  Central differences of the energy over a few nodes.
    n, N, dt = 16, 40, 1e-3
    V0, mu, lam = 2e-4, 30.0, 50.0
    cfg = oracle.make_config(n, 1.0, V0, model=model, gravity=(0.0, 0.0, 0.0))
    g = np.random.default_rng(42)
    x = _cloud(N, n, 0.4, 0.6)
    F0 = np.eye(3) + 0.1 * g.normal(size=(N, 3, 3))
    st = oracle.State(x, F=F0, mu=mu, lam=lam)
    gm, gmv, err = oracle.p2g_standard(cfg, st, dt)
    assert err == 0

    def energy(delta):
        s = oracle.State(x, F=F0, mu=mu, lam=lam)
        assert oracle.g2p_standard(cfg, s, delta / dt, dt) == 0
        return sum(V0 * _energy(model, Fp, mu, lam) for Fp in s.F)

    nodes = np.flatnonzero(gm)[:: max(1, len(np.flatnonzero(gm)) // 12)]
    h = 1e-7
    for I in nodes:
        for r in range(3):
            d = np.zeros((n ** 3, 3))
            d[I, r] = h
            fd = -(energy(d) - energy(-d)) / (2 * h)
            assert abs(gmv[I, r] / dt - fd) <= 1e-6 * max(1.0, abs(fd)), (I, r, gmv[I, r] / dt, fd)


def test_standard_free_fall_and_momentum():
    # Uniform velocity at rest shape: no force, the step adds dt g (Eq. 3, 4);
    # with no gravity, walls or rigids, a deformed block keeps its momentum.
    n, N, dt = 32, 300, 1e-3
    cfg = oracle.make_config(n, 1.0, 1e-5)
    v0 = np.array([0.2, 0.1, -0.3])
    st = oracle.State(_cloud(N, n, 0.4, 0.6), np.tile(v0, (N, 1)), mu=10.0, lam=10.0)
    x0 = st.x.copy()
    assert oracle.run_solver(cfg, st, dt, 1, "standard") == 0
    gvec = np.array(cfg.gravity[:])
    assert np.max(np.abs(st.v - (v0 + dt * gvec))) < 1e-12
    assert np.max(np.abs(st.x - (x0 + dt * (v0 + dt * gvec)))) < 1e-14
    cfg0 = oracle.make_config(n, 0.7, 1e-4, gravity=(0.0, 0.0, 0.0))
    g = np.random.default_rng(43)
    st = oracle.State(_cloud(N, n), g.normal(size=(N, 3)), F=np.eye(3) + 0.05 * g.normal(size=(N, 3, 3)),
                      mu=40.0, lam=60.0)
    P0 = st.v.sum(0)
    assert oracle.run_solver(cfg0, st, 2e-4, 3, "standard") == 0
    assert rel(st.v.sum(0), P0) < 1e-11


# ------------------------------------------------------------------ PB-MPM

def test_pb_constraint_limits():
    # Sec. III-C co-rotational constraint: with beta = 1 the corrected
    # deformation (I + dt C') F is the polar rotation of (I + dt C) F; with
    # beta = 0 it is (I + dt C) F / det((I + dt C) F); in between it is their
    # blend, so C' is affine in beta.
    from scipy.linalg import polar

    g = np.random.default_rng(44)
    dt = 0.02
    for _ in range(30):
        C = g.normal(size=(3, 3))
        F = np.eye(3) + 0.2 * g.normal(size=(3, 3))
        Fh = (np.eye(3) + dt * C) @ F
        if np.linalg.det(Fh) <= 0.1 or np.linalg.det(F) <= 0.1:
            continue
        R, _ = polar(Fh)
        c1 = oracle.pb_constraint(C, F, dt, 1.0)
        c0 = oracle.pb_constraint(C, F, dt, 0.0)
        assert np.max(np.abs((np.eye(3) + dt * c1) @ F - R)) < 1e-12
        assert np.max(np.abs((np.eye(3) + dt * c0) @ F - Fh / np.linalg.det(Fh))) < 1e-12
        b = g.uniform()
        assert np.max(np.abs(oracle.pb_constraint(C, F, dt, b) - (b * c1 + (1 - b) * c0))) < 1e-10


def test_pb_single_particle_step_closed_form():
    # One particle, no gravity, walls or rigids: the grid field of an APIC
    # transfer from a single particle is affine around it, so every G2P returns
    # the particle's velocity and the C the constraint produced (Eq. 8, 9).
    # With beta = 1 the constraint is idempotent, hence after any number of
    # cycles F_new = polar rotation of (I + dt C0) F and x moves by dt v.
    from scipy.linalg import polar

    n, dt = 32, 0.02
    cfg = oracle.make_config(n, 1.0, 1e-5, gravity=(0.0, 0.0, 0.0))
    g = np.random.default_rng(45)
    for iters in (1, 3, 10):
        C0, F0 = 2.0 * g.normal(size=(3, 3)), np.eye(3) + 0.1 * g.normal(size=(3, 3))
        v0, x0 = g.normal(size=3) * 0.1, np.array([0.47, 0.52, 0.49])
        st = oracle.State(x0[None], v0[None], C0[None], F0[None], mu=1.0, lam=1.0)
        assert oracle.run_solver(cfg, st, dt, 1, "pb", iters=iters, beta=1.0) == 0
        R, _ = polar((np.eye(3) + dt * C0) @ F0)
        assert np.max(np.abs(st.F[0] - R)) < 1e-11
        assert np.max(np.abs(st.v[0] - v0)) < 1e-13
        assert np.max(np.abs(st.x[0] - (x0 + dt * v0))) < 1e-14


def test_pb_gravity_enters_once_per_step():
    # At rest shape (F = I, C = 0) the constraint changes nothing, so a falling
    # cloud gains dt g per step whatever the number of cycles (reading: gravity
    # in the first cycle's node loop only).
    n, N, dt = 32, 200, 0.02
    cfg = oracle.make_config(n, 1.0, 1e-5)
    v0 = np.array([0.1, 0.0, -0.05])
    gvec = np.array(cfg.gravity[:])
    for iters in (1, 5):
        st = oracle.State(_cloud(N, n, 0.45, 0.55), np.tile(v0, (N, 1)), mu=1.0, lam=1.0)
        x0 = st.x.copy()
        assert oracle.run_solver(cfg, st, dt, 1, "pb", iters=iters, beta=0.5) == 0
        assert np.max(np.abs(st.v - (v0 + dt * gvec))) < 1e-12
        assert np.max(np.abs(st.x - (x0 + dt * (v0 + dt * gvec)))) < 1e-13
        assert np.max(np.abs(st.F - np.eye(3))) < 1e-12


# ------------------------------------------------- arc and mesh slicer

def test_arc_sdf_brute_force_and_tangent():
    # Sec. IV-C arc (suture needle): distance to the nearest point of the arc
    # against dense sampling of the arc; the tangent is the unit vector along
    # increasing angle at that point, perpendicular to its radius.
    q = np.array([0.9, 0.3, -0.2, 0.25])
    r = oracle.make_rigid(W.arc((0.5, 0.45, 0.55), tuple(q / np.linalg.norm(q)), arc_radius=0.06, start=0.4,
                                sweep=3.5, radius=0.003, margin=1.0))
    c, Rm = oracle.rigid_pose(r)
    th = 0.4 + np.linspace(0.0, 3.5, 200001)
    samples = c + (0.06 * np.stack([np.cos(th), np.sin(th), 0 * th], -1)) @ Rm.T
    g = np.random.default_rng(35)
    for _ in range(100):
        x = c + g.uniform(-0.12, 0.12, 3)
        code, n, t, d = oracle.geometry(r, x)
        ref = np.min(np.linalg.norm(samples - x, axis=1))
        assert abs(d - ref) < 1e-8, (d, ref)
        assert code == "oned"
        qpt = x - d * n  # the nearest point
        rad = Rm.T @ (qpt - c)
        assert abs(np.linalg.norm(rad[:2]) - 0.06) < 1e-12 and abs(rad[2]) < 1e-12
        assert abs(np.linalg.norm(t) - 1) < 1e-12 and abs(np.dot(t, qpt - c)) < 1e-12


def _flat_mesh(a, b):
    pts = [(-a, -b, 0.0), (a, -b, 0.0), (a, b, 0.0), (-a, b, 0.0)]
    return pts, [(0, 1, 2), (0, 2, 3)], [0, 1]


def test_flat_mesh_slicer_equals_quad_slicer():
    # A triangle-mesh slicer (Sec. IV-B) made of the quad's two triangles with
    # the spine along the quad's y = -b edge is the QuadSlicer (pinned against
    # brute-force sampling): same regions, distances and normals everywhere.
    a, b, h = 0.07, 0.04, 0.006
    q = np.array([0.8, -0.3, 0.4, 0.2])
    q = tuple(q / np.linalg.norm(q))
    kw = dict(thickness=h, spine_radius=0.004, margin=0.002)
    quad = oracle.make_rigid(W.quad_slicer((0.5, 0.5, 0.5), q, half_edge=a, half_depth=b, **kw))
    pts, tris, spine = _flat_mesh(a, b)
    mesh = oracle.make_rigid(W.mesh_slicer((0.5, 0.5, 0.5), q, pts, tris, spine, **kw))
    g = np.random.default_rng(36)
    seen = set()
    for _ in range(3000):
        x = 0.5 + g.uniform(-0.1, 0.1, 3) * np.array([1.0, 1.0, 0.15]) @ np.eye(3)
        cq, nq, _, dq = oracle.geometry(quad, x)
        cm, nm, _, dm = oracle.geometry(mesh, x)
        assert cq == cm
        seen.add(cq)
        assert abs(dq - dm) < 1e-13
        assert np.max(np.abs(nq - nm)) < 1e-12
    assert {"none", "regular", "sticky"} <= seen


def test_curved_mesh_slicer_brute_force():
    # Curved, jittered blade mesh: the distance used by the region test is the
    # distance to the nearest surface point (no sampled surface point is closer,
    # and the sampled minimum is within the sampling error), and the normal is
    # a unit vector from that point toward the query (face interiors: the
    # face normal, signed by side).
    pts, tris, spine = W.curved_blade_mesh()
    # no spine here (the wide margin would make every point sticky)
    r = oracle.make_rigid(W.mesh_slicer((0.5, 0.5, 0.5), (1, 0, 0, 0), pts, tris, [], thickness=0.004,
                                        spine_radius=0.002, margin=1.0))
    u = np.linspace(0, 1, 41)
    U, V = np.meshgrid(u, u, indexing="ij")
    keep = U + V <= 1
    U, V = U[keep], V[keep]
    samples = np.concatenate([pts[t0] + U[:, None] * (pts[t1] - pts[t0]) + V[:, None] * (pts[t2] - pts[t0])
                              for t0, t1, t2 in tris]) + 0.5
    g = np.random.default_rng(37)
    n_regular = 0
    for _ in range(150):
        x = 0.5 + g.uniform(-1, 1, 3) * np.array([0.1, 0.05, 0.04])
        code, n, _, d = oracle.geometry(r, x)
        if code != "regular":
            continue
        n_regular += 1
        dist = np.linalg.norm(samples - x, axis=1)
        assert d <= dist.min() + 1e-12
        assert dist.min() - d < 2e-5  # sampling error of a 40 x 40 barycentric grid
        assert abs(np.linalg.norm(n) - 1) < 1e-12
        qpt = x - d * n  # lies on the mesh, at distance d
        assert np.linalg.norm(samples - qpt, axis=1).min() < 3e-3
    assert n_regular > 100
