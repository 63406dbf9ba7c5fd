"""Pins of the oracle's insect module (Sec. 3): rotation conventions against
scipy's independent rotation library, orthonormality, the smoothed mask
(Eq. smoothing_mask_as_function_of_delta), volumes, the first force row, the
solid velocity against finite differences of material-point positions, and
the left/right mirror symmetry."""
import math

import numpy as np
import pytest

import workloads

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation
DEG = math.pi / 180


@pytest.mark.parametrize("xi", [0.3, -1.1, 2.5])
def test_rotation_matrices_are_passive(orc, xi):
    for ax in "xyz":
        ref = Rotation.from_euler(ax, xi).as_matrix().T
        assert np.allclose(orc.rot(ax, xi), ref, atol=1e-15)


def test_body_matrix_yaw_pitch_roll(orc):
    """M_body = R_x(psi) R_y(beta) R_z(gamma): yaw first, then pitch, then roll
    (Eq. M_body_yawpitchroll) -- the transpose of scipy's intrinsic Z-Y-X."""
    ins = workloads.model_insect()
    psi, beta, gamma = 0.2, -0.7, 1.1
    ins["body_angles"] = (psi, beta, gamma)
    fr = orc.frames(ins, 0.0)
    ref = Rotation.from_euler("ZYX", [gamma, beta, psi]).as_matrix().T
    assert np.allclose(fr["M_body"], ref, atol=1e-15)


@pytest.mark.parametrize("t", [0.0, 0.13, 0.61])
def test_frames_orthonormal(orc, t):
    ins = workloads.model_insect()
    ins["body_angles"] = (0.1, -0.3, 0.7)
    ins["kinematics"]["theta"] = (0.1, [0.05], [0.2])
    fr = orc.frames(ins, t)
    mats = [fr["M_body"]] + fr["M_stroke"] + fr["M_wing"]
    for M in mats:
        assert np.allclose(M @ M.T, np.eye(3), atol=1e-15)
        assert abs(np.linalg.det(M) - 1.0) <= 1e-14


def test_kinematic_angles_follow_their_series(orc):
    ins = workloads.single_wing()
    fr = orc.frames(ins, 0.3)
    phi, alpha, theta = fr["angles"]
    assert abs(phi - 60 * DEG * math.sin(2 * math.pi * 0.3)) <= 1e-15
    assert abs(alpha - 45 * DEG * math.cos(2 * math.pi * 0.3)) <= 1e-15
    assert theta == 0.0


@pytest.mark.parametrize("profile", ["cos", "tanh"])
def test_mask_profile(orc, profile):
    h = 0.07
    assert orc.mask_profile(profile, 0.0, h) == pytest.approx(0.5, abs=1e-16)
    for d in np.linspace(-2 * h, 2 * h, 17):
        s = orc.mask_profile(profile, d, h) + orc.mask_profile(profile, -d, h)
        assert abs(s - 1.0) <= 1e-15
    xs = [orc.mask_profile(profile, d, h) for d in np.linspace(-3 * h, 3 * h, 50)]
    assert all(a >= b for a, b in zip(xs, xs[1:]))
    if profile == "cos":
        assert orc.mask_profile(profile, -h, h) == 1.0
        assert orc.mask_profile(profile, h, h) == 0.0
        assert orc.mask_profile(profile, -1.01 * h, h) == 1.0
        assert orc.mask_profile(profile, 1.01 * h, h) == 0.0
    else:
        # tanh layer: 0.88 -> 0.12 across delta in [-h, h]
        assert orc.mask_profile(profile, -h, h) == pytest.approx(0.5 * (1 + math.tanh(1)))


def test_sphere_volume_converges(orc):
    r = 0.8
    errs = []
    for n in (24, 48):
        cfg = {"n": (n, n, n), "L": (4.0, 4.0, 4.0), "nu": 0.0, "eta": 1.0}
        ins = workloads.sphere((2.0, 2.0, 2.0), r, profile="cos")
        chi, col, us = orc.mask_grid(cfg, ins, 0.0)
        vol = chi.sum() * (4.0 / n) ** 3
        errs.append(abs(vol - 4 / 3 * math.pi * r ** 3) / (4 / 3 * math.pi * r ** 3))
        assert set(np.unique(col)) <= {0, 1}
    # the smoothing layer's curvature error is O(h^2): about 4x per halving
    assert errs[0] / errs[1] > 3.0 and errs[1] < 1e-2


def test_plate_volume_converges(orc):
    """A plate at rest (all angles zero) covers chord x span x thickness in the
    limit of a thin smoothing layer."""
    errs = []
    for n in (48, 96):
        cfg = {"n": (n, n, n), "L": (4.0, 4.0, 4.0), "nu": 0.0, "eta": 1.0}
        ins = workloads.single_wing(cfg["L"], cfg["n"])
        ins["wing"] = (0.15, 0.15, 1.0, 0.25)
        ins["kinematics"] = {"phi": (0.0, [], []), "alpha": (0.0, [], []),
                             "theta": (0.0, [], [])}
        chi, col, us = orc.mask_grid(cfg, ins, 0.0)
        vol = chi.sum() * (4.0 / n) ** 3
        errs.append(abs(vol - 0.3 * 1.0 * 0.25) / 0.075)
        assert np.all(us == 0)
        assert set(np.unique(col)) == {0, 2}
    assert errs[0] / errs[1] > 2.0 and errs[1] < 0.04


def test_first_force_row_uniform_flow(orc):
    """Unit-speed uniform u past a fixed mask: the first force row is
    u sum chi dV / C_eta (Eq. force_with_unst_corrections, no correction)."""
    n, eta = 16, 0.02
    cfg = {"n": (n, n, n), "L": (4.0, 4.0, 4.0), "nu": 0.01, "eta": eta, "dt_fixed": 1e-3,
           "mean_mode": "fixed", "u_inf": (0.6, 0.0, 0.8)}
    ins = workloads.sphere((2.0, 2.0, 2.0), 0.7, profile="cos")
    sim = orc.Simulation(cfg, ins)
    sim.set_state(workloads.uniform(cfg["n"], (0.6, 0.0, 0.8)))
    row = sim.step(1)[0]
    chi, _, _ = orc.mask_grid(cfg, ins, 0.0)
    expect = np.array([0.6, 0.0, 0.8]) * chi.sum() * (4.0 / n) ** 3 / eta
    assert np.allclose(row[2:5], expect, rtol=1e-12, atol=1e-12)
    # symmetric body about its centre: no moment
    assert np.abs(row[5:8]).max() <= 1e-10 * np.abs(expect).max()


def _global_point(orc, ins, t, side, xw):
    fr = orc.frames(ins, t)
    pb = np.array(ins["pivot_l"] if side == 0 else ins["pivot_r"])
    xb = fr["M_stroke"][side].T @ (fr["M_wing"][side].T @ np.asarray(xw)) + pb
    return np.array(ins["x_cntr"]) + fr["M_body"].T @ xb


def _moved(ins, eps):
    """The descriptor advanced by eps along its body rates and centre velocity."""
    d = dict(ins)
    ang, rate = np.array(ins["body_angles"]), np.array(ins["body_rates"])
    d["body_angles"] = tuple(ang + eps * rate)
    d["x_cntr"] = tuple(np.array(ins["x_cntr"]) + eps * np.array(ins["u_cntr"]))
    return d


@pytest.mark.parametrize("side,t", [(0, 0.11), (1, 0.11), (0, 0.47), (1, 0.83)])
def test_solid_velocity_is_rate_of_position(orc, side, t):
    """u_s at a wing point equals d/dt of that material point's global position
    X(t) = x_cntr + M_body^-1 (M_stroke^-1 M_wing(t)^-1 x^(w) + x_pivot),
    by central differences -- an independent check of the nested angular
    velocities of Sec. 3.1 and Sec. 3.3 and of Eq. wing_velocity_field."""
    ins = workloads.model_insect()
    ins["body_angles"] = (0.2, -0.4, 0.3)
    ins["body_rates"] = (0.7, -1.3, 0.9)
    ins["u_cntr"] = (0.1, -0.2, 0.3)
    ins["kinematics"]["theta"] = (0.1, [0.15], [0.2])
    xw = (0.02, 0.55, 0.0)
    eps = 1e-5
    X = _global_point(orc, ins, t, side, xw)
    Xp = _global_point(orc, _moved(ins, eps), t + eps, side, xw)
    Xm = _global_point(orc, _moved(ins, -eps), t - eps, side, xw)
    vel = (Xp - Xm) / (2 * eps)
    chi, col, us = orc.solid_at(ins, t, 0.01, X)
    assert chi == 1.0 and col == 2 + side
    assert np.abs(us - vel).max() <= 1e-8 * max(1.0, np.abs(vel).max())


def test_body_velocity_is_rate_of_position(orc):
    ins = workloads.model_insect()
    ins["nwings"] = 0
    ins["body_angles"] = (0.2, -0.4, 0.3)
    ins["body_rates"] = (0.7, -1.3, 0.9)
    ins["u_cntr"] = (0.1, -0.2, 0.3)
    xb = np.array([0.3, 0.02, -0.01])
    eps = 1e-5
    pos = lambda d: np.array(d["x_cntr"]) + orc.frames(d, 0.0)["M_body"].T @ xb
    vel = (pos(_moved(ins, eps)) - pos(_moved(ins, -eps))) / (2 * eps)
    chi, col, us = orc.solid_at(ins, 0.0, 0.01, pos(ins))
    assert chi == 1.0 and col == 1
    assert np.abs(us - vel).max() <= 1e-8


def test_wings_are_mirror_images(orc):
    """With the body frame aligned with the global frame, the right wing is the
    left wing reflected in the plane y = y_cntr (Sec. 3.3 mirror matrices)."""
    n = 32
    cfg = {"n": (n, n, n), "L": (4.0, 4.0, 4.0), "nu": 0.0, "eta": 1.0}
    ins = workloads.model_insect(cfg["L"], cfg["n"])
    chi, col, us = orc.mask_grid(cfg, ins, 0.17)
    mirror = lambda a: np.roll(a[:, ::-1, :], 1, axis=1)   # y_j -> y_{n-j}
    assert np.allclose(chi, mirror(chi), atol=1e-14)
    cm = mirror(col)
    swapped = np.where(cm == 2, 3, np.where(cm == 3, 2, cm))
    wing = (col >= 2) & (chi > 1e-9)
    wing[:, n // 2, :] = False   # on the mirror plane both wings tie up to rounding
    assert np.array_equal(col[wing], swapped[wing])
    off = np.ones_like(chi, bool)
    off[:, n // 2, :] = False
    assert np.allclose(us[0][off], mirror(us[0])[off], atol=1e-13)
    assert np.allclose(us[1][off], -mirror(us[1])[off], atol=1e-13)
    assert np.allclose(us[2][off], mirror(us[2])[off], atol=1e-13)
    assert (col == 2).any() and (col == 3).any() and (col == 1).any()


def test_thorax_surface_and_volume(orc):
    """The thorax signed distance vanishes on the ellipsoid (a, b, b) and the
    smoothed mask integrates to its volume 4/3 pi a b^2."""
    ins = workloads.model_insect()
    ins["nwings"] = 0
    c = np.array(ins["x_cntr"])
    a, b = ins["body_axes"]
    h = 0.01
    for p in ([a, 0, 0], [-a, 0, 0], [0, b, 0], [0, 0, -b],
              [0.6 * a, 0.8 * b / math.sqrt(2), 0.8 * b / math.sqrt(2)]):
        chi, col, _ = orc.solid_at(ins, 0.0, h, c + np.array(p))
        assert abs(chi - 0.5) <= 1e-9 and col == 1
    chi, _, _ = orc.solid_at(ins, 0.0, h, c + np.array([a + 2 * h, 0, 0]))
    assert chi == 0.0
    errs = []
    for n in (48, 96):
        cfg = {"n": (n, n, n), "L": (2.0, 2.0, 2.0), "nu": 0.0, "eta": 1.0}
        body = dict(ins, x_cntr=(1.0, 1.0, 1.0))
        m, _, _ = orc.mask_grid(cfg, body, 0.0)
        vol = m.sum() * (2.0 / n) ** 3
        errs.append(abs(vol - 4 / 3 * math.pi * a * b * b) / (4 / 3 * math.pi * a * b * b))
    assert errs[1] < errs[0] and errs[1] < 0.02


def test_unsteady_force_correction(orc):
    """With a vanishing penalization (huge C_eta) the force row is the
    unsteady correction alone: (sum chi u_s dV at t_n - at t_{n-1}) / dt_{n-1},
    zero on the first step (Eq. force_with_unst_corrections, backward
    difference)."""
    n, dt = 24, 0.01
    cfg = {"n": (n, n, n), "L": (4.0, 4.0, 4.0), "nu": 0.01, "eta": 1e30, "dt_fixed": dt,
           "mean_mode": "fixed"}
    ins = workloads.single_wing(cfg["L"], cfg["n"])
    sim = orc.Simulation(cfg, ins)
    sim.set_state(workloads.uniform(cfg["n"], (0.0, 0.0, 0.0)))
    rows = sim.step(3)
    dV = (4.0 / n) ** 3
    Is = []
    for k in range(3):
        chi, col, us = orc.mask_grid(cfg, ins, k * dt)
        Is.append(np.array([np.sum(us[c] * chi * (col == 2)) * dV for c in range(3)]))
    assert np.abs(rows[0, 8:11]).max() <= 1e-20   # colour 2 block starts at column 8
    for k in (1, 2):
        expect = (Is[k] - Is[k - 1]) / dt
        assert np.allclose(rows[k, 8:11], expect, rtol=1e-10, atol=1e-14)
        assert np.abs(expect).max() > 1e-4
