"""Pins of the oracle's power (Sec. 3.5, Eq. insect_power) and free flight
(Sec. 3.6, Eq. oh_my_god_look_a_vector): quaternion and yaw-pitch-roll
frames agree, rigid rotation at a constant body rate, free fall with the AB2
start-up error in closed form, a body held by its dof mask is the tethered
run, the wing's angular acceleration is the derivative of its rate, and the
aerodynamic power is minus the penalization force times the wing's own velocity."""
import math

import numpy as np
import pytest

import workloads


def test_quaternion_frame_is_the_yaw_pitch_roll_frame(orc):
    for psi, beta, gamma in ((0.3, -0.5, 0.7), (1.2, 0.4, -2.0), (0.0, 0.0, 0.0)):
        ins = {"body": "ellipsoid", "body_axes": (0.5, 0.12), "x_cntr": (1, 1, 1),
               "body_angles": (psi, beta, gamma)}
        tethered = orc.frames(ins, 0.0)["M_body"]
        free = dict(ins, free_flight={"mass": 1.0, "J_body": (1.0, 1.0, 1.0)})
        assert np.abs(orc.frames(free, 0.0)["M_body"] - tethered).max() <= 1e-15
        q = orc.quat_from_angles(psi, beta, gamma)
        assert abs(np.linalg.norm(q) - 1.0) <= 1e-15


def test_constant_body_rate_is_a_rigid_rotation(orc):
    """With no moments and equal principal moments, Omega^(b) stays constant
    and the body-to-global map evolves as R(t) = R(0) exp(t [Omega]x); the
    quaternion right-hand side integrated by a high-order method reproduces it."""
    from scipy.integrate import solve_ivp
    from scipy.linalg import expm
    W = np.array([0.7, -1.1, 0.4])
    ins = {"body": "ellipsoid", "body_axes": (0.5, 0.12), "x_cntr": (1, 1, 1),
           "body_angles": (0.3, -0.2, 0.5),
           "free_flight": {"mass": 1.0, "J_body": (2.0, 2.0, 2.0), "Omega_body": tuple(W)}}
    q0 = orc.quat_from_angles(0.3, -0.2, 0.5)

    def F(t, y):
        return orc.body_rhs(ins, (0, 0, 0), (0, 0, 0), (y[0:3], y[3:6], y[6:10], y[10:13]))

    y0 = np.concatenate([[1, 1, 1], [0, 0, 0], q0, W])
    T = 1.3
    sol = solve_ivp(F, (0, T), y0, method="DOP853", rtol=1e-12, atol=1e-13)
    yT = sol.y[:, -1]
    assert np.abs(yT[10:13] - W).max() <= 1e-12
    R0 = orc.frames(ins, 0.0)["M_body"].T
    K = np.array([[0, -W[2], W[1]], [W[2], 0, -W[0]], [-W[1], W[0], 0]])
    Rt = R0 @ expm(T * K)
    # the frame of the integrated quaternion (make_insect starts it from the angles)
    import ctypes as C
    m = orc.make_insect(ins)
    m.quat[:] = list(yT[6:10] / np.linalg.norm(yT[6:10]))
    frs = orc.Frames()
    orc.lib().orc_frames_at(C.byref(m), 0.0, C.byref(frs))
    M_T = np.array(frs.M_body[:]).reshape(3, 3)
    assert np.abs(M_T.T - Rt).max() <= 1e-9


def _invisible_body(L, n, **ff):
    """A body too small to touch a grid point: chi = 0 everywhere, so the
    aerodynamic force and moment vanish exactly."""
    d = L[0] / n[0]
    return {"body": "sphere", "nwings": 0, "profile": "cos", "c_smth": 0.1,
            "body_axes": (1e-6, 0.0), "x_cntr": (2.0 + 0.5 * d, 2.0 + 0.5 * d, 2.0 + 0.5 * d),
            "free_flight": ff}


def test_free_fall_with_the_ab2_start(orc):
    """Gravity only: u_z = -g t exactly; the Euler start leaves z one
    g dt^2/2 above z0 - g t^2/2 for every later step."""
    n, L = (8, 8, 8), (4.0, 4.0, 4.0)
    g, dt = 9.81, 2e-3
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "dt_fixed": dt, "mean_mode": "fixed"}
    ins = _invisible_body(L, n, mass=0.7, gravity=g, J_body=(1.0, 1.0, 1.0))
    sim = orc.Simulation(cfg, ins)
    sim.set_state(np.zeros((3,) + n[::-1]))
    z0 = ins["x_cntr"][2]
    rows = sim.step(12)
    assert np.abs(rows[:, 2:20]).max() == 0.0
    t = 12 * dt
    assert abs(sim.ins.u_cntr[2] + g * t) <= 1e-13
    assert abs(sim.ins.x_cntr[2] - (z0 - 0.5 * g * t * t + 0.5 * g * dt * dt)) <= 1e-13
    assert sim.ins.x_cntr[0] == ins["x_cntr"][0] and sim.ins.u_cntr[0] == 0.0


def test_dof_mask_holds_the_body_as_tethered(orc):
    cfg, ins = workloads.config_model_insect(24)
    cfg = dict(cfg, n=(24, 24, 24))
    ins = workloads.model_insect(cfg["L"], cfg["n"])
    u0 = workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"])
    a = orc.Simulation(cfg, ins)
    a.set_state(u0)
    ra = a.step(4)
    held = dict(ins, free_flight={"mass": 0.1, "gravity": 9.81, "J_body": (1e-3, 2e-3, 2e-3),
                                  "dof": (0, 0, 0, 0, 0, 0)})
    b = orc.Simulation(cfg, held)
    b.set_state(u0)
    rb = b.step(4)
    assert np.array_equal(ra, rb)
    assert np.array_equal(a.get_state(), b.get_state())
    assert tuple(b.ins.x_cntr) == tuple(ins["x_cntr"])


def test_wing_angular_acceleration_is_the_rate_derivative(orc):
    ins = workloads.model_insect((4.0, 4.0, 4.0), (32, 32, 32))
    ins["kinematics"]["theta"] = (0.1, [0.2], [0.15])
    for t in (0.05, 0.31, 0.77):
        eps = 1e-5
        fp, fm = orc.frames(ins, t + eps), orc.frames(ins, t - eps)
        fr = orc.frames(ins, t)
        for s in range(2):
            fd = (fp["Omega_w_w"][s] - fm["Omega_w_w"][s]) / (2 * eps)
            assert np.abs(fr["dOmega_w_w"][s] - fd).max() <= 1e-6 * max(1.0, np.abs(fd).max())


def test_aerodynamic_power_is_force_times_wing_velocity(orc):
    """-m . Omega_rel = -sum_x f . (Omega_rel x (x - pivot)) with the penalization
    force density f = chi (u - u_s)/C_eta of the wing's points (first step: no
    unsteady correction)."""
    cfg, _ = workloads.config_model_insect(32)
    ins = workloads.model_insect(cfg["L"], cfg["n"])
    ins["J_wing"] = (1e-3, 2e-4, 1.2e-3, 1e-5, 0.0, 0.0)
    u0 = workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"])
    sim = orc.Simulation(cfg, ins)
    sim.set_state(u0)
    f = orc.Spectral(cfg).physical_fields(sim.uh, 0.0, ins)
    rows = sim.step(1)
    fr = orc.frames(ins, 0.0)
    n = cfg["n"][0]
    L = cfg["L"][0]
    dV = (L / n) ** 3
    x = np.arange(n) * L / n
    Z, Y, X = np.meshgrid(x, x, x, indexing="ij")
    for s, col in ((0, 2), (1, 3)):
        w = fr["M_body"].T @ fr["Omega_w_b"][s]
        p = fr["pivot_g"][s]
        sel = f[7] == col
        r = np.stack([X - p[0], Y - p[1], Z - p[2]])
        urel = np.cross(w, r, axis=0)
        dens = f[6] * (f[0:3] - f[8:11]) / cfg["eta"]
        expect = -(dens * urel)[:, sel].sum() * dV
        assert rows[0, 22 + s] == pytest.approx(expect, rel=1e-10, abs=1e-12)
    assert abs(rows[0, 22]) > 1e-6


def test_inertial_power_is_the_rate_of_rotational_energy(orc):
    """With J constant in the wing frame, Omega . (J Omega' + Omega x J Omega)
    = d/dt (Omega . J Omega / 2): the central difference of that energy, and a
    zero average over one stroke."""
    ins = workloads.model_insect((4.0, 4.0, 4.0), (32, 32, 32))
    ins["kinematics"]["theta"] = (0.1, [0.2], [0.15])
    J6 = (1e-3, 2e-4, 1.2e-3, 1e-5, -2e-5, 3e-5)
    ins["J_wing"] = J6
    J = np.array([[J6[0], J6[3], J6[4]], [J6[3], J6[1], J6[5]], [J6[4], J6[5], J6[2]]])

    def energy(t, s):
        w = orc.frames(ins, t)["Omega_w_w"][s]
        return 0.5 * w @ J @ w

    for t in (0.05, 0.42, 0.9):
        _, pin = orc.wing_power(ins, t)
        for s in range(2):
            eps = 1e-5
            fd = (energy(t + eps, s) - energy(t - eps, s)) / (2 * eps)
            assert pin[s] == pytest.approx(fd, rel=1e-6, abs=1e-9)
    ts = np.arange(400) / 400
    avg = np.mean([orc.wing_power(ins, t)[1] for t in ts], axis=0)
    peak = max(abs(orc.wing_power(ins, t)[1]).max() for t in ts[::20])
    assert np.abs(avg).max() <= 1e-12 * max(1.0, peak) + 1e-15
