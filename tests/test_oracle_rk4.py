"""Pins of the oracle's RK4 scheme with explicit diffusion (Sec. 2.4 names it
as the alternative time integrator): exact amplification factors of the two
linear cases, fourth-order convergence with a fixed mask, agreement with an
independent high-order integration of the same semi-discrete system when the
mask moves (which fixes the stage times), and the explicit-diffusion step limit."""
import math

import numpy as np
import pytest

import workloads


def _R(z):
    """RK4 amplification factor for y' = -y/tau, z = dt/tau."""
    return 1 - z + z * z / 2 - z ** 3 / 6 + z ** 4 / 24


def test_viscous_decay_amplification(orc):
    """u = (0, a sin kx, 0): the Lamb vector is a gradient, so du/dt = -nu k^2 u
    and every step multiplies u by R(nu k^2 dt)."""
    n, L = (16, 8, 8), (2.0, 1.0, 1.0)
    nu, dt = 0.05, 2e-3
    cfg = {"n": n, "L": L, "nu": nu, "eta": 1.0, "dt_fixed": dt, "mean_mode": "fixed",
           "time_scheme": "rk4"}
    k = 2 * math.pi * 3 / L[0]
    x = np.arange(n[0]) * L[0] / n[0]
    u0 = np.zeros((3, n[2], n[1], n[0]))
    u0[1] = 0.8 * np.sin(k * x)[None, None, :]
    sim = orc.Simulation(cfg, None)
    sim.set_state(u0)
    sim.step(12)
    assert np.abs(sim.get_state() - _R(nu * k * k * dt) ** 12 * u0).max() <= 1e-14


def test_relaxation_amplification(orc):
    """chi = 1 everywhere, u_s = 0, uniform u, free mean, nu = 0: du/dt = -u/C_eta."""
    eta, dt = 0.05, 0.004
    cfg = {"n": (8, 8, 8), "L": (2 * math.pi,) * 3, "nu": 0.0, "eta": eta, "dt_fixed": dt,
           "mean_mode": "free", "time_scheme": "rk4"}
    ins = workloads.sphere((0.0, 0.0, 0.0), 100.0, profile="cos")
    u0 = np.array([0.3, -0.2, 0.5])
    sim = orc.Simulation(cfg, ins)
    sim.set_state(workloads.uniform(cfg["n"], u0))
    rows = sim.step(10)
    got = sim.get_state().mean(axis=(1, 2, 3))
    assert np.abs(got - _R(dt / eta) ** 10 * u0).max() <= 1e-14
    # the force row is taken at the start of each step
    vol = (2 * math.pi) ** 3
    assert np.allclose(rows[3, 2:5], _R(dt / eta) ** 3 * u0 * vol / eta, rtol=1e-12)


def test_fourth_order_with_a_fixed_sphere(orc):
    cfg, ins = workloads.config_tg_sphere(16)
    cfg = {k: v for k, v in cfg.items() if k != "dt_fixed"}
    cfg["time_scheme"] = "rk4"
    u0 = workloads.initial_field(cfg)
    res = []
    for dt in (0.008, 0.004, 0.002):
        sim = orc.Simulation(dict(cfg, dt_fixed=dt), ins)
        sim.set_state(u0)
        sim.step(int(round(0.08 / dt)))
        res.append(sim.get_state())
    d0, d1 = np.linalg.norm(res[0] - res[1]), np.linalg.norm(res[1] - res[2])
    assert 13.0 < d0 / d1 < 20.0


@pytest.mark.slow
def test_moving_wing_matches_independent_integration(orc):
    """A flapping plate (tanh layer) on 8^3: the oracle's RK4 against scipy's
    DOP853 on the same semi-discrete system du/dt = N(u, t) - nu k^2 u, whose
    right-hand side evaluates the mask at the time it is asked for.  Stages
    taken at the wrong times give errors of order dt (about 1e-3 here)."""
    from scipy.integrate import solve_ivp
    n, L = (8, 8, 8), (4.0, 4.0, 4.0)
    cfg = {"n": n, "L": L, "nu": 0.02, "eta": 2.5e-2, "mean_mode": "fixed", "time_scheme": "rk4"}
    ins = dict(workloads.single_wing(L, n), profile="tanh")
    sp = orc.Spectral(cfg)
    u0 = workloads.random_smooth_field(n, 3, amplitude=0.2)
    sim = orc.Simulation(dict(cfg, dt_fixed=1e-3), ins)
    sim.set_state(u0)
    uh0 = sim.uh.copy()
    hx = n[0] // 2 + 1
    kx = 2 * np.pi * np.arange(hx) / L[0]
    ky = 2 * np.pi * np.fft.fftfreq(n[1], 1 / n[1]) / L[1]
    kz = 2 * np.pi * np.fft.fftfreq(n[2], 1 / n[2]) / L[2]
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    K2 = KX ** 2 + KY ** 2 + KZ ** 2

    def F(t, y):
        uh = y.view(np.complex128).reshape(uh0.shape)
        nh, _ = sp.rhs(uh, t, ins)
        return (nh - cfg["nu"] * K2[None] * uh).reshape(-1).view(np.float64)

    T = 0.02
    ref = solve_ivp(F, (0, T), uh0.reshape(-1).view(np.float64).copy(), method="DOP853",
                    rtol=1e-11, atol=1e-13)
    uref = ref.y[:, -1].view(np.complex128).reshape(uh0.shape)
    errs = []
    for dt in (0.004, 0.002):
        s = orc.Simulation(dict(cfg, dt_fixed=dt), ins)
        s.set_state(u0)
        s.step(int(round(T / dt)))
        errs.append(np.abs(s.uh - uref).max())
    assert errs[0] <= 1e-5 and errs[1] <= 2e-6 and errs[0] / errs[1] > 3.5


def test_explicit_diffusion_limits_the_step(orc):
    n, L = (12, 12, 12), (1.0, 1.0, 1.0)
    nu = 0.5
    cfg = {"n": n, "L": L, "nu": nu, "eta": 1.0, "cfl": 0.1, "mean_mode": "fixed",
           "time_scheme": "rk4"}
    sim = orc.Simulation(cfg, None)
    sim.set_state(workloads.random_smooth_field(n, 5, amplitude=0.01))
    rows = sim.step(1)
    k2max = 3 * (2 * math.pi * 4 / 1.0) ** 2
    assert rows[0, 1] == pytest.approx(2.5 / (nu * k2max), rel=1e-14)
