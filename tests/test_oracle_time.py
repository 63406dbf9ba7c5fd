"""Pins of the oracle's time stepping (Algorithm 1 steps b-e; AB2 with an
integrating factor, Sec. 2.4) and of its penalization term (Eq.
PNST_org_momentum), each against a closed form the method fixes."""
import math

import numpy as np
import pytest

import workloads


def _free_cfg(n, **kw):
    c = {"n": n, "L": (2 * math.pi,) * 3, "nu": 0.0, "eta": 1.0, "mean_mode": "free"}
    c.update(kw)
    return c


def _weights(nx, nxh):
    w = np.full(nxh, 2.0)
    w[0] = 1.0
    if nx % 2 == 0:
        w[nx // 2] = 1.0
    return w


# ---------------------------------------------------------------- P5 relaxation

def _solid_box():
    """A sphere much larger than the box: chi = 1 at every grid point."""
    return workloads.sphere((0.0, 0.0, 0.0), 100.0, profile="cos")


def test_penalization_relaxation_recurrence(orc):
    """Inside the solid, d_t u = -u/C_eta (Sec. 2.1).  With chi = 1 and u_s = 0
    a uniform u is a pure k = 0 mode and the scheme must reproduce the AB2
    recurrence u1 = u0 (1 - dt/eta), u_{n+1} = u_n - dt/eta (1.5 u_n - 0.5 u_{n-1})."""
    eta, dt = 0.05, 0.004
    cfg = _free_cfg((8, 8, 8), nu=0.01, eta=eta, dt_fixed=dt)
    u0 = np.array([0.3, -0.2, 0.5])
    sim = orc.Simulation(cfg, _solid_box())
    sim.set_state(workloads.uniform(cfg["n"], u0))
    rows = sim.step(10)
    hist = [u0, u0 * (1 - dt / eta)]
    for _ in range(9):
        hist.append(hist[-1] - dt / eta * (1.5 * hist[-1] - 0.5 * hist[-2]))
    got = sim.get_state().mean(axis=(1, 2, 3))
    assert np.abs(got - hist[10]).max() <= 1e-14
    # force on the solid: sum chi (u - u_s) dV / C_eta over the whole box
    vol = (2 * math.pi) ** 3
    assert np.allclose(rows[0, 2:5], u0 * vol / eta, rtol=1e-13)
    assert np.allclose(rows[3, 2:5], hist[3] * vol / eta, rtol=1e-12)


def test_penalization_relaxation_second_order(orc):
    eta, T = 0.05, 0.1
    errs = []
    for dt in (0.004, 0.002, 0.001):
        cfg = _free_cfg((8, 8, 8), nu=0.0, eta=eta, dt_fixed=dt)
        sim = orc.Simulation(cfg, _solid_box())
        sim.set_state(workloads.uniform(cfg["n"], (1.0, 0.0, 0.0)))
        sim.step(int(round(T / dt)))
        errs.append(abs(sim.get_state()[0].mean() - math.exp(-T / eta)))
    assert 3.6 < errs[0] / errs[1] < 4.4
    assert 3.6 < errs[1] / errs[2] < 4.4


# -------------------------------------------------------------- P6 IF-AB2 form

def test_ab2_exact_for_linear_forcing(orc):
    """At nu = 0 AB2 integrates N(t) = a + b t exactly for any step sequence
    after the Euler start, whose local error b dt0^2/2 is carried along."""
    cfg = _free_cfg((8, 6, 4), nu=0.0)
    sp = orc.Spectral(cfg)
    rng = np.random.default_rng(4)
    shp = sp.shape()
    u0 = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    a = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    b = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    dts = [0.1, 0.13, 0.07, 0.11, 0.05, 0.09, 0.12]
    u, t, prev = u0.copy(), 0.0, None
    for n, dt in enumerate(dts):
        nh = a + b * t
        u = sp.ab2_update(u, nh, prev if prev is not None else np.zeros_like(nh), dt,
                          dts[n - 1] if n else 0.0, n)
        prev, t = nh, t + dt
    exact = u0 + a * t + b * t * t / 2 - b * dts[0] ** 2 / 2
    assert np.abs(u - exact).max() <= 1e-13 * np.abs(exact).max()


def test_ab2_integrating_factor_second_order(orc):
    """u' = -nu k^2 u + a + b t has the closed form
    e^{-lt} u0 + a (1 - e^{-lt})/l + b (t/l - (1 - e^{-lt})/l^2), l = nu k^2;
    the scheme must converge to it at second order on variable steps."""
    nu = 0.3
    cfg = _free_cfg((8, 8, 8), nu=nu)
    sp = orc.Spectral(cfg)
    nx, ny, nz = cfg["n"]
    shp = sp.shape()
    rng = np.random.default_rng(9)
    u0 = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    a = rng.standard_normal(shp) + 1j * rng.standard_normal(shp)
    b = rng.standard_normal(shp)
    kx = np.arange(nx // 2 + 1)
    ky = np.fft.fftfreq(ny, 1.0 / ny)
    kz = np.fft.fftfreq(nz, 1.0 / nz)
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    lam = nu * (KX ** 2 + KY ** 2 + KZ ** 2)
    lam = np.where(lam == 0, 1e-300, lam)
    T = 0.3
    errs = []
    for refine in (1, 2, 4):
        pattern = [0.011, 0.017, 0.008, 0.014]
        dts = []
        while sum(dts) < T - 1e-12:
            dts.append(pattern[len(dts) % 4] / refine)
        dts[-1] -= sum(dts) - T
        u, t, prev = u0.copy(), 0.0, None
        for n, dt in enumerate(dts):
            nh = a + b * t
            u = sp.ab2_update(u, nh, prev if prev is not None else np.zeros_like(nh), dt,
                              dts[n - 1] if n else 0.0, n)
            prev, t = nh, t + dt
        E = np.exp(-lam * T)
        with np.errstate(invalid="ignore", over="ignore"):
            exact = E * u0 + a * (1 - E) / lam + b * (T / lam - (1 - E) / lam ** 2)
        exact[:, 0, 0, 0] = u0[:, 0, 0, 0] + a[:, 0, 0, 0] * T + b[:, 0, 0, 0] * T * T / 2
        errs.append(np.abs(u - exact).max())
    assert 3.3 < errs[0] / errs[1] < 4.7
    assert 3.3 < errs[1] / errs[2] < 4.7


# --------------------------------------------------------------- P7 TG decay

def test_taylor_green_2d_decay(orc):
    """The z-invariant Taylor-Green vortex has u x omega = -grad(sin^2 x sin^2 y)
    (removed by the projection) and |k|^2 = 2, so the amplitude decays as
    exp(-2 nu t) to round-off with the mask off."""
    nu, dt = 0.01, 1e-3
    cfg = {"n": (16, 16, 8), "L": (2 * math.pi,) * 3, "nu": nu, "eta": 1.0,
           "dt_fixed": dt, "mean_mode": "fixed"}
    u0 = workloads.taylor_green_2d(cfg["n"], cfg["L"])
    sim = orc.Simulation(cfg, None)
    sim.set_state(u0)
    sim.step(20)
    ref = u0 * math.exp(-2 * nu * 20 * dt)
    assert np.abs(sim.get_state() - ref).max() <= 1e-12


# ----------------------------------------------------- P8 energy, budget

def test_energy_conservation_semi_discrete(orc):
    """At nu = 0 without a mask, sum_k w Re(u_hat* . N_hat) = 0: u.(u x omega)
    vanishes pointwise and projection and truncation are self-adjoint."""
    cfg = _free_cfg((16, 12, 10), L=(2.0, 3.0, 2.5))
    sp = orc.Spectral(cfg)
    uh = sp.project(sp.dealias(sp.forward(workloads.random_field(cfg["n"], seed=8))))
    nh, _ = sp.rhs(uh)
    w = _weights(cfg["n"][0], uh.shape[-1])
    dot = np.sum(w * np.real(np.conj(uh) * nh))
    scale = np.sum(w * np.abs(uh) * np.abs(nh))
    assert abs(dot) <= 1e-14 * scale


@pytest.mark.slow
def test_energy_drift_second_order(orc):
    T = 0.2
    drifts = []
    for dt in (0.01, 0.005):
        cfg = _free_cfg((16, 16, 16), dt_fixed=dt)
        sim = orc.Simulation(cfg, None)
        sim.set_state(workloads.random_smooth_field(cfg["n"], seed=3, kmax=3))
        e0 = 0.5 * np.sum(sim.get_state() ** 2)
        sim.step(int(round(T / dt)))
        drifts.append(abs(0.5 * np.sum(sim.get_state() ** 2) - e0))
    assert 3.0 < drifts[0] / drifts[1] < 5.0


def test_energy_budget_with_penalization(orc):
    """For u_s = 0 the right-hand side changes the energy at the rate
    -sum chi |u|^2 dV / C_eta (the Lamb vector does no work); checked on the
    3-D Taylor-Green field with the fixed sphere, whose modes survive the
    truncation and the projection unchanged."""
    cfg, ins = workloads.config_tg_sphere(16)
    u0 = workloads.initial_field(cfg)
    sp = orc.Spectral(cfg)
    uh = sp.forward(u0)
    nh, sums = sp.rhs(uh, 0.0, ins)
    chi, col, us = orc.mask_grid(cfg, ins, 0.0)
    assert np.all(us == 0) and chi.max() > 0.9
    dV = (2 * math.pi / 16) ** 3
    w = _weights(16, uh.shape[-1])
    rate = (2 * math.pi) ** 3 * np.sum(w * np.real(np.conj(uh) * nh))
    expect = -np.sum(chi * np.sum(u0 ** 2, axis=0)) * dV / cfg["eta"]
    assert abs(rate - expect) <= 1e-12 * abs(expect)
    assert abs(sums[orc.SUM_EKIN] - 0.5 * np.sum(u0 ** 2) * dV) <= 1e-13 * sums[orc.SUM_EKIN]
    assert abs(sums[orc.SUM_UMAX] - np.sqrt(np.sum(u0 ** 2, axis=0)).max()) <= 1e-14


def test_adaptive_dt_rule(orc):
    """dt = min(CFL dx / max|u|, C_eta, dt_max) (reading of Algorithm 1 step b)."""
    n = (8, 8, 8)
    L = (4.0, 4.0, 4.0)
    for umax, eta, dtmax, expect in [(2.0, 1.0, 0.0, 0.1 * 0.5 / 2.0),
                                     (0.01, 1e-3, 0.0, 1e-3),
                                     (2.0, 1.0, 1e-3, 1e-3)]:
        cfg = {"n": n, "L": L, "nu": 0.0, "eta": eta, "cfl": 0.1, "dt_max": dtmax,
               "mean_mode": "free"}
        sim = orc.Simulation(cfg, None)
        sim.set_state(workloads.uniform(n, (umax, 0.0, 0.0)))
        row = sim.step(1)[0]
        assert abs(row[1] - expect) <= 1e-15 * expect
        assert abs(row[21] - umax) <= 1e-14 * umax
