"""Pins of the oracle's wake-removal terms (Sec. 2.3): the vorticity sponge
-(1/C_sp) curl nabla^-2 (chi_sp omega) and the Dirichlet layer u = u_inf.

The sponge is pinned by what the paper asks of it: it damps vorticity where
chi_sp = 1 (its curl is -chi_sp omega / C_sp when chi_sp omega is solenoidal),
it is divergence-free, it leaves the mean alone, and with chi_sp = 1 everywhere
the AB2 step reduces to the relaxation recurrence at rate 1/C_sp."""
import math

import numpy as np
import pytest


def _cfg(n, L, **kw):
    c = {"n": n, "L": L, "nu": 0.0, "eta": 1e-2, "dt_fixed": 1e-3, "mean_mode": "fixed"}
    c.update(kw)
    return c


def _grid(n, L):
    nx, ny, nz = n
    z, y, x = np.meshgrid(np.arange(nz) * L[2] / nz, np.arange(ny) * L[1] / ny,
                          np.arange(nx) * L[0] / nx, indexing="ij")
    return x, y, z


def test_sponge_everywhere_is_a_relaxation(orc):
    """chi_sp = 1 everywhere, nu = 0: u = (0, a sin kx, b cos kx) has a gradient
    Lamb vector, so N = -u / C_sp and AB2 with constant dt gives
    u^1 = u^0 (1 - dt/C), u^{n+1} = u^n - dt/C (3/2 u^n - 1/2 u^{n-1})."""
    n, L = (16, 8, 8), (2.0, 1.0, 1.0)
    Csp, dt = 0.05, 1e-3
    cfg = _cfg(n, L, sponge_c=Csp, sponge_width=(L[0], 0.0, 0.0), dt_fixed=dt)
    x, y, z = _grid(n, L)
    k = 2 * math.pi * 2 / L[0]
    u0 = np.zeros((3,) + x.shape)
    u0[1] = 0.7 * np.sin(k * x)
    u0[2] = 0.4 * np.cos(k * x)
    sim = orc.Simulation(cfg, None)
    sim.set_state(u0)
    amp = [1.0, 1.0 - dt / Csp]
    sim.step(1)
    for _ in range(9):
        amp.append(amp[-1] - dt / Csp * (1.5 * amp[-1] - 0.5 * amp[-2]))
        sim.step(1)
    u = sim.get_state()
    assert np.abs(u - amp[-1] * u0).max() <= 1e-13
    assert abs(u.mean()) <= 1e-15


def test_sponge_curl_damps_vorticity_in_its_slab(orc):
    """u = (sin ky, 0, 0): omega = (0, 0, -k cos ky) and chi_sp(x) omega is
    solenoidal, so curl S = -chi_sp omega / C_sp at every grid point."""
    n, L = (24, 12, 8), (3.0, 1.5, 1.0)
    Csp = 0.1
    cfg = _cfg(n, L, sponge_c=Csp, sponge_width=(0.75, 0.0, 0.0))
    sp = orc.Spectral(cfg)
    x, y, z = _grid(n, L)
    k = 2 * math.pi / L[1]
    u = np.zeros((3,) + x.shape)
    u[0] = np.sin(k * y)
    w = sp.inverse(sp.curl(sp.forward(u)))
    assert np.abs(w[2] + k * np.cos(k * y)).max() <= 1e-12
    chi = np.array([[[sp.sponge_mask((xi, yi, zi)) for xi in x[0, 0]] for yi in y[0, :, 0]]
                    for zi in z[:, 0, 0]])
    assert chi.sum() == 6 * n[1] * n[2]
    assert set(np.unique(chi)) == {0.0, 1.0}
    assert (chi[:, :, x[0, 0] >= 2.25] == 1).all() and (chi[:, :, x[0, 0] < 2.25] == 0).all()
    V = chi[None] * w
    S = sp.sponge_term(sp.forward(V))
    curlS = sp.inverse(sp.curl(S))
    assert np.abs(curlS + V / Csp).max() <= 1e-11 * np.abs(V / Csp).max()


def test_sponge_is_solenoidal_and_keeps_the_mean(orc):
    import workloads
    n, L = (16, 12, 10), (2.0, 1.5, 1.25)
    cfg = _cfg(n, L, sponge_c=0.1, sponge_width=(0.5, 0.25, 0.0))
    sp = orc.Spectral(cfg)
    V = workloads.random_field(n, seed=11)
    S = sp.sponge_term(sp.forward(V))
    hx = n[0] // 2 + 1
    kx = 2 * np.pi * np.arange(hx) / L[0]
    ky = 2 * np.pi * np.fft.fftfreq(n[1], 1.0 / n[1]) / L[1]
    kz = 2 * np.pi * np.fft.fftfreq(n[2], 1.0 / n[2]) / L[2]
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    div = KX * S[0] + KY * S[1] + KZ * S[2]
    assert np.abs(div).max() <= 1e-13 * np.abs(S).max() * max(abs(kx).max(), abs(ky).max(), abs(kz).max())
    assert np.abs(S[:, 0, 0, 0]).max() == 0.0
    # linear in chi_sp omega and scaled by 1 / C_sp
    cfg2 = dict(cfg, sponge_c=0.05)
    S2 = orc.Spectral(cfg2).sponge_term(sp.forward(2 * V))
    assert np.abs(S2 - 4 * S).max() <= 1e-13 * np.abs(S).max()


def test_dirichlet_layer_penalizes_towards_inflow(orc):
    n, L = (16, 8, 8), (4.0, 2.0, 2.0)
    uinf = (0.25, -0.1, 0.05)
    cfg = _cfg(n, L, u_inf=uinf, layer_width=(0.5, 0.0, 0.0), eta=2e-3)
    sp = orc.Spectral(cfg)
    sim = orc.Simulation(cfg, None)
    sim.set_state(np.zeros((3, 8, 8, 16)))
    # the state's mean is held at u_inf, so u = u_inf everywhere: no layer force
    f = sp.physical_fields(sim.uh)
    assert np.abs(f[11:14]).max() <= 1e-12
    # a zero-mean perturbation: NL = u x omega - chi_d (u - u_inf) / C_eta
    mean_free = dict(cfg, mean_mode="free", u_inf=(0.0, 0.0, 0.0))
    x, y, z = _grid(n, L)
    u = np.zeros((3,) + x.shape)
    u[1] = 0.3 * np.sin(2 * np.pi * x / L[0])
    sim2 = orc.Simulation(mean_free, None)
    sim2.set_state(u)
    cfg_layer = dict(cfg, u_inf=(0.0, 0.0, 0.0))
    f2 = orc.Spectral(cfg_layer).physical_fields(sim2.uh)
    lamb = np.cross(f2[0:3], f2[3:6], axis=0)
    chi_d = (x >= 3.5).astype(float)
    expect = lamb - chi_d[None] * f2[0:3] / 2e-3
    assert np.abs(f2[11:14] - expect).max() <= 1e-10
    assert chi_d.sum() == 2 * 8 * 8


def test_uniform_inflow_is_steady_with_sponge_and_layer(orc):
    n, L = (16, 8, 8), (4.0, 2.0, 2.0)
    cfg = _cfg(n, L, u_inf=(0.25, 0.0, 0.0), nu=0.01, sponge_c=0.1,
               sponge_width=(0.5, 0.5, 0.0), layer_width=(0.25, 0.0, 0.0))
    sim = orc.Simulation(cfg, None)
    u0 = np.zeros((3, 8, 8, 16))
    u0[0] = 0.25
    sim.set_state(u0)
    sim.step(5)
    assert np.abs(sim.get_state() - u0).max() <= 1e-14
