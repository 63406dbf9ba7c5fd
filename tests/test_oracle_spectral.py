"""Pins of the oracle's spectral operators (Sec. 2.4): exact derivatives of
single Fourier modes, the rotational-form nonlinear term of a two-mode field
worked out by hand, the Leray projection (Algorithm 1 step d) and the 2/3
rule's retained set."""
import math

import numpy as np
import pytest

import workloads


def _cfg(n, L=(2 * math.pi,) * 3, **kw):
    c = {"n": n, "L": L, "nu": 0.0, "eta": 1.0, "mean_mode": "free"}
    c.update(kw)
    return c


def _coords(cfg):
    x, y, z = workloads.grid(cfg["n"], cfg["L"])
    Z, Y, X = np.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


@pytest.mark.parametrize("m", [1, 2, 5])
def test_curl_of_single_modes_is_exact(orc, m):
    cfg = _cfg((16, 12, 20), L=(3.0, 2.5, 4.0))
    sp = orc.Spectral(cfg)
    X, Y, Z = _coords(cfg)
    kx = 2 * math.pi * m / cfg["L"][0]
    kz = 2 * math.pi * min(m, 3) / cfg["L"][2]
    ky = 2 * math.pi * min(m, 2) / cfg["L"][1]
    # u = (cos(kz z), sin(kx x), sin(ky y)):
    # curl u = (ky cos(ky y), -kz sin(kz z), kx cos(kx x))
    u = np.stack([np.cos(kz * Z), np.sin(kx * X), np.sin(ky * Y)])
    w = sp.inverse(sp.curl(sp.forward(u)))
    ref = np.stack([ky * np.cos(ky * Y), -kz * np.sin(kz * Z), kx * np.cos(kx * X)])
    assert np.abs(w - ref).max() <= 1e-13 * max(kx, ky, kz)


def test_lamb_vector_of_two_modes(orc):
    """u = (sin z, sin x, 0): omega = (0, cos z, cos x) and
    u x omega = (sin x cos x, -sin z cos x, sin z cos z).  The first and last
    components are gradients, the middle one is solenoidal, so the projected,
    dealiased term is exactly (0, -sin z cos x, 0)."""
    cfg = _cfg((16, 16, 16))
    sp = orc.Spectral(cfg)
    X, Y, Z = _coords(cfg)
    u = np.stack([np.sin(Z), np.sin(X), np.zeros_like(X)])
    nh, sums = sp.rhs(sp.forward(u))
    nl = sp.inverse(nh)
    ref = np.stack([np.zeros_like(X), -np.sin(Z) * np.cos(X), np.zeros_like(X)])
    assert np.abs(nl - ref).max() <= 1e-14
    assert sums[orc.SUM_NONFINITE] == 0


def test_projection(orc):
    cfg = _cfg((12, 16, 10), L=(1.0, 2.0, 3.0))
    sp = orc.Spectral(cfg)
    f = sp.forward(workloads.random_field(cfg["n"], seed=21))
    pf = sp.project(f)
    nx, ny, nz = cfg["n"]
    kx = 2 * math.pi * np.arange(nx // 2 + 1) / cfg["L"][0]
    ky = 2 * math.pi * np.fft.fftfreq(ny, 1.0 / ny) / cfg["L"][1]
    kz = 2 * math.pi * np.fft.fftfreq(nz, 1.0 / nz) / cfg["L"][2]
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    # numpy's fftfreq numbers the Nyquist plane -n/2, as the solver does
    kmag = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    div = KX * pf[0] + KY * pf[1] + KZ * pf[2]
    bound = (kmag * np.sqrt(np.sum(np.abs(f) ** 2, axis=0))).max()
    assert np.abs(div).max() <= 1e-14 * bound
    assert np.abs(sp.project(pf) - pf).max() <= 1e-15 * np.abs(f).max() * 10
    # a pure gradient field projects to zero, a curl field is unchanged
    X, Y, Z = _coords(cfg)
    a, b, c = (2 * math.pi / cfg["L"][i] for i in range(3))
    phi_grad = np.stack([a * np.cos(a * X) * np.sin(c * Z), np.zeros_like(X),
                         c * np.sin(a * X) * np.cos(c * Z)])
    assert np.abs(sp.project(sp.forward(phi_grad))).max() <= 1e-15 * 10
    sol = np.stack([np.sin(b * Y), np.sin(c * Z), np.sin(a * X)])
    sh = sp.forward(sol)
    assert np.abs(sp.project(sh) - sh).max() <= 1e-16 * 10


@pytest.mark.parametrize("n,strict,kept", [(96, 0, 32), (96, 1, 31), (512, 0, 170),
                                           (512, 1, 170), (32, 0, 10), (12, 0, 4)])
def test_dealias_cutoff(orc, n, strict, kept):
    """2/3 rule: keep |m| <= floor(n/3) (strict: |m| < n/3), per axis."""
    nn = (n, 6, 6) if n > 64 else (n, n, n)
    cfg = _cfg(nn, dealias_strict=strict)
    sp = orc.Spectral(cfg)
    f = np.ones(sp.shape(1), complex)
    d = sp.dealias(f)[0]
    row = d[0, 0]
    assert np.all(row[: kept + 1] == 1) and np.all(row[kept + 1:] == 0)
    if nn[1] == n:
        col = d[0, :, 0]
        m = np.fft.fftfreq(n, 1.0 / n).astype(int)
        m[n // 2] = -n // 2
        assert np.array_equal(col == 1, np.abs(m) <= kept)


def test_set_get_state_round_trip(orc):
    cfg, ins = workloads.config_tg_sphere(16)
    u0 = workloads.initial_field(cfg)
    sim = orc.Simulation(cfg, ins)
    sim.set_state(u0)
    assert np.abs(sim.get_state() - u0).max() <= 1e-15 * 10


def test_mean_mode_fixed_holds_u_inf(orc):
    cfg = _cfg((8, 8, 8), mean_mode="fixed", u_inf=(0.25, -0.5, 1.0), eta=1e-2, dt_fixed=1e-3)
    sim = orc.Simulation(cfg, None)
    sim.set_state(workloads.random_smooth_field(cfg["n"], seed=2, mean=(3.0, 3.0, 3.0)))
    sim.step(3)
    u = sim.get_state()
    assert np.allclose(u.mean(axis=(1, 2, 3)), (0.25, -0.5, 1.0), atol=1e-14)
