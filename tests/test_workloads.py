"""The seeded synthetic inputs: closed-form properties of the turbulent inflow
field (the 1024^3 turbulent-insect input) and of the shear waves."""
import math

import numpy as np

import workloads


def _spectrum(u, L):
    n = u.shape[1:][::-1]
    uh = np.fft.fftn(u, axes=(1, 2, 3)) / np.prod(n)
    k = [2 * np.pi * np.fft.fftfreq(n[j], L[j] / n[j]) for j in range(3)]
    KZ, KY, KX = np.meshgrid(k[2], k[1], k[0], indexing="ij")
    return uh, KX, KY, KZ


def test_turbulent_field_properties():
    n, L = (32, 24, 40), (4.0, 3.0, 5.0)
    u = workloads.turbulent_field(n, L, mean=(0.25, 0.0, 0.0))
    assert u.shape == (3, 40, 24, 32)
    for c, mu in enumerate((0.25, 0.0, 0.0)):
        assert abs(u[c].mean() - mu) <= 1e-14
    fl = u - np.array([0.25, 0.0, 0.0])[:, None, None, None]
    assert abs(math.sqrt((fl ** 2).sum(0).mean() / 3) - 0.1) <= 1e-13
    uh, KX, KY, KZ = _spectrum(fl, L)
    kk = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    mag = np.sqrt((np.abs(uh) ** 2).sum(0))
    live = mag > 1e-12 * mag.max()
    assert kk[live].min() >= 2.0 - 1e-12 and kk[live].max() <= 8.0 + 1e-12
    div = np.abs(KX * uh[0] + KY * uh[1] + KZ * uh[2]).max()
    assert div <= 1e-13 * (kk * mag).max()


def test_turbulent_field_matches_direct_mode_sum():
    n, L = (16, 16, 16), (4.0, 4.0, 4.0)
    u = workloads.turbulent_field(n, L)
    m, a = workloads.turbulent_modes(L)
    rng = np.random.default_rng(3)
    for _ in range(20):
        ix, iy, iz = (int(rng.integers(0, 16)) for _ in range(3))
        x = np.array([ix, iy, iz]) * 4.0 / 16
        ph = np.exp(1j * (2 * np.pi * m / 4.0) @ x)
        direct = 2 * (a * ph[:, None]).sum(0).real
        assert np.abs(u[:, iz, iy, ix] - direct).max() <= 1e-13


def test_turbulent_shell_energy_follows_minus_five_thirds():
    m, a = workloads.turbulent_modes((4.0, 4.0, 4.0))
    k = np.sqrt(((2 * np.pi * m / 4.0) ** 2).sum(1))
    e = 2 * (np.abs(a) ** 2).sum(1)
    # per mode the energy is E(k) / (4 pi k^2) times a chi-square(4) draw
    # projected to the plane: its mean over modes scales as k^(-5/3 - 2)
    lo, hi = k < 4.0, k > 5.5
    ratio = e[lo].mean() / e[hi].mean()
    expect = np.mean(k[lo] ** (-11 / 3)) / np.mean(k[hi] ** (-11 / 3))
    assert 0.6 * expect <= ratio <= 1.6 * expect


def test_shear_waves_points_match_grid():
    n, L = (16, 12, 8), (2.0, 3.0, 4.0)
    u = workloads.shear_waves(n, L, mean=(0.1, 0.2, 0.3))
    pts = np.array([[3, 4, 5], [0, 0, 0], [15, 11, 7]])
    v = workloads.shear_waves(n, L, mean=(0.1, 0.2, 0.3), points=pts)
    for i, (ix, iy, iz) in enumerate(pts):
        assert np.allclose(v[:, i], u[:, iz, iy, ix], rtol=0, atol=1e-15)
    e = 0.5 * (u ** 2).sum(0).mean() * np.prod(L)
    assert abs(e - workloads.shear_waves_energy(L, mean=(0.1, 0.2, 0.3))) <= 1e-13 * e
