"""Pins of the oracle's own FFT (Sec. 2.4: fields are truncated Fourier series
evaluated by the FFT).  The FFT is checked against a brute-force direct DFT,
against numpy's independent FFT library, by its round trip and by Parseval's
identity -- none of which reuses the oracle's transform code."""
import math

import numpy as np
import pytest

import workloads


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 12, 12), (12, 8, 6)])
def test_fft_matches_direct_dft(orc, shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(7)
    u = rng.standard_normal(shape)
    fast = orc.fft3_r2c(u)
    slow = orc.dft3_r2c(u)
    scale = np.abs(slow).max()
    assert np.abs(fast - slow).max() <= 1e-14 * scale * math.log2(u.size)


@pytest.mark.parametrize("shape", [(16, 16, 16), (24, 12, 18), (10, 14, 30), (27, 25, 8)])
def test_fft_matches_numpy(orc, shape):
    rng = np.random.default_rng(11)
    u = rng.standard_normal(shape)
    ref = np.fft.rfftn(u)
    got = orc.fft3_r2c(u)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


@pytest.mark.parametrize("n", [2, 3, 5, 7, 12, 30, 96, 128, 243])
def test_fft1_both_signs_match_numpy(orc, n):
    rng = np.random.default_rng(n)
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    assert np.allclose(orc.fft1(x, -1), np.fft.fft(x), rtol=0, atol=1e-12 * n)
    assert np.allclose(orc.fft1(x, +1), n * np.fft.ifft(x), rtol=0, atol=1e-12 * n)


@pytest.mark.parametrize("shape", [(8, 8, 8), (16, 12, 24), (6, 10, 14)])
def test_round_trip(orc, shape):
    rng = np.random.default_rng(3)
    u = rng.standard_normal(shape)
    nz, ny, nx = shape
    back = orc.fft3_c2r(orc.fft3_r2c(u), nx) / u.size
    assert np.abs(back - u).max() <= 1e-15 * math.log2(u.size) * 4


def test_inverse_drops_imaginary_dc_and_nyquist(orc):
    """A Hermitian half spectrum synthesises a real field; the c2r takes the
    real parts of the x = 0 and x = nx/2 columns only."""
    nz, ny, nx = 4, 4, 8
    X = np.zeros((nz, ny, nx // 2 + 1), complex)
    X[0, 0, 0] = 2.0 + 5.0j
    X[0, 0, nx // 2] = 1.0 - 3.0j
    u = orc.fft3_c2r(X, nx)
    xs = np.arange(nx)
    assert np.allclose(u[0, 0], 2.0 + np.cos(math.pi * xs), atol=1e-15)


def test_parseval(orc):
    """sum |u|^2 dV = L^3 sum_k w_k |u_hat_k|^2, w = 1 at m_x in {0, nx/2}
    and 2 elsewhere, with u_hat = FFT(u)/N."""
    cfg = {"n": (16, 12, 10), "L": (1.3, 2.0, 0.7), "nu": 0.0, "eta": 1.0}
    sp = orc.Spectral(cfg)
    u = workloads.random_field(cfg["n"], seed=5)
    uh = sp.forward(u)
    nx = cfg["n"][0]
    w = np.full(uh.shape[-1], 2.0)
    w[0] = 1.0
    w[nx // 2] = 1.0
    vol = np.prod(cfg["L"])
    dV = vol / np.prod(cfg["n"])
    lhs = np.sum(u * u) * dV
    rhs = vol * np.sum(w * np.abs(uh) ** 2)
    assert abs(lhs - rhs) <= 1e-13 * lhs
