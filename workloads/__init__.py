"""Seeded synthetic inputs and run configurations.

This module is shared by the tests, the benchmark and the oracle harness.  It
holds parameters and input fields only -- none of the method's arithmetic --
so that neither the CUDA path nor the oracle depends on the other through it.

Configurations (grid n = (nx, ny, nz), box L, viscosity nu, penalization
constant eta = C_eta, time-step options) and insect descriptors are plain
dicts.  Angles are in radians; kinematic angles are Fourier series
``a0/2 + sum_i a_i cos(2 pi i f t) + b_i sin(2 pi i f t)`` given as
``(a0, [a_1..], [b_1..])``.
"""
from __future__ import annotations

import math

import numpy as np

DEG = math.pi / 180.0


# ------------------------------------------------------------------ helpers

def grid(n, L):
    """Coordinates x_i = i L/n of the periodic grid, as (x, y, z) arrays."""
    nx, ny, nz = n
    Lx, Ly, Lz = L
    x = np.arange(nx) * (Lx / nx)
    y = np.arange(ny) * (Ly / ny)
    z = np.arange(nz) * (Lz / nz)
    return x, y, z


def mean_tip_speed(phi_m, freq=1.0, R=1.0):
    """U_tip = 2 Phi R f with stroke amplitude Phi = 2 phi_m (mean tip speed)."""
    return 4.0 * phi_m * freq * R


def peak_tip_speed(phi_m, freq=1.0, R=1.0):
    """U_tip = 2 pi phi_m f R, the peak speed of phi = phi_m sin(2 pi f t)."""
    return 2.0 * math.pi * phi_m * freq * R


def nu_from_re(re, U, length):
    return U * length / re


def boundary_layer_points(nu, eta, dx):
    """K = delta_eta / dx with delta_eta = sqrt(nu C_eta), the number of grid
    points across the penalization boundary layer (recommended 0.1 - 0.4)."""
    return math.sqrt(nu * eta) / dx


# -------------------------------------------------------------- input fields

def taylor_green_3d(n, L=(2 * math.pi,) * 3):
    """u = (sin x cos y cos z, -cos x sin y cos z, 0) scaled to the box."""
    x, y, z = grid(n, L)
    X = 2 * math.pi * x / L[0]
    Y = 2 * math.pi * y / L[1]
    Z = 2 * math.pi * z / L[2]
    Zg, Yg, Xg = np.meshgrid(Z, Y, X, indexing="ij")
    u = np.zeros((3,) + Xg.shape)
    u[0] = np.sin(Xg) * np.cos(Yg) * np.cos(Zg)
    u[1] = -np.cos(Xg) * np.sin(Yg) * np.cos(Zg)
    return u


def taylor_green_2d(n, L=(2 * math.pi,) * 3, amplitude=1.0):
    """z-invariant u = A (sin x cos y, -cos x sin y, 0)."""
    x, y, z = grid(n, L)
    X = 2 * math.pi * x / L[0]
    Y = 2 * math.pi * y / L[1]
    Zg, Yg, Xg = np.meshgrid(z, Y, X, indexing="ij")
    u = np.zeros((3,) + Xg.shape)
    u[0] = amplitude * np.sin(Xg) * np.cos(Yg)
    u[1] = -amplitude * np.cos(Xg) * np.sin(Yg)
    return u


SHEAR_WAVES = ((0.6, (0, 3, 5), 0.3), (0.4, (7, 0, -2), 1.1), (0.5, (4, 9, 0), -0.7))


def shear_waves(n, L, mean=(0.0, 0.0, 0.0), points=None):
    """Divergence-free band-limited field: component c is a single Fourier mode
    that does not depend on coordinate c, amplitude a_c, integer wavenumbers
    SHEAR_WAVES[c][1], phase SHEAR_WAVES[c][2], plus a uniform mean.  With
    `points` (an (m, 3) integer array of (ix, iy, iz)) it returns the values
    there, shape (3, m); otherwise the whole grid [3][nz][ny][nx]."""
    nx, ny, nz = n
    if points is not None:
        fx = points[:, 0] / nx
        fy = points[:, 1] / ny
        fz = points[:, 2] / nz
    else:
        fz = (np.arange(nz) / nz)[:, None, None]
        fy = (np.arange(ny) / ny)[None, :, None]
        fx = (np.arange(nx) / nx)[None, None, :]
    shape = (len(points),) if points is not None else (nz, ny, nx)
    out = np.empty((3,) + shape)
    trig = (np.sin, np.cos, np.sin)
    for c, (a, m, ph) in enumerate(SHEAR_WAVES):
        arg = 2 * math.pi * (m[0] * fx + m[1] * fy + m[2] * fz) + ph
        out[c] = mean[c] + a * trig[c](arg)
    return out


def shear_waves_energy(L, mean=(0.0, 0.0, 0.0)):
    """1/2 integral |u|^2 over the box for shear_waves: each mode averages a^2/2."""
    vol = L[0] * L[1] * L[2]
    return 0.5 * vol * sum(mean[c] ** 2 + SHEAR_WAVES[c][0] ** 2 / 2 for c in range(3))


def uniform(n, u0):
    nx, ny, nz = n
    u = np.zeros((3, nz, ny, nx))
    for c in range(3):
        u[c] = u0[c]
    return u


def random_field(n, seed, amplitude=1.0, mean=(0.0, 0.0, 0.0)):
    """Gaussian white noise on the grid, seeded; band limiting and the
    divergence-free projection are left to the solver's set_state."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    u = amplitude * rng.standard_normal((3, nz, ny, nx))
    for c in range(3):
        u[c] += mean[c]
    return u


def random_smooth_field(n, seed, amplitude=1.0, kmax=4, mean=(0.0, 0.0, 0.0)):
    """Sum of a few random Fourier modes with integer wavenumbers |m| <= kmax,
    built directly in physical space (cosines with random phases)."""
    nx, ny, nz = n
    rng = np.random.default_rng(seed)
    zi, yi, xi = np.meshgrid(np.arange(nz) / nz, np.arange(ny) / ny, np.arange(nx) / nx,
                             indexing="ij")
    u = np.zeros((3, nz, ny, nx))
    for c in range(3):
        for _ in range(12):
            m = rng.integers(-kmax, kmax + 1, size=3)
            ph = rng.uniform(0, 2 * math.pi)
            a = rng.standard_normal() * amplitude / 4
            u[c] += a * np.cos(2 * math.pi * (m[0] * xi + m[1] * yi + m[2] * zi) + ph)
        u[c] += mean[c]
    return u


# ------------------------------------------------------------ insect shapes

def sphere(center, radius, profile="tanh", c_smth=1.0):
    """Fixed sphere, u_s = 0 (config "plain method, 32^3")."""
    return {"body": "sphere", "nwings": 0, "profile": profile, "c_smth": c_smth,
            "x_cntr": tuple(center), "body_axes": (radius, 0.0)}


def flapping_kinematics(phi_m=60 * DEG, alpha_m=45 * DEG, freq=1.0):
    """phi = phi_m sin(2 pi f t), alpha = alpha_m cos(2 pi f t), theta = 0."""
    return {"phi": (0.0, [0.0], [phi_m]), "alpha": (0.0, [alpha_m], [0.0]),
            "theta": (0.0, [0.0], [0.0])}


def plate_wing(dx, chord=0.3, span=1.0, thickness_cells=4.0):
    """Rectangular plate: (c_le, c_te, R, h); feathering axis at mid-chord."""
    return (0.5 * chord, 0.5 * chord, span, thickness_cells * dx)


def single_wing(L=(4.0, 4.0, 4.0), n=(256, 256, 256), phi_m=60 * DEG, alpha_m=45 * DEG,
                freq=1.0):
    """One rigid flat-plate wing pivoting at its root in the box centre."""
    dx = max(L[i] / n[i] for i in range(3))
    return {"body": "none", "nwings": 1, "profile": "cos", "c_smth": 1.0,
            "x_cntr": tuple(0.5 * l for l in L), "eta_stroke": -90 * DEG,
            "pivot_l": (0.0, 0.0, 0.0), "wing": plate_wing(dx), "freq": freq,
            "kinematics": flapping_kinematics(phi_m, alpha_m, freq)}


def model_insect(L=(4.0, 4.0, 4.0), n=(512, 512, 512)):
    """Ellipsoidal body (0.5, 0.12, 0.12) plus two mirror-symmetric plates."""
    dx = max(L[i] / n[i] for i in range(3))
    return {"body": "ellipsoid", "nwings": 2, "profile": "cos", "c_smth": 1.0,
            "x_cntr": tuple(0.5 * l for l in L), "body_axes": (0.5, 0.12),
            "eta_stroke": -90 * DEG, "pivot_l": (0.0, 0.15, 0.0),
            "pivot_r": (0.0, -0.15, 0.0), "wing": plate_wing(dx), "freq": 1.0,
            "kinematics": flapping_kinematics()}


def contour_wing_outline(span=0.96, chord=0.3, harmonics=16):
    """A synthetic wing outline for the contour parametrization of Sec. 3.4:
    an ellipse of the given span and chord centred at mid-span on the y^(w)
    axis, with a slight forward sweep of the tip, written as the truncated
    Fourier series R(theta) = a0/2 + sum a_i cos(i theta) + b_i sin(i theta)
    (coefficients from 256 samples of the outline; made-up geometry, not
    measured wing data)."""
    a, b, sweep = 0.5 * chord, 0.5 * span, 0.04
    th = 2 * math.pi * np.arange(256) / 256
    R = a * b / np.sqrt((b * np.cos(th)) ** 2 + (a * np.sin(th)) ** 2)
    R = R * (1.0 + sweep * np.sin(th) * np.cos(th))
    F = np.fft.rfft(R) / 256
    return {"center": (0.0, 0.5 * span + 0.02),
            "a0": float(2 * F[0].real),
            "a": [float(2 * F[i].real) for i in range(1, harmonics + 1)],
            "b": [float(-2 * F[i].imag) for i in range(1, harmonics + 1)]}


def realistic_insect(L=(4.0, 4.0, 4.0), n=(512, 512, 512)):
    """Ellipsoid thorax with a head and two eyes (Sec. 3.2) and two contour
    wings (Sec. 3.4) with the flapping kinematics of the model insect."""
    ins = model_insect(L, n)
    ins["head"] = ((0.62, 0.0, 0.04), 0.13)
    ins["eyes"] = ((0.66, 0.09, 0.08), 0.06)
    ins["contour"] = contour_wing_outline()
    return ins


def curved_insect(L=(4.0, 4.0, 4.0), n=(512, 512, 512)):
    """The realistic insect with its thorax bent along a circular centre line
    (the body form of the fruit fly of Sec. 5.3): centre-line circle of
    radius 1 below the body origin, head and eyes moved to its front end,
    pitched body.  Made-up geometry, no paper values."""
    ins = realistic_insect(L, n)
    ins["body"] = "curved"
    ins["body_arc"] = (1.0, 0.0, -1.0)
    ins["head"] = ((0.56, 0.0, -0.16), 0.13)
    ins["eyes"] = ((0.6, 0.09, -0.1), 0.06)
    ins["body_angles"] = (0.0, -0.3, 0.0)
    return ins


# ------------------------------------------------------------ configurations

def config_tg_sphere(n=32):
    """Plain method, FP64: Taylor-Green in a 2 pi box with a fixed sphere."""
    L = (2 * math.pi,) * 3
    cfg = {"name": f"tg_sphere_{n}", "n": (n, n, n), "L": L, "nu": 0.01, "eta": 1e-2,
           "dt_fixed": 1e-3, "steps": 20, "mean_mode": "fixed"}
    cfg["init"] = ("taylor_green_3d",)
    ins = sphere((math.pi, math.pi, math.pi), 0.5, profile="tanh")
    return cfg, ins


def config_single_wing(n=256):
    """One flapping plate at Re = 100 (chord, mean tip speed), 4^3 box."""
    L = (4.0, 4.0, 4.0)
    U = mean_tip_speed(60 * DEG)
    cfg = {"name": f"single_wing_{n}", "n": (n, n, n), "L": L,
           "nu": nu_from_re(100.0, U, 0.3), "eta": 2.5e-3, "cfl": 0.1, "mean_mode": "fixed"}
    cfg["init"] = ("uniform", (0.0, 0.0, 0.0))
    ins = single_wing(L, cfg["n"])
    return cfg, ins


def config_model_insect(n=512):
    """Model insect at Re = 300 in uniform inflow (0.25, 0, 0), 4^3 box."""
    L = (4.0, 4.0, 4.0)
    U = mean_tip_speed(60 * DEG)
    cfg = {"name": f"model_insect_{n}", "n": (n, n, n), "L": L,
           "nu": nu_from_re(300.0, U, 0.3), "eta": 1e-3, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.25, 0.0, 0.0)}
    cfg["init"] = ("uniform", (0.25, 0.0, 0.0))
    ins = model_insect(L, cfg["n"])
    return cfg, ins


def turbulent_modes(L, seed=6513, kmin=2.0, kmax=8.0, urms=0.1):
    """Modes of a seeded random-phase isotropic divergence-free field.

    For every integer wave vector m in the half space (m_x > 0, or m_x = 0 and
    m_y > 0, or m_x = m_y = 0 and m_z > 0) with kmin <= |k| <= kmax,
    k = 2 pi m / L, in the order of the loops below: a complex Gaussian vector
    from default_rng(seed), its component along k removed, scaled by
    sqrt(E(|k|) / (4 pi |k|^2)) with E(k) = k^(-5/3).  The field is
    u(x) = sum 2 Re(a e^{i k.x}); the amplitudes are rescaled so that
    u_rms = sqrt(<|u|^2>/3) = urms, using <|u|^2> = sum 2 |a|^2.
    Returns (m int array (M, 3), a complex array (M, 3))."""
    rng = np.random.default_rng(seed)
    mmax = [int(math.ceil(kmax * L[j] / (2 * math.pi))) for j in range(3)]
    ms, amps = [], []
    for mx in range(0, mmax[0] + 1):
        for my in range(-mmax[1], mmax[1] + 1):
            for mz in range(-mmax[2], mmax[2] + 1):
                if mx == 0 and (my < 0 or (my == 0 and mz <= 0)):
                    continue
                k = np.array([2 * math.pi * mx / L[0], 2 * math.pi * my / L[1], 2 * math.pi * mz / L[2]])
                kk = float(np.sqrt(k @ k))
                if kk < kmin or kk > kmax:
                    continue
                a = rng.standard_normal(3) + 1j * rng.standard_normal(3)
                a = a - k * (k @ a) / (kk * kk)
                a = a * math.sqrt(kk ** (-5.0 / 3.0) / (4 * math.pi * kk * kk))
                ms.append((mx, my, mz))
                amps.append(a)
    m = np.array(ms, dtype=np.int64)
    a = np.array(amps)
    scale = urms * math.sqrt(3.0) / math.sqrt(float(np.sum(2 * np.abs(a) ** 2)))
    return m, a * scale


def turbulent_field(n, L, mean=(0.0, 0.0, 0.0), seed=6513, kmin=2.0, kmax=8.0, urms=0.1,
                    device=None, zchunk=32):
    """turbulent_modes evaluated on the grid plus a uniform mean,
    [3][nz][ny][nx].  Modes are grouped by (m_y, m_z); each z plane is a
    (ny x P) by (P x nx) complex product of separable exponentials.  With
    `device` (a torch CUDA device) the field is built there as a float32 torch
    tensor; otherwise as a float64 numpy array."""
    nx, ny, nz = n
    m, a = turbulent_modes(L, seed, kmin, kmax, urms)
    pairs = sorted(set((int(r[1]), int(r[2])) for r in m))
    index = {p: i for i, p in enumerate(pairs)}
    P = len(pairs)
    x = np.arange(nx) * L[0] / nx
    F = np.zeros((3, P, nx), complex)
    for (mx, my, mz), amp in zip(m, a):
        e = np.exp(1j * 2 * math.pi * mx / L[0] * x)
        F[:, index[(int(my), int(mz))], :] += 2 * amp[:, None] * e[None, :]
    y = np.arange(ny) * L[1] / ny
    z = np.arange(nz) * L[2] / nz
    Ey = np.exp(1j * 2 * math.pi * np.outer([p[0] for p in pairs], y) / L[1])     # (P, ny)
    Ez = np.exp(1j * 2 * math.pi * np.outer([p[1] for p in pairs], z) / L[2])     # (P, nz)
    if device is None:
        u = np.empty((3, nz, ny, nx))
        for z0 in range(0, nz, zchunk):
            z1 = min(nz, z0 + zchunk)
            G = Ez[:, z0:z1].T[:, None, :] * Ey.T[None, :, :]                     # (zc, ny, P)
            for c in range(3):
                u[c, z0:z1] = (G @ F[c]).real + mean[c]
        return u
    import torch
    u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device=device)
    Ft = torch.as_tensor(F, dtype=torch.complex64, device=device)
    Eyt = torch.as_tensor(Ey.T, dtype=torch.complex64, device=device)
    Ezt = torch.as_tensor(Ez.T, dtype=torch.complex64, device=device)
    for z0 in range(0, nz, zchunk):
        z1 = min(nz, z0 + zchunk)
        G = Ezt[z0:z1, None, :] * Eyt[None, :, :]
        for c in range(3):
            u[c, z0:z1] = torch.matmul(G, Ft[c]).real + mean[c]
    return u


ENSEMBLE_GRIDS = ((64, 64, 64), (96, 96, 96), (128, 128, 128), (96, 96, 192))


def config_ensemble(count=40, seed=1506):
    """Uneven ensemble of independent single-wing runs.  Per run, drawn in this
    order from default_rng(seed): a grid index into ENSEMBLE_GRIDS, phi_0 ~
    U[40, 80] deg, f ~ U[0.8, 1.2], Re ~ U[50, 400] (chord and mean tip speed
    4 phi_0 f R).  Box 4^3 (4 x 4 x 8 for the 96 x 96 x 192 grid), C_eta =
    2.5e-3, quiescent start, CFL 0.1 adaptive."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        g = int(rng.integers(0, len(ENSEMBLE_GRIDS)))
        phi0 = float(rng.uniform(40.0, 80.0)) * DEG
        f = float(rng.uniform(0.8, 1.2))
        re = float(rng.uniform(50.0, 400.0))
        n = ENSEMBLE_GRIDS[g]
        L = (4.0, 4.0, 8.0) if n[2] == 192 else (4.0, 4.0, 4.0)
        cfg = {"name": f"ensemble_{i}", "n": n, "L": L,
               "nu": nu_from_re(re, mean_tip_speed(phi0, f), 0.3), "eta": 2.5e-3, "cfl": 0.1,
               "mean_mode": "fixed", "init": ("uniform", (0.0, 0.0, 0.0)),
               "draw": {"grid": g, "phi0_deg": phi0 / DEG, "freq": f, "re": re}}
        out.append((cfg, single_wing(L, n, phi_m=phi0, freq=f)))
    return out


def config_turbulent_insect(n=1024):
    """The model insect in turbulent inflow: mean (0.25, 0, 0) plus the
    isotropic field of turbulent_field (seed 6513, 2 <= |k| <= 8, u_rms 0.1);
    Re = 1000 on the chord and mean tip speed, C_eta = 5e-4, 4^3 box."""
    L = (4.0, 4.0, 4.0)
    U = mean_tip_speed(60 * DEG)
    cfg = {"name": f"turbulent_insect_{n}", "n": (n, n, n), "L": L,
           "nu": nu_from_re(1000.0, U, 0.3), "eta": 5e-4, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.25, 0.0, 0.0)}
    cfg["init"] = ("turbulent", 6513)
    return cfg, model_insect(L, cfg["n"])


def initial_field(cfg, dtype=np.float64):
    """The configuration's initial velocity on the grid, [3][nz][ny][nx]."""
    kind = cfg["init"][0]
    if kind == "taylor_green_3d":
        u = taylor_green_3d(cfg["n"], cfg["L"])
    elif kind == "uniform":
        nx, ny, nz = cfg["n"]
        u = np.empty((3, nz, ny, nx), dtype)
        for c in range(3):
            u[c] = cfg["init"][1][c]
        return u
    elif kind == "random_smooth":
        u = random_smooth_field(cfg["n"], cfg["init"][1], mean=cfg.get("u_inf", (0, 0, 0)))
    elif kind == "turbulent":
        u = turbulent_field(cfg["n"], cfg["L"], mean=cfg.get("u_inf", (0, 0, 0)), seed=cfg["init"][1])
    else:
        raise ValueError(kind)
    return u.astype(dtype, copy=False)


def steps_per_wingbeat(cfg, peak_speed=2 * math.pi * 60 * DEG):
    """Rough step count of one wingbeat under the CFL limit at peak tip speed."""
    dx = min(cfg["L"][i] / cfg["n"][i] for i in range(3))
    dt = min(cfg.get("cfl", 0.1) * dx / peak_speed, cfg["eta"])
    return int(math.ceil(1.0 / dt))
