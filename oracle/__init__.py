"""Plain FP64 CPU oracle of the penalized pseudo-spectral Navier-Stokes step.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``.  The product path (the CUDA
library and its binding) never imports, links or runs anything here.

The arithmetic lives in plain C (``fft.c``, ``insect.c``, ``solver.c``); this
module compiles it with gcc and marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
# the same sources built with OpenMP: used only to time the oracle on all host
# cores (bench.py's CPU baseline); the tests use the single-threaded build
_LIB_OMP_PATH = os.path.join(_HERE, "liboracle_omp.so")
_SOURCES = ["fft.c", "insect.c", "solver.c"]
_use_openmp = False

MAX_FOURIER = 8
MAX_CONTOUR = 32
ROW_COLS = 26
NSUMS = 39
SUM_EKIN, SUM_UMAX, SUM_NONFINITE = 36, 37, 38


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile liboracle.so with gcc (no fast-math, no FMA contraction); with
    openmp, liboracle_omp.so from the same sources with -fopenmp (its loops
    over independent lines, planes and points split across threads)."""
    path = _LIB_OMP_PATH if openmp else _LIB_PATH
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(path):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(path) >= newest:
            return path
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           *(["-fopenmp"] if openmp else []),
           "-o", path + ".tmp"] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(path + ".tmp", path)
    return path


def build_all() -> None:
    """Both builds (the OpenMP one only where gcc offers -fopenmp)."""
    build()
    try:
        build(openmp=True)
    except (OSError, subprocess.CalledProcessError):
        pass


def use_openmp() -> bool:
    """Load the OpenMP build in this process (before any other oracle call);
    False when it cannot be built here, and the single-threaded one stays."""
    global _use_openmp
    if _lib is not None:
        raise RuntimeError("the oracle library is already loaded in this process")
    try:
        build(openmp=True)
    except (OSError, subprocess.CalledProcessError):
        return False
    _use_openmp = True
    return True


def threads() -> int:
    """Threads the loaded build runs its loops on (1 for the plain build)."""
    if not _use_openmp:
        return 1
    env = os.environ.get("OMP_NUM_THREADS")
    return int(env) if env and env.isdigit() else (os.cpu_count() or 1)


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("dealias_strict", C.c_int),
                ("Lx", C.c_double), ("Ly", C.c_double), ("Lz", C.c_double),
                ("nu", C.c_double), ("eta", C.c_double), ("cfl", C.c_double),
                ("dt_fixed", C.c_double), ("dt_max", C.c_double),
                ("mean_mode", C.c_int), ("pad_", C.c_int),
                ("u_inf", C.c_double * 3),
                ("sponge_c", C.c_double), ("sponge_width", C.c_double * 3),
                ("layer_width", C.c_double * 3),
                ("time_scheme", C.c_int), ("pad2_", C.c_int)]


_F = C.c_double * MAX_FOURIER


class Insect(C.Structure):
    _fields_ = [("body_type", C.c_int), ("nwings", C.c_int), ("profile", C.c_int),
                ("nfourier", C.c_int), ("c_smth", C.c_double),
                ("x_cntr", C.c_double * 3), ("u_cntr", C.c_double * 3),
                ("psi", C.c_double), ("beta", C.c_double), ("gamma", C.c_double),
                ("psi_dot", C.c_double), ("beta_dot", C.c_double), ("gamma_dot", C.c_double),
                ("body_a", C.c_double), ("body_b", C.c_double),
                ("pivot_l", C.c_double * 3), ("pivot_r", C.c_double * 3),
                ("eta_stroke", C.c_double),
                ("wing_c_le", C.c_double), ("wing_c_te", C.c_double),
                ("wing_R", C.c_double), ("wing_h", C.c_double), ("freq", C.c_double),
                ("phi_a0", C.c_double), ("phi_a", _F), ("phi_b", _F),
                ("alpha_a0", C.c_double), ("alpha_a", _F), ("alpha_b", _F),
                ("theta_a0", C.c_double), ("theta_a", _F), ("theta_b", _F),
                ("head_x0", C.c_double * 3), ("head_r", C.c_double),
                ("eye_x0", C.c_double * 3), ("eye_r", C.c_double),
                ("wing_shape", C.c_int), ("ncontour", C.c_int),
                ("contour_xc", C.c_double), ("contour_yc", C.c_double),
                ("contour_a0", C.c_double), ("contour_a", C.c_double * MAX_CONTOUR),
                ("contour_b", C.c_double * MAX_CONTOUR),
                ("J_wing", C.c_double * 6),
                ("free_flight", C.c_int), ("pad3_", C.c_int),
                ("mass", C.c_double), ("gravity", C.c_double), ("J_body", C.c_double * 3),
                ("dof", C.c_double * 6), ("quat", C.c_double * 4), ("Omega_body", C.c_double * 3),
                ("body_arc", C.c_double * 3)]


class Scalars(C.Structure):
    _fields_ = [("t", C.c_double), ("dt_prev", C.c_double), ("n", C.c_int64),
                ("Is_prev", (C.c_double * 3) * 3), ("Js_prev", (C.c_double * 3) * 3),
                ("body_rhs_prev", C.c_double * 13)]


class Frames(C.Structure):
    _fields_ = [("M_body", C.c_double * 9), ("Omega_b_g", C.c_double * 3),
                ("M_stroke", (C.c_double * 9) * 2), ("M_wing", (C.c_double * 9) * 2),
                ("Omega_w_b", (C.c_double * 3) * 2), ("Omega_w_w", (C.c_double * 3) * 2),
                ("dOmega_w_w", (C.c_double * 3) * 2),
                ("pivot_g", (C.c_double * 3) * 2),
                ("phi", C.c_double), ("alpha", C.c_double), ("theta", C.c_double),
                ("phi_dot", C.c_double), ("alpha_dot", C.c_double), ("theta_dot", C.c_double),
                ("phi_ddot", C.c_double), ("alpha_ddot", C.c_double), ("theta_ddot", C.c_double)]


_lib = None
_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_cp = np.ctypeslib.ndpointer(dtype=np.complex128, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build(openmp=_use_openmp))
        L = _lib
        L.orc_fft1.argtypes = [C.c_int, _cp, C.c_int]
        L.orc_fft3_r2c.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _cp]
        L.orc_fft3_c2r.argtypes = [C.c_int, C.c_int, C.c_int, _cp, _dp]
        L.orc_dft3_r2c.argtypes = [C.c_int, C.c_int, C.c_int, _dp, _cp]
        L.orc_rot_x.argtypes = [C.c_double, _dp]
        L.orc_rot_y.argtypes = [C.c_double, _dp]
        L.orc_rot_z.argtypes = [C.c_double, _dp]
        L.orc_frames_at.argtypes = [C.POINTER(Insect), C.c_double, C.POINTER(Frames)]
        L.orc_mask_profile.argtypes = [C.c_int, C.c_double, C.c_double]
        L.orc_mask_profile.restype = C.c_double
        L.orc_solid_at.argtypes = [C.POINTER(Insect), C.POINTER(Frames), C.c_double, _dp,
                                   C.POINTER(C.c_double), C.POINTER(C.c_int), _dp]
        L.orc_mask_grid.argtypes = [C.POINTER(Params), C.POINTER(Insect), C.c_double,
                                    _dp, _ip, _dp]
        L.orc_dealias.argtypes = [C.POINTER(Params), _cp, C.c_int]
        L.orc_project.argtypes = [C.POINTER(Params), _cp]
        L.orc_curl.argtypes = [C.POINTER(Params), _cp, _cp]
        L.orc_forward.argtypes = [C.POINTER(Params), _dp, _cp, C.c_int]
        L.orc_inverse.argtypes = [C.POINTER(Params), _cp, _dp, C.c_int]
        L.orc_set_state.argtypes = [C.POINTER(Params), _dp, _cp, _cp, C.POINTER(Scalars)]
        L.orc_get_state.argtypes = [C.POINTER(Params), _cp, _dp]
        L.orc_sponge_term.argtypes = [C.POINTER(Params), _cp, _cp]
        L.orc_sponge_mask.argtypes = [C.POINTER(Params), _dp]
        L.orc_sponge_mask.restype = C.c_double
        L.orc_layer_mask.argtypes = [C.POINTER(Params), _dp]
        L.orc_layer_mask.restype = C.c_double
        L.orc_body_distance.argtypes = [C.POINTER(Insect), _dp]
        L.orc_body_distance.restype = C.c_double
        L.orc_wing_distance.argtypes = [C.POINTER(Insect), _dp]
        L.orc_wing_distance.restype = C.c_double
        L.orc_quat_from_angles.argtypes = [C.c_double, C.c_double, C.c_double, C.POINTER(C.c_double)]
        L.orc_body_rhs.argtypes = [C.POINTER(Insect), _dp, _dp, _dp]
        L.orc_wing_power.argtypes = [C.POINTER(Insect), C.POINTER(Frames), _dp, _dp, _dp]
        L.orc_rhs.argtypes = [C.POINTER(Params), C.POINTER(Insect), C.c_double, _cp, _cp, _dp]
        L.orc_rhs.restype = C.c_int
        L.orc_physical_fields.argtypes = [C.POINTER(Params), C.POINTER(Insect), C.c_double, _cp,
                                          _dp]
        L.orc_ab2_update.argtypes = [C.POINTER(Params), _cp, _cp, _cp, C.c_double,
                                     C.c_double, C.c_int64]
        L.orc_step.argtypes = [C.POINTER(Params), C.POINTER(Insect), _cp, _cp,
                               C.POINTER(Scalars), _dp]
        L.orc_step.restype = C.c_int
    return _lib


# ---------------------------------------------------------------- marshalling

def make_params(cfg: dict) -> Params:
    p = Params()
    p.nx, p.ny, p.nz = cfg["n"]
    p.Lx, p.Ly, p.Lz = cfg["L"]
    p.nu = cfg["nu"]
    p.eta = cfg["eta"]
    p.cfl = cfg.get("cfl", 0.1)
    p.dt_fixed = cfg.get("dt_fixed", 0.0)
    p.dt_max = cfg.get("dt_max", 0.0)
    p.dealias_strict = int(cfg.get("dealias_strict", 0))
    p.mean_mode = 1 if cfg.get("mean_mode", "fixed") == "free" else 0
    p.u_inf[:] = cfg.get("u_inf", (0.0, 0.0, 0.0))
    p.sponge_c = cfg.get("sponge_c", 0.0)
    p.sponge_width[:] = cfg.get("sponge_width", (0.0, 0.0, 0.0))
    p.layer_width[:] = cfg.get("layer_width", (0.0, 0.0, 0.0))
    p.time_scheme = {"ab2": 0, "rk4": 1}[cfg.get("time_scheme", "ab2")]
    return p


def make_insect(d: dict | None) -> Insect | None:
    if d is None:
        return None
    s = Insect()
    s.body_type = {"none": 0, "sphere": 1, "ellipsoid": 2, "curved": 3}[d.get("body", "none")]
    if "body_arc" in d:
        s.body_arc[:] = d["body_arc"]     # (radius, x centre, z centre), body frame
    s.nwings = d.get("nwings", 0)
    s.profile = {"cos": 0, "tanh": 1}[d.get("profile", "cos")]
    s.c_smth = d.get("c_smth", 1.0)
    s.x_cntr[:] = d.get("x_cntr", (0, 0, 0))
    s.u_cntr[:] = d.get("u_cntr", (0, 0, 0))
    s.psi, s.beta, s.gamma = d.get("body_angles", (0, 0, 0))
    s.psi_dot, s.beta_dot, s.gamma_dot = d.get("body_rates", (0, 0, 0))
    s.body_a, s.body_b = d.get("body_axes", (0.0, 0.0))
    s.pivot_l[:] = d.get("pivot_l", (0, 0, 0))
    s.pivot_r[:] = d.get("pivot_r", (0, 0, 0))
    s.eta_stroke = d.get("eta_stroke", 0.0)
    s.wing_c_le, s.wing_c_te, s.wing_R, s.wing_h = d.get("wing", (0, 0, 0, 0))
    s.freq = d.get("freq", 1.0)
    kin = d.get("kinematics", {})
    nf = 0
    for name in ("phi", "alpha", "theta"):
        a0, a, b = kin.get(name, (0.0, [], []))
        setattr(s, name + "_a0", a0)
        arr_a, arr_b = getattr(s, name + "_a"), getattr(s, name + "_b")
        for i, v in enumerate(a):
            arr_a[i] = v
        for i, v in enumerate(b):
            arr_b[i] = v
        nf = max(nf, len(a), len(b))
    s.nfourier = nf
    if "head" in d:
        s.head_x0[:], s.head_r = d["head"]
    if "eyes" in d:
        s.eye_x0[:], s.eye_r = d["eyes"]
    if "J_wing" in d:
        s.J_wing[:] = d["J_wing"]
    if "free_flight" in d:
        ff = d["free_flight"]
        s.free_flight = 1
        s.mass, s.gravity = ff["mass"], ff.get("gravity", 0.0)
        s.J_body[:] = ff["J_body"]
        s.dof[:] = ff.get("dof", (1.0,) * 6)
        s.Omega_body[:] = ff.get("Omega_body", (0.0, 0.0, 0.0))
        eps = (C.c_double * 4)()
        lib().orc_quat_from_angles(s.psi, s.beta, s.gamma, eps)
        s.quat[:] = eps[:]
    if "contour" in d:
        c = d["contour"]
        s.wing_shape = 1
        s.contour_xc, s.contour_yc = c["center"]
        s.contour_a0 = c["a0"]
        for i, v in enumerate(c.get("a", [])):
            s.contour_a[i] = v
        for i, v in enumerate(c.get("b", [])):
            s.contour_b[i] = v
        s.ncontour = max(len(c.get("a", [])), len(c.get("b", [])))
    return s


def _ins_ptr(ins):
    return C.byref(ins) if ins is not None else None


def half_shape(n):
    nx, ny, nz = n
    return (nz, ny, nx // 2 + 1)


def fft3_r2c(u: np.ndarray) -> np.ndarray:
    nz, ny, nx = u.shape
    out = np.zeros((nz, ny, nx // 2 + 1), np.complex128)
    lib().orc_fft3_r2c(nx, ny, nz, np.ascontiguousarray(u, np.float64), out)
    return out


def fft3_c2r(uh: np.ndarray, nx: int) -> np.ndarray:
    nz, ny, _ = uh.shape
    out = np.zeros((nz, ny, nx), np.float64)
    lib().orc_fft3_c2r(nx, ny, nz, np.ascontiguousarray(uh, np.complex128), out)
    return out


def dft3_r2c(u: np.ndarray) -> np.ndarray:
    nz, ny, nx = u.shape
    out = np.zeros((nz, ny, nx // 2 + 1), np.complex128)
    lib().orc_dft3_r2c(nx, ny, nz, np.ascontiguousarray(u, np.float64), out)
    return out


def fft1(x: np.ndarray, sign: int) -> np.ndarray:
    a = np.ascontiguousarray(x, np.complex128).copy()
    lib().orc_fft1(a.size, a, sign)
    return a


def rot(axis: str, xi: float) -> np.ndarray:
    R = np.zeros(9)
    getattr(lib(), "orc_rot_" + axis)(xi, R)
    return R.reshape(3, 3)


def frames(insect: dict, t: float) -> dict:
    ins = make_insect(insect)
    fr = Frames()
    lib().orc_frames_at(C.byref(ins), t, C.byref(fr))
    m = lambda a: np.array(a[:]).reshape(3, 3)
    return {
        "M_body": m(fr.M_body), "Omega_b_g": np.array(fr.Omega_b_g[:]),
        "M_stroke": [m(fr.M_stroke[i]) for i in range(2)],
        "M_wing": [m(fr.M_wing[i]) for i in range(2)],
        "Omega_w_b": [np.array(fr.Omega_w_b[i][:]) for i in range(2)],
        "Omega_w_w": [np.array(fr.Omega_w_w[i][:]) for i in range(2)],
        "dOmega_w_w": [np.array(fr.dOmega_w_w[i][:]) for i in range(2)],
        "pivot_g": [np.array(fr.pivot_g[i][:]) for i in range(2)],
        "angles": (fr.phi, fr.alpha, fr.theta),
        "rates": (fr.phi_dot, fr.alpha_dot, fr.theta_dot),
    }


def mask_profile(profile: str, delta: float, h: float) -> float:
    return lib().orc_mask_profile({"cos": 0, "tanh": 1}[profile], delta, h)


def solid_at(insect: dict, t: float, h: float, x) -> tuple:
    ins = make_insect(insect)
    fr = Frames()
    lib().orc_frames_at(C.byref(ins), t, C.byref(fr))
    chi, col = C.c_double(), C.c_int()
    us = np.zeros(3)
    lib().orc_solid_at(C.byref(ins), C.byref(fr), h, np.asarray(x, np.float64), C.byref(chi),
                       C.byref(col), us)
    return chi.value, col.value, us


def mask_grid(cfg: dict, insect: dict, t: float):
    p, ins = make_params(cfg), make_insect(insect)
    nx, ny, nz = cfg["n"]
    chi = np.zeros((nz, ny, nx))
    col = np.zeros((nz, ny, nx), np.int32)
    us = np.zeros((3, nz, ny, nx))
    lib().orc_mask_grid(C.byref(p), C.byref(ins), t, chi, col, us)
    return chi, col, us


class Spectral:
    """Operators on half-spectrum fields uh[c][z][y][x] of a configuration."""

    def __init__(self, cfg: dict):
        self.cfg = cfg
        self.p = make_params(cfg)
        self.n = tuple(cfg["n"])

    def shape(self, ncomp=3):
        return (ncomp,) + half_shape(self.n)

    def forward(self, u):
        ncomp = u.shape[0]
        out = np.zeros(self.shape(ncomp), np.complex128)
        lib().orc_forward(C.byref(self.p), np.ascontiguousarray(u, np.float64), out, ncomp)
        return out

    def inverse(self, uh):
        ncomp = uh.shape[0]
        nx, ny, nz = self.n
        out = np.zeros((ncomp, nz, ny, nx))
        lib().orc_inverse(C.byref(self.p), np.ascontiguousarray(uh), out, ncomp)
        return out

    def dealias(self, fh):
        f = np.ascontiguousarray(fh).copy()
        lib().orc_dealias(C.byref(self.p), f, f.shape[0])
        return f

    def project(self, fh):
        f = np.ascontiguousarray(fh).copy()
        lib().orc_project(C.byref(self.p), f)
        return f

    def curl(self, uh):
        out = np.zeros_like(uh)
        lib().orc_curl(C.byref(self.p), np.ascontiguousarray(uh), out)
        return out

    def rhs(self, uh, t=0.0, insect=None):
        nh = np.zeros_like(uh)
        sums = np.zeros(NSUMS)
        ins = make_insect(insect)
        lib().orc_rhs(C.byref(self.p), _ins_ptr(ins), t, np.ascontiguousarray(uh), nh, sums)
        return nh, sums

    def sponge_term(self, vh):
        """-(i k x vh) / (C_sp |k|^2), zero at k = 0 (no truncation, no projection)."""
        sh = np.zeros_like(vh)
        lib().orc_sponge_term(C.byref(self.p), np.ascontiguousarray(vh), sh)
        return sh

    def sponge_mask(self, X):
        return lib().orc_sponge_mask(C.byref(self.p), np.ascontiguousarray(X, dtype=np.float64))

    def layer_mask(self, X):
        return lib().orc_layer_mask(C.byref(self.p), np.ascontiguousarray(X, dtype=np.float64))

    def physical_fields(self, uh, t=0.0, insect=None):
        """[14][nz][ny][nx]: u, omega, chi, colour, u_s, u x omega - chi/C_eta (u - u_s)."""
        nx, ny, nz = self.n
        out = np.zeros((14, nz, ny, nx))
        ins = make_insect(insect)
        lib().orc_physical_fields(C.byref(self.p), _ins_ptr(ins), t, np.ascontiguousarray(uh), out)
        return out

    def ab2_update(self, uh, nh, nh_prev, dt, dt_prev, n):
        u = np.ascontiguousarray(uh).copy()
        lib().orc_ab2_update(C.byref(self.p), u, np.ascontiguousarray(nh),
                             np.ascontiguousarray(nh_prev), dt, dt_prev, n)
        return u


class Simulation:
    """The oracle's time stepper: state u_hat, N_hat^{n-1}, t, dt_{n-1}, n."""

    def __init__(self, cfg: dict, insect: dict | None = None):
        self.cfg = cfg
        self.p = make_params(cfg)
        self.ins = make_insect(insect)
        self.sp = Spectral(cfg)
        self.uh = np.zeros(self.sp.shape(), np.complex128)
        self.nh_prev = np.zeros_like(self.uh)
        self.s = Scalars()
        self.rows = []

    def set_state(self, u: np.ndarray):
        lib().orc_set_state(C.byref(self.p), np.ascontiguousarray(u, np.float64), self.uh,
                            self.nh_prev, C.byref(self.s))
        self.rows = []

    def get_state(self) -> np.ndarray:
        nx, ny, nz = self.cfg["n"]
        out = np.zeros((3, nz, ny, nx))
        lib().orc_get_state(C.byref(self.p), self.uh, out)
        return out

    def step(self, n: int = 1):
        for _ in range(n):
            row = np.zeros(ROW_COLS)
            rc = lib().orc_step(C.byref(self.p), _ins_ptr(self.ins), self.uh, self.nh_prev,
                                C.byref(self.s), row)
            if rc == 2:
                raise ValueError("oracle: free flight runs with the AB2 scheme only")
            if rc != 0:
                raise FloatingPointError("oracle: non-finite value in the step")
            self.rows.append(row)
        return np.array(self.rows[-n:])

    @property
    def t(self):
        return self.s.t

    @property
    def nstep(self):
        return self.s.n


def body_distance(insect: dict, xb):
    """Signed distance of the body at a body-frame point (Sec. 3.2)."""
    return lib().orc_body_distance(C.byref(make_insect(insect)), np.ascontiguousarray(xb, np.float64))


def wing_distance(insect: dict, xw):
    """Signed distance of a wing at a wing-frame point (Sec. 3.4)."""
    return lib().orc_wing_distance(C.byref(make_insect(insect)), np.ascontiguousarray(xw, np.float64))


def quat_from_angles(psi, beta, gamma):
    """Initial free-flight quaternion of the yaw, pitch and roll angles (Sec. 3.6)."""
    eps = (C.c_double * 4)()
    lib().orc_quat_from_angles(psi, beta, gamma, eps)
    return np.array(eps[:])


def body_rhs(insect: dict, F, m_b, state=None):
    """Right-hand side of the 13 free-flight equations for a descriptor whose
    body state is `state` = (x, u, quat, Omega) or the descriptor's own."""
    ins = make_insect(insect)
    if state is not None:
        x, u, q, w = state
        ins.x_cntr[:], ins.u_cntr[:], ins.quat[:], ins.Omega_body[:] = x, u, q, w
    f = np.zeros(13)
    lib().orc_body_rhs(C.byref(ins), np.ascontiguousarray(F, np.float64),
                       np.ascontiguousarray(m_b, np.float64), f)
    return f


def wing_power(insect: dict, t: float, row=None):
    """(P_aero[2], P_inert[2]) of the wings at time t (Sec. 3.5) for a force row
    (zeros if none: only the inertial power is then meaningful)."""
    ins = make_insect(insect)
    fr = Frames()
    lib().orc_frames_at(C.byref(ins), t, C.byref(fr))
    r = np.zeros(ROW_COLS) if row is None else np.ascontiguousarray(row, np.float64)
    pa, pi = np.zeros(2), np.zeros(2)
    lib().orc_wing_power(C.byref(ins), C.byref(fr), r, pa, pi)
    return pa, pi
