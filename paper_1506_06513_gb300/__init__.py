"""Python binding of libflusi (include/flusi.h).

The ``flusi_*`` functions below have the C names and marshal arguments only;
every step of the solver runs in the CUDA kernels of ``libflusi.so``.
PyTorch supplies device memory (the workspace) and the stream.  There is no
fallback: importing the binding fails loudly when the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libflusi.so")

FLUSI_OK, FLUSI_EINVAL, FLUSI_ENOMEM, FLUSI_ECUDA, FLUSI_ENONFINITE, FLUSI_ETIMEOUT, FLUSI_ESTATE = range(7)
FLUSI_FP64, FLUSI_FP32, FLUSI_FP32_SPLITBF16, FLUSI_FP32_SPLITBF16X3 = 0, 1, 2, 3
# Solver precision names and their flusi_precision values
PRECISIONS = {"fp64": FLUSI_FP64, "fp32": FLUSI_FP32, "bf16x2": FLUSI_FP32_SPLITBF16,
              "bf16x3": FLUSI_FP32_SPLITBF16X3}
FLUSI_HOST_FP64, FLUSI_HOST_FP32, FLUSI_DEVICE = 0, 1, 2
MAX_FOURIER = 8
MAX_CONTOUR = 32
FORCE_COLS = 26
PROFILE_MAX = 40
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENONFINITE", "ETIMEOUT", "ESTATE"]


class FlusiError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"flusi {STATUS_NAMES[code] if 0 <= code < 7 else code}: {msg}")
        self.code = code


class Options(C.Structure):
    _fields_ = [("cfl", C.c_double), ("dt_fixed", C.c_double), ("dt_max", C.c_double),
                ("u_inf", C.c_double * 3), ("mean_mode", C.c_int), ("dealias_strict", C.c_int),
                ("force_ring", C.c_int), ("use_graph", C.c_int),
                ("sponge_c", C.c_double), ("sponge_width", C.c_double * 3),
                ("layer_width", C.c_double * 3),
                ("time_scheme", C.c_int), ("use_tma", C.c_int)]


MAX_STAGES = 8
TUNING_SETTINGS = ("y_plan", "zf_plan", "y_cols", "z_cols", "x_kernel", "y_pair")


class Tuning(C.Structure):
    _fields_ = [("y_plan", C.c_int), ("zf_plan", C.c_int), ("y_cols", C.c_int), ("z_cols", C.c_int),
                ("x_kernel", C.c_int), ("y_pair", C.c_int),
                ("y_radix", C.c_int * MAX_STAGES), ("zf_radix", C.c_int * MAX_STAGES),
                ("zi_radix", C.c_int * MAX_STAGES),
                ("y_tile_cols", C.c_int), ("z_tile_cols", C.c_int), ("x_line_kernel", C.c_int),
                ("y_paired", C.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k in TUNING_SETTINGS}
        for k in ("y_radix", "zf_radix", "zi_radix"):
            d[k] = [r for r in getattr(self, k) if r]
        for k in ("y_tile_cols", "z_tile_cols", "x_line_kernel", "y_paired"):
            d[k] = getattr(self, k)
        return d


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
                ("wing_c_le", C.c_double), ("wing_c_te", C.c_double), ("wing_R", C.c_double),
                ("wing_h", C.c_double), ("freq", C.c_double),
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
                ("free_flight", C.c_int), ("pad2_", C.c_int),
                ("mass", C.c_double), ("gravity", C.c_double), ("J_body", C.c_double * 3),
                ("dof", C.c_double * 6), ("quat", C.c_double * 4), ("Omega_body", C.c_double * 3),
                ("body_arc", C.c_double * 3)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libflusi.so is not built ({LIB_PATH}); run __graft_entry__.build() "
                          "or python -m paper_1506_06513_gb300._build")
    lib = C.CDLL(LIB_PATH)
    h, vp, dp, ip = C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_int
    sig = {
        "flusi_create": ([ip, ip, ip, dp, C.c_double, C.c_double, ip, C.POINTER(h)], ip),
        "flusi_default_options": ([C.POINTER(Options)], None),
        "flusi_set_options": ([h, C.POINTER(Options)], ip),
        "flusi_workspace_bytes": ([h, C.POINTER(C.c_size_t)], ip),
        "flusi_bind": ([h, vp, C.c_size_t, vp], ip),
        "flusi_set_state": ([h, vp, ip], ip),
        "flusi_set_kinematics": ([h, C.POINTER(Insect)], ip),
        "flusi_get_body": ([h, dp], ip),
        "flusi_debug_wait_timeout": ([h, C.c_double], ip),
        "flusi_debug_inject": ([h, ip, ip, ip, ip, C.c_double, C.c_double], ip),
        "flusi_step": ([h, ip], ip),
        "flusi_sync": ([h], ip),
        "flusi_forces": ([h, dp, ip, C.POINTER(C.c_int), C.POINTER(C.c_longlong)], ip),
        "flusi_get_state": ([h, vp, ip, dp, C.POINTER(C.c_longlong)], ip),
        "flusi_get_spectrum": ([h, dp], ip),
        "flusi_debug_fields": ([h, vp], ip),
        "flusi_profile_step": ([h, ip, dp, C.POINTER(C.c_char_p), C.POINTER(C.c_int)], ip),
        "flusi_kernels_per_step": ([h, C.POINTER(C.c_int)], ip),
        "flusi_forces_async": ([h, dp, ip, C.POINTER(C.c_int), C.POINTER(C.c_longlong)], ip),
        "flusi_get_tuning": ([h, C.POINTER(Tuning)], ip),
        "flusi_set_tuning": ([h, C.POINTER(Tuning)], ip),
        "flusi_autotune": ([h, ip, C.c_char_p, C.POINTER(Tuning)], ip),
        "flusi_penalization_sums_noalloc": ([ip, ip, ip, dp, C.c_double, C.POINTER(Insect), C.c_double,
                                             vp, dp, vp], ip),
        "flusi_checkpoint_bytes": ([h, C.POINTER(C.c_size_t)], ip),
        "flusi_save": ([h, vp, C.c_size_t], ip),
        "flusi_load": ([h, vp, C.c_size_t], ip),
        "flusi_ensemble_create": ([C.POINTER(h), ip, vp, C.POINTER(h)], ip),
        "flusi_ensemble_step": ([h, ip], ip),
        "flusi_ensemble_destroy": ([h], ip),
        "flusi_ensemble_batches": ([h, C.POINTER(C.c_int), C.POINTER(C.c_int)], ip),
        "flusi_destroy": ([h], ip),
        "flusi_last_error": ([h], C.c_char_p),
        "flusi_build_id": ([], C.c_char_p),
        "flusi_fma_peak": ([ip, C.c_double, dp, dp], ip),
        "flusi_divergence": ([h, dp, dp], ip),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    from . import _build
    built, want = lib.flusi_build_id().decode(), _build.source_hash()
    if built != want:
        raise ImportError(f"libflusi.so was built from other sources (build id {built}, sources {want}); "
                          "rebuild it with __graft_entry__.build() or python -m paper_1506_06513_gb300._build")
    return lib


lib = _load()


def _check(handle, rc):
    if rc != FLUSI_OK:
        raise FlusiError(rc, lib.flusi_last_error(handle).decode())
    return rc


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------- C-ABI calls

def flusi_create(n, L, nu, eta, precision):
    out = C.c_void_p()
    Ls = (C.c_double * 3)(*L)
    rc = lib.flusi_create(int(n[0]), int(n[1]), int(n[2]), Ls, float(nu), float(eta),
                          int(precision), C.byref(out))
    _check(None, rc)
    return out


def flusi_default_options():
    o = Options()
    lib.flusi_default_options(C.byref(o))
    return o


def flusi_set_options(h, opt: Options):
    return _check(h, lib.flusi_set_options(h, C.byref(opt)))


def flusi_workspace_bytes(h):
    b = C.c_size_t()
    _check(h, lib.flusi_workspace_bytes(h, C.byref(b)))
    return b.value


def flusi_bind(h, dev_ptr: int, nbytes: int, stream: int):
    return _check(h, lib.flusi_bind(h, C.c_void_p(dev_ptr), nbytes, C.c_void_p(stream)))


def flusi_set_state(h, u, where):
    """u: numpy float64/float32 array (host) or an int device pointer."""
    ptr = C.c_void_p(u) if isinstance(u, int) else C.c_void_p(u.ctypes.data)
    return _check(h, lib.flusi_set_state(h, ptr, where))


def flusi_set_kinematics(h, insect: Insect | None):
    return _check(h, lib.flusi_set_kinematics(h, C.byref(insect) if insect is not None else None))


def flusi_get_body(h):
    """Body state (x_cntr, u_cntr, quat, Omega_body) as a dict of arrays."""
    y = np.zeros(13)
    _check(h, lib.flusi_get_body(h, _dptr(y)))
    return {"x_cntr": y[0:3], "u_cntr": y[3:6], "quat": y[6:10], "Omega_body": y[10:13]}


def flusi_step(h, n):
    return _check(h, lib.flusi_step(h, int(n)))


def flusi_sync(h):
    return _check(h, lib.flusi_sync(h))


def flusi_forces(h, cap=4096):
    rows = np.zeros((cap, FORCE_COLS))
    count, lost = C.c_int(), C.c_longlong()
    _check(h, lib.flusi_forces(h, _dptr(rows), cap, C.byref(count), C.byref(lost)))
    return rows[: count.value].copy(), lost.value


def flusi_forces_async(h, rows: np.ndarray, start: int = 0):
    """Enqueue the copy of the undrained rows into rows[start:] (a C-contiguous
    float64 array [cap][FORCE_COLS], best page-locked) without waiting; returns
    (count, lost).  The rows are valid after the next synchronizing call."""
    if rows.dtype != np.float64 or rows.ndim != 2 or rows.shape[1] != FORCE_COLS or not rows.flags.c_contiguous:
        raise ValueError("rows must be a C-contiguous float64 array [cap][FORCE_COLS]")
    if not 0 <= start <= rows.shape[0]:
        raise ValueError("start outside rows")
    count, lost = C.c_int(), C.c_longlong()
    ptr = C.cast(C.c_void_p(rows.ctypes.data + start * FORCE_COLS * 8), C.POINTER(C.c_double))
    _check(h, lib.flusi_forces_async(h, ptr, rows.shape[0] - start, C.byref(count), C.byref(lost)))
    return count.value, lost.value


def flusi_get_state(h, out, where):
    """out: numpy array (host) or an int device pointer; returns (t, step)."""
    ptr = C.c_void_p(out) if isinstance(out, int) else C.c_void_p(out.ctypes.data)
    t, step = C.c_double(), C.c_longlong()
    _check(h, lib.flusi_get_state(h, ptr, where, C.byref(t), C.byref(step)))
    return t.value, step.value


def flusi_get_spectrum(h, shape):
    nz, ny, hx = shape
    out = np.zeros((3, nz, ny, hx, 2))
    _check(h, lib.flusi_get_spectrum(h, _dptr(out)))
    return out[..., 0] + 1j * out[..., 1]


def flusi_debug_fields(h, dev_ptr: int):
    return _check(h, lib.flusi_debug_fields(h, C.c_void_p(dev_ptr)))


def flusi_profile_step(h, n):
    ms = (C.c_double * PROFILE_MAX)()
    names = (C.c_char_p * PROFILE_MAX)()
    nk = C.c_int()
    _check(h, lib.flusi_profile_step(h, int(n), ms, names, C.byref(nk)))
    return {names[i].decode(): ms[i] for i in range(nk.value)}


def flusi_kernels_per_step(h):
    c = C.c_int()
    _check(h, lib.flusi_kernels_per_step(h, C.byref(c)))
    return c.value


def flusi_get_tuning(h):
    """Plans, tile caps and x kernel of the handle, with what the passes take."""
    t = Tuning()
    _check(h, lib.flusi_get_tuning(h, C.byref(t)))
    return t.as_dict()


def flusi_set_tuning(h, **settings):
    """Change some of y_plan, zf_plan, y_cols, z_cols, x_kernel; the others keep
    their current values."""
    t = Tuning()
    _check(h, lib.flusi_get_tuning(h, C.byref(t)))
    for k, v in settings.items():
        if k not in TUNING_SETTINGS:
            raise ValueError(f"unknown tuning setting {k!r}")
        setattr(t, k, int(v))
    return _check(h, lib.flusi_set_tuning(h, C.byref(t)))


def flusi_autotune(h, steps=5, cache_path=None):
    t = Tuning()
    path = os.fsencode(cache_path) if cache_path is not None else None
    _check(h, lib.flusi_autotune(h, int(steps), path, C.byref(t)))
    return t.as_dict()


NOALLOC_SUMS = 38
NOALLOC_MAX_POINTS = 1024 ** 3


def flusi_penalization_sums_noalloc(n, L, eta, insect: Insect | None, t, u_dev: int, stream: int = 0):
    """Force, moment, energy and CFL sums of a device FP64 velocity field
    [3][nz][ny][nx] without a handle or any allocation (see flusi.h).
    Returns FLUSI_NOALLOC_SUMS doubles."""
    out = np.zeros(NOALLOC_SUMS)
    Ls = (C.c_double * 3)(*L)
    rc = lib.flusi_penalization_sums_noalloc(int(n[0]), int(n[1]), int(n[2]), Ls, float(eta),
                                             C.byref(insect) if insect is not None else None,
                                             float(t), C.c_void_p(u_dev), _dptr(out),
                                             C.c_void_p(stream))
    _check(None, rc)
    return out


def flusi_checkpoint_bytes(h):
    b = C.c_size_t()
    _check(h, lib.flusi_checkpoint_bytes(h, C.byref(b)))
    return b.value


def flusi_save(h):
    """The handle's checkpoint as a numpy uint8 array (see flusi.h)."""
    buf = np.empty(flusi_checkpoint_bytes(h), np.uint8)
    _check(h, lib.flusi_save(h, C.c_void_p(buf.ctypes.data), buf.nbytes))
    return buf


def flusi_load(h, buf: np.ndarray):
    buf = np.ascontiguousarray(buf, np.uint8)
    return _check(h, lib.flusi_load(h, C.c_void_p(buf.ctypes.data), buf.nbytes))


def flusi_ensemble_create(handles, stream: int):
    arr = (C.c_void_p * len(handles))(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    out = C.c_void_p()
    _check(None, lib.flusi_ensemble_create(arr, len(handles), C.c_void_p(stream), C.byref(out)))
    return out


def flusi_ensemble_step(e, n):
    return _check(None, lib.flusi_ensemble_step(e, int(n)))


def flusi_ensemble_destroy(e):
    return lib.flusi_ensemble_destroy(e)


def flusi_destroy(h):
    return lib.flusi_destroy(h)


def flusi_last_error(h):
    return lib.flusi_last_error(h).decode()


def flusi_debug_inject(h, component, mode, value):
    """Write the complex `value` into the state's coefficient of `mode` =
    (mx, my, mz) of velocity component `component` (a host-side fault
    injector for the failure path)."""
    v = complex(value)
    _check(h, lib.flusi_debug_inject(h, int(component), int(mode[0]), int(mode[1]), int(mode[2]),
                                     v.real, v.imag))


def flusi_divergence(h):
    """(max |k . u_hat|, max |k| |u_hat|) of the state, reduced in FP64 on the device."""
    d, ku = C.c_double(), C.c_double()
    _check(h, lib.flusi_divergence(h, C.byref(d), C.byref(ku)))
    return d.value, ku.value


def flusi_build_id():
    return lib.flusi_build_id().decode()


def flusi_fma_peak(fp64, target_ms=30.0):
    """Measured FMA rate of the current device in flop/s, and the timed launch's ms."""
    f, ms = C.c_double(), C.c_double()
    _check(None, lib.flusi_fma_peak(int(fp64), float(target_ms), C.byref(f), C.byref(ms)))
    return f.value, ms.value


# ------------------------------------------------------------ descriptors

def make_insect(d: dict | None) -> Insect | None:
    """flusi_insect from a plain descriptor dict (see workloads)."""
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
    nf = 0
    for name in ("phi", "alpha", "theta"):
        a0, a, b = d.get("kinematics", {}).get(name, (0.0, [], []))
        setattr(s, name + "_a0", a0)
        for i, v in enumerate(a):
            getattr(s, name + "_a")[i] = v
        for i, v in enumerate(b):
            getattr(s, name + "_b")[i] = v
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
        s.quat[:] = ff.get("quat", (0.0, 0.0, 0.0, 0.0))   # zero: from the body angles
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


def make_options(cfg: dict) -> Options:
    o = flusi_default_options()
    o.cfl = cfg.get("cfl", 0.1)
    o.dt_fixed = cfg.get("dt_fixed", 0.0)
    o.dt_max = cfg.get("dt_max", 0.0)
    o.u_inf[:] = cfg.get("u_inf", (0.0, 0.0, 0.0))
    o.mean_mode = 1 if cfg.get("mean_mode", "fixed") == "free" else 0
    o.dealias_strict = int(cfg.get("dealias_strict", 0))
    o.force_ring = int(cfg.get("force_ring", 4096))
    o.use_graph = int(cfg.get("use_graph", 1))
    o.sponge_c = cfg.get("sponge_c", 0.0)
    o.sponge_width[:] = cfg.get("sponge_width", (0.0, 0.0, 0.0))
    o.layer_width[:] = cfg.get("layer_width", (0.0, 0.0, 0.0))
    o.time_scheme = {"ab2": 0, "rk4": 1}[cfg.get("time_scheme", "ab2")]
    o.use_tma = int(cfg.get("use_tma", 1))
    return o


class Solver:
    """A bound handle: torch owns the workspace and the stream."""

    def __init__(self, cfg: dict, insect: dict | None = None, precision: str = "fp64",
                 device: int = 0, stream=None):
        import torch
        self.torch = torch
        self.cfg = cfg
        if precision not in PRECISIONS:
            raise ValueError(f"precision must be one of {sorted(PRECISIONS)}")
        self.prec = PRECISIONS[precision]
        self.n = tuple(cfg["n"])
        self.h = flusi_create(self.n, cfg["L"], cfg["nu"], cfg["eta"], self.prec)
        flusi_set_options(self.h, make_options(cfg))
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        nbytes = flusi_workspace_bytes(self.h)
        self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        base = self.ws.data_ptr()
        aligned = (base + 255) // 256 * 256
        flusi_bind(self.h, aligned, nbytes, self.stream.cuda_stream)
        self.insect = make_insect(insect)
        if self.insect is not None:
            flusi_set_kinematics(self.h, self.insect)

    def set_state(self, u):
        """u: numpy [3][nz][ny][nx] (float64 or float32) or a torch CUDA tensor
        in the solver's precision."""
        nx, ny, nz = self.n
        if isinstance(u, np.ndarray):
            if u.shape != (3, nz, ny, nx):
                raise ValueError(f"u has shape {u.shape}, expected {(3, nz, ny, nx)}")
            if u.dtype not in (np.float64, np.float32):
                u = u.astype(np.float64)
            where = FLUSI_HOST_FP64 if u.dtype == np.float64 else FLUSI_HOST_FP32
            flusi_set_state(self.h, np.ascontiguousarray(u), where)
        else:
            u = self._device_array(u)
            self.stream.wait_stream(self.torch.cuda.current_stream(self.device))
            flusi_set_state(self.h, u.data_ptr(), FLUSI_DEVICE)
            self.stream.synchronize()   # u (possibly a converted copy) is read asynchronously

    def _device_array(self, u):
        """A contiguous CUDA tensor [3][nz][ny][nx] in the handle's precision on
        the handle's device (the C call reads exactly that many values)."""
        torch = self.torch
        nx, ny, nz = self.n
        if tuple(u.shape) != (3, nz, ny, nx):
            raise ValueError(f"u has shape {tuple(u.shape)}, expected {(3, nz, ny, nx)}")
        dt = torch.float64 if self.prec == FLUSI_FP64 else torch.float32
        return u.to(device=self.device, dtype=dt).contiguous()

    def step(self, n=1):
        flusi_step(self.h, n)

    def sync(self):
        flusi_sync(self.h)

    def forces(self, cap=4096):
        return flusi_forces(self.h, cap)

    def forces_async(self, rows, start=0):
        """Enqueue the copy of the undrained force rows into rows[start:]
        (page-locked float64 [cap][FORCE_COLS]); returns (count, lost).  The
        rows are there after the next synchronizing call."""
        return flusi_forces_async(self.h, rows, start)

    def body(self):
        """Free flight: the body state after the enqueued steps (synchronizes)."""
        return flusi_get_body(self.h)

    def get_state(self, dtype=np.float64):
        nx, ny, nz = self.n
        out = np.zeros((3, nz, ny, nx), dtype)
        t, step = flusi_get_state(self.h, out, FLUSI_HOST_FP64 if dtype == np.float64 else FLUSI_HOST_FP32)
        return out, t, step

    def get_state_device(self, out):
        torch = self.torch
        nx, ny, nz = self.n
        dt = torch.float64 if self.prec == FLUSI_FP64 else torch.float32
        if (tuple(out.shape) != (3, nz, ny, nx) or out.dtype != dt or not out.is_contiguous()
                or out.device != self.device):
            raise ValueError("out must be a contiguous [3][nz][ny][nx] tensor in the handle's "
                             "precision on the handle's device")
        return flusi_get_state(self.h, out.data_ptr(), FLUSI_DEVICE)

    def divergence(self):
        """(max |k . u_hat|, max |k| |u_hat|) over the kept modes, FP64 on the device."""
        return flusi_divergence(self.h)

    def get_spectrum(self):
        nx, ny, nz = self.n
        return flusi_get_spectrum(self.h, (nz, ny, nx // 2 + 1))

    def debug_fields(self):
        torch = self.torch
        nx, ny, nz = self.n
        dt = torch.float64 if self.prec == FLUSI_FP64 else torch.float32
        out = torch.empty((14, nz, ny, nx), dtype=dt, device=self.device)
        flusi_debug_fields(self.h, out.data_ptr())
        self.stream.synchronize()
        return out

    def profile(self, n=3):
        return flusi_profile_step(self.h, n)

    def tuning(self):
        return flusi_get_tuning(self.h)

    def set_tuning(self, **settings):
        flusi_set_tuning(self.h, **settings)

    def autotune(self, steps=5, cache_path=None):
        """Time the plan, tile and x-kernel choices and keep the fastest
        (flusi_autotune); the state is left as it was."""
        return flusi_autotune(self.h, steps, cache_path)

    def save(self):
        """Checkpoint for an exact restart (flusi_save)."""
        return flusi_save(self.h)

    def load(self, buf):
        flusi_load(self.h, buf)

    def close(self):
        if self.h:
            flusi_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """Independent solvers stepped together: one CUDA graph holds one step of
    every member (flusi_ensemble_*).  The solvers stay owned by the caller."""

    def __init__(self, solvers, stream=None):
        import torch
        self.solvers = list(solvers)
        dev = self.solvers[0].device
        self.stream = stream if stream is not None else torch.cuda.Stream(device=dev)
        self.e = flusi_ensemble_create([s.h for s in self.solvers], self.stream.cuda_stream)

    def step(self, n=1):
        flusi_ensemble_step(self.e, n)

    def batches(self):
        """(groups sharing launches, members in them) of the captured step."""
        g, m = C.c_int(), C.c_int()
        _check(None, lib.flusi_ensemble_batches(self.e, C.byref(g), C.byref(m)))
        return g.value, m.value

    def sync(self):
        self.stream.synchronize()

    def close(self):
        if self.e:
            flusi_ensemble_destroy(self.e)
            self.e = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
