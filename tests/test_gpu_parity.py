"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

FP64 tolerances follow from double rounding through O(log N) FFT stages and
20 time steps: 1e-11 relative L2 for the state, 1e-10 for force rows.  FP32
results are compared at 1e-5 relative L2 per step (single-precision FFTs of
length <= 1024 accumulate ~log2(N) * 6e-8 relative error per transform).
"""
import math

import numpy as np
import pytest

import oracle
from parity import check_state
import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from conftest import build_flusi
    return build_flusi()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def rows_err(a, b):
    """max deviation of force/moment/energy columns relative to each column's scale"""
    a, b = np.asarray(a), np.asarray(b)
    err = 0.0
    for j in range(b.shape[1]):
        scale = max(np.abs(b[:, j]).max(), 1e-300)
        err = max(err, np.abs(a[:, j] - b[:, j]).max() / scale if scale > 1e-12 else
                  np.abs(a[:, j] - b[:, j]).max())
    return err


def free_cfg(n, L, **kw):
    c = {"n": n, "L": L, "nu": 0.02, "eta": 1e-2, "dt_fixed": 1e-3, "mean_mode": "fixed"}
    c.update(kw)
    return c


GRIDS = [((16, 16, 16), (2 * math.pi,) * 3), ((24, 16, 12), (3.0, 2.0, 1.5)),
         ((48, 36, 24), (4.0, 3.0, 2.0)), ((8, 32, 18), (1.0, 4.0, 2.25))]


@pytest.mark.parametrize("n,L", GRIDS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_transform_round_trip(fl, n, L, prec):
    """set_state (r2c x, y, z + 2/3 rule + projection) and get_state (c2r)."""
    cfg = free_cfg(n, L)
    u0 = workloads.random_field(n, seed=sum(n))
    ref = oracle.Simulation(cfg, None)
    ref.set_state(u0)
    sim = fl.Solver(cfg, None, precision=prec)
    sim.set_state(u0)
    uh = sim.get_spectrum()
    u, t, step = sim.get_state()
    sim.close()
    tol = 1e-13 if prec == "fp64" else 3e-6
    check_state(uh, ref.uh, tol)
    check_state(u, ref.get_state(), tol)
    assert t == 0.0 and step == 0


ODD = [((54, 27, 81), (2.0, 1.0, 3.0)),     # radix 3 only; odd y and z lengths
       ((18, 9, 27), (2.0, 1.0, 3.0))]      # the smallest odd lengths (9 = 3 3)


@pytest.mark.parametrize("n,L", ODD)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_odd_lengths(fl, n, L, prec):
    """Odd y and z lengths (radix-3 plans only, K = (n - 1)/3 ... kept modes
    around an odd row count): the transform round trip, then three steps with
    a sphere against the oracle."""
    cfg = free_cfg(n, L, u_inf=(0.3, 0.0, 0.0))
    u0 = workloads.random_smooth_field(n, 3, mean=(0.3, 0.0, 0.0))
    ins = workloads.sphere(tuple(0.5 * x for x in L), 0.3 * min(L), profile="cos")
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    tol = 1e-13 if prec == "fp64" else 3e-6
    check_state(sim.get_spectrum(), ref.uh, tol)
    rows_ref = ref.step(3)
    sim.step(3)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    sim.close()
    tol_u, tol_f = (1e-11, 1e-10) if prec == "fp64" else (3e-5, 1e-4)
    check_state(u, ref.get_state(), tol_u)
    assert rel_l2(rows[:, 2:20], rows_ref[:, 2:20]) <= tol_f


def test_device_in_and_out(fl):
    """set_state / get_state with device arrays; the field's modes are all
    inside the 2/3-rule set of this grid, so it comes back unchanged."""
    import torch
    n, L = (24, 32, 18), (3.0, 4.0, 2.25)
    cfg = free_cfg(n, L)
    u0 = workloads.shear_waves(n, L)
    for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
        sim = fl.Solver(cfg, None, precision=prec)
        sim.set_state(torch.tensor(u0, dtype=dt, device="cuda"))
        out = torch.empty((3,) + tuple(reversed(n)), dtype=dt, device="cuda")
        sim.get_state_device(out)
        sim.close()
        tol = 1e-13 if prec == "fp64" else 3e-6
        check_state(out.cpu().numpy(), u0, tol)


CASES = {
    "tg_sphere_16": lambda: workloads.config_tg_sphere(16),
    "insect_32": lambda: (dict(workloads.config_model_insect(32)[0]),
                          workloads.model_insect((4.0, 4.0, 4.0), (32, 32, 32))),
    "realistic_48x32x32": lambda: (dict(workloads.config_model_insect(32)[0], n=(48, 32, 32)),
                                   workloads.realistic_insect((4.0, 4.0, 4.0), (48, 32, 32))),
    "curved_48x32x32": lambda: (dict(workloads.config_model_insect(32)[0], n=(48, 32, 32)),
                                workloads.curved_insect((4.0, 4.0, 4.0), (48, 32, 32))),
    "wing_48x36x24": lambda: ({"n": (48, 36, 24), "L": (4.0, 3.0, 2.0), "nu": 0.0125664,
                               "eta": 2.5e-3, "cfl": 0.1, "mean_mode": "fixed",
                               "init": ("random_smooth", 5)},
                              dict(workloads.single_wing((4.0, 3.0, 2.0), (48, 36, 24)),
                                   x_cntr=(2.0, 1.5, 1.0))),
}


def _initial(cfg):
    if cfg["init"][0] == "uniform":
        return workloads.initial_field(cfg) + 0.05 * workloads.random_smooth_field(cfg["n"], 1)
    return workloads.initial_field(cfg)


@pytest.mark.parametrize("case", sorted(CASES))
def test_physical_fields(fl, case):
    """u, omega, chi, colour, u_s and u x omega - chi/C_eta (u - u_s) on the
    grid (the fused x pass) against the oracle, at t = 0 and after 3 steps."""
    cfg, ins = CASES[case]()
    u0 = _initial(cfg)
    sim = fl.Solver(cfg, ins, precision="fp64")
    sim.set_state(u0)
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    for nsteps in (0, 3):
        if nsteps:
            sim.step(nsteps)
            ref.step(nsteps)
        got = sim.debug_fields().cpu().numpy()
        exp = oracle.Spectral(cfg).physical_fields(ref.uh, ref.t, ins)
        for sl, name in ((slice(0, 3), "u"), (slice(3, 6), "omega"), (slice(11, 14), "nl")):
            check_state(got[sl], exp[sl], 1e-11, name)
        assert np.abs(got[6] - exp[6]).max() <= 1e-12, "chi"
        solid = exp[6] > 1e-9
        # where two parts give the same chi (the mirror plane) either colour is valid
        assert (got[7][solid] == exp[7][solid]).mean() > 0.995, "colour"
        same = solid & (got[7] == exp[7])
        for c in range(3):
            assert np.abs(got[8 + c][same] - exp[8 + c][same]).max(initial=0) <= 1e-12, "u_s"
    sim.close()


def test_c0_full_step_fp64(fl):
    """Taylor-Green + fixed sphere, 32^3, FP64, dt = 1e-3, 20 steps."""
    cfg, ins = workloads.config_tg_sphere(32)
    u0 = workloads.initial_field(cfg)
    sim = fl.Solver(cfg, ins, precision="fp64")
    sim.set_state(u0)
    sim.step(20)
    rows, lost = sim.forces()
    u, t, step = sim.get_state()
    sim.close()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(20)
    assert step == 20 and lost == 0 and rows.shape == (20, 26)
    assert abs(t - ref.t) <= 1e-15
    check_state(u, ref.get_state(), 1e-11)
    assert rows_err(rows, ref_rows) <= 1e-10


@pytest.mark.parametrize("case", ["insect_32", "realistic_48x32x32", "curved_48x32x32", "wing_48x36x24"])
def test_flapping_steps_fp64(fl, case):
    """Moving wings, adaptive dt (CFL and dt <= C_eta), unsteady corrections."""
    cfg, ins = CASES[case]()
    u0 = _initial(cfg)
    sim = fl.Solver(cfg, ins, precision="fp64")
    sim.set_state(u0)
    sim.step(12)
    rows, _ = sim.forces()
    u, t, step = sim.get_state()
    sim.close()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(12)
    assert np.abs(rows[:, 1] - ref_rows[:, 1]).max() <= 1e-13 * ref_rows[:, 1].max()
    check_state(u, ref.get_state(), 1e-10)
    assert rows_err(rows, ref_rows) <= 1e-8


def test_fp32_matches_oracle(fl):
    cfg, ins = CASES["insect_32"]()
    u0 = _initial(cfg)
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    sim.step(1)
    ref_rows = ref.step(1)
    check_state(sim.get_state()[0], ref.get_state(), 1e-5)
    sim.step(9)
    ref_rows = np.vstack([ref_rows, ref.step(9)])
    rows, _ = sim.forces()
    check_state(sim.get_state()[0], ref.get_state(), 1e-4)
    assert rel_l2(rows[:, 2:20], ref_rows[:, 2:20]) <= 1e-4
    sim.close()


def test_relaxation_free_mean(fl):
    """chi = 1 everywhere, u_s = 0, free mean: the AB2 relaxation recurrence."""
    cfg = {"n": (8, 8, 8), "L": (2 * math.pi,) * 3, "nu": 0.01, "eta": 0.05, "dt_fixed": 0.004,
           "mean_mode": "free"}
    ins = workloads.sphere((0.0, 0.0, 0.0), 100.0, profile="cos")
    u0 = np.array([0.3, -0.2, 0.5])
    sim = fl.Solver(cfg, ins, precision="fp64")
    sim.set_state(workloads.uniform(cfg["n"], u0))
    sim.step(10)
    hist = [u0, u0 * (1 - 0.004 / 0.05)]
    for _ in range(9):
        hist.append(hist[-1] - 0.08 * (1.5 * hist[-1] - 0.5 * hist[-2]))
    got = sim.get_state()[0].mean(axis=(1, 2, 3))
    sim.close()
    assert np.abs(got - hist[10]).max() <= 1e-14


def test_graph_and_eager_are_identical(fl):
    cfg, ins = CASES["insect_32"]()
    u0 = _initial(cfg)
    out = []
    for g in (1, 0):
        c = dict(cfg, use_graph=g)
        sim = fl.Solver(c, ins, precision="fp32")
        sim.set_state(u0)
        sim.step(5)
        out.append(sim.get_state()[0])
        sim.close()
    assert np.array_equal(out[0], out[1])


def test_nonfinite_state_is_reported(fl):
    cfg, ins = CASES["insect_32"]()
    u0 = _initial(cfg)
    bad = u0.copy()
    bad[1, 3, 4, 5] = np.nan
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(bad)
    sim.step(2)
    with pytest.raises(fl.FlusiError) as e:
        sim.sync()
    assert e.value.code == fl.FLUSI_ENONFINITE
    with pytest.raises(fl.FlusiError) as e:
        sim.step(1)
    assert e.value.code == fl.FLUSI_ESTATE
    sim.set_state(u0)
    sim.step(1)
    sim.sync()
    rows, _ = sim.forces()
    assert rows.shape[0] == 1 and np.isfinite(rows).all()
    sim.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16x2"])
def test_fault_injected_into_a_running_state(fl, prec):
    """A host-side injector (flusi_debug_inject) writes a coefficient of the
    live state between steps: a finite value is stepped on (the state then
    differs from the clean run); a NaN makes the next step report
    FLUSI_ENONFINITE at the next synchronizing call, later steps are refused
    with FLUSI_ESTATE, and a new state recovers the handle."""
    if prec == "bf16x2":
        n, L = (256, 16, 12), (4.0, 0.25, 0.1875)
        cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
               "u_inf": (0.3, 0.0, 0.0)}
        ins = workloads.sphere((2.0, 0.125, 0.09375), 0.06, profile="cos")
        u0 = workloads.random_smooth_field(n, 3, mean=(0.3, 0.0, 0.0))
    else:
        cfg, ins = CASES["insect_32"]()
        u0 = _initial(cfg)
    clean = fl.Solver(cfg, ins, precision=prec)
    clean.set_state(u0)
    clean.step(4)
    u_clean = clean.get_state()[0]
    clean.close()
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    sim.step(3)
    fl.flusi_debug_inject(sim.h, 1, (1, -2, 1), 0.01)
    sim.step(1)
    u = sim.get_state()[0]
    assert np.isfinite(u).all() and not np.array_equal(u, u_clean)
    with pytest.raises(fl.FlusiError) as e:
        fl.flusi_debug_inject(sim.h, 0, (cfg["n"][0] // 3 + 1, 0, 0), 1.0)
    assert e.value.code == fl.FLUSI_EINVAL
    fl.flusi_debug_inject(sim.h, 2, (2, 1, -1), complex(float("nan"), 0.0))
    sim.step(2)
    with pytest.raises(fl.FlusiError) as e:
        sim.sync()
    assert e.value.code == fl.FLUSI_ENONFINITE
    with pytest.raises(fl.FlusiError) as e:
        sim.step(1)
    assert e.value.code == fl.FLUSI_ESTATE
    sim.set_state(u0)
    sim.step(1)
    rows, _ = sim.forces()
    assert np.isfinite(rows).all()
    sim.close()


@pytest.mark.parametrize("n", [(32, 32, 32), (48, 36, 24), (24, 96, 64), (16, 1024, 12)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_tma_tiles_equal_copied_tiles(fl, n, prec):
    """The y and z passes give identical results whether their tiles arrive by
    TMA boxes or by 16-byte copies (use_tma 1 and 0): the same data lands in
    the same shared-memory slots before the same transforms.  The grids cover
    one- and multi-plane y tiles, radix 3, and split boxes (n = 1024)."""
    L = tuple(0.125 * m for m in n)
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0)}
    ins = workloads.sphere(tuple(0.5 * x for x in L), 0.3 * min(L), profile="cos")
    u0 = workloads.random_smooth_field(n, 5, mean=(0.3, 0.0, 0.0))
    out = []
    for tma in (1, 0):
        sim = fl.Solver(dict(cfg, use_tma=tma), ins, precision=prec)
        sim.set_state(u0)
        sim.step(3)
        out.append((sim.forces()[0], sim.get_state()[0], sim.get_spectrum()))
        sim.close()
    (ra, ua, sa), (rb, ub, sb) = out
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub) and np.array_equal(sa, sb)


@pytest.mark.parametrize("n", [(48, 36, 24), (96, 24, 12)])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_strict_dealiasing(fl, n, prec):
    """dealias_strict keeps |m| < n/3 (one mode fewer per axis where 3 divides
    n): five steps with a sphere in a mean flow against the oracle with the
    same option, and the dropped modes zero in the spectrum."""
    L = tuple(0.125 * m for m in n)
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0), "dealias_strict": 1}
    ins = workloads.sphere(tuple(0.5 * x for x in L), 0.3 * min(L), profile="cos")
    u0 = workloads.random_smooth_field(n, 7, mean=(0.3, 0.0, 0.0))
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    sim.step(5)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    uh = sim.get_spectrum()
    sim.close()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(5)
    tol_u, tol_r = (1e-11, 1e-9) if prec == "fp64" else (2e-5, 1e-4)
    check_state(u, ref.get_state(), tol_u)
    assert rows_err(rows, ref_rows) <= tol_r
    for ax, m in ((2, np.arange(n[0] // 2 + 1)), (1, np.fft.fftfreq(n[1], 1.0 / n[1])),
                  (0, np.fft.fftfreq(n[2], 1.0 / n[2]))):
        nn = n[2 - ax]
        drop = np.abs(m) >= nn / 3
        sl = [slice(None)] * 4
        sl[1 + ax] = drop
        assert np.abs(uh[tuple(sl)]).max(initial=0.0) == 0.0


def test_bounded_wait_reports_a_timeout(fl):
    """A device-side wait that runs out (an mbarrier nothing completes, the
    bounded wait of the TMA tile loads) sets FLUSI_ETIMEOUT in the status word:
    the next synchronizing call reports it within the bound, the handle refuses
    steps until a new state is set, and the context stays usable."""
    import time
    cfg, ins = CASES["insect_32"]()
    u0 = _initial(cfg)
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    sim.step(2)
    sim.sync()
    assert fl.lib.flusi_debug_wait_timeout(sim.h, 0.0) == fl.FLUSI_EINVAL
    t0 = time.perf_counter()
    assert fl.lib.flusi_debug_wait_timeout(sim.h, 20.0) == fl.FLUSI_OK
    with pytest.raises(fl.FlusiError) as e:
        sim.sync()
    assert e.value.code == fl.FLUSI_ETIMEOUT
    assert time.perf_counter() - t0 < 5.0
    with pytest.raises(fl.FlusiError) as e:
        sim.step(1)
    assert e.value.code == fl.FLUSI_ESTATE
    sim.set_state(u0)
    sim.step(3)
    rows, _ = sim.forces()
    assert rows.shape[0] == 3 and np.isfinite(rows).all()
    sim.close()


def test_force_ring_drain(fl):
    cfg, ins = CASES["insect_32"]()
    cfg = dict(cfg, force_ring=4)
    u0 = _initial(cfg)
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    sim.step(3)
    rows, lost = sim.forces()
    assert rows.shape[0] == 3 and lost == 0
    sim.step(10)
    rows2, lost2 = sim.forces()
    assert rows2.shape[0] == 4 and lost2 == 6
    assert np.all(np.diff(rows2[:, 0]) > 0) and rows2[0, 0] > rows[-1, 0]
    rows3, lost3 = sim.forces()
    assert rows3.shape[0] == 0 and lost3 == 0
    sim.close()


def shear_waves_curl(n, L, pts):
    """Closed-form curl of workloads.shear_waves at integer grid points: component
    c is a_c f_c(k_c . x + phase_c) with f = (sin, cos, sin), so
    d_j u_c = a_c f_c'(arg) k_cj."""
    X = [pts[:, j] * L[j] / n[j] for j in range(3)]
    grad = np.zeros((3, 3, len(pts)))     # grad[c, j] = d u_c / d x_j
    deriv = (np.cos, lambda a: -np.sin(a), np.cos)
    for c, (a, m, ph) in enumerate(workloads.SHEAR_WAVES):
        k = [2 * math.pi * m[j] / L[j] for j in range(3)]
        arg = k[0] * X[0] + k[1] * X[1] + k[2] * X[2] + ph
        for j in range(3):
            grad[c, j] = a * deriv[c](arg) * k[j]
    return np.array([grad[2, 1] - grad[1, 2], grad[0, 2] - grad[2, 0], grad[1, 0] - grad[0, 1]])


def test_bench_configuration_sampled(fl):
    """The 512^3 FP32 model-insect step in the benchmark's launch
    configuration, checked where the oracle can follow point by point:
    the mask and solid velocity at sampled grid points near the insect, the
    band-limited initial field, its vorticity and the nonlinear term
    u x omega - chi/C_eta (u - u_s) at sampled points, and the kinetic energy of
    the first force row against its closed form."""
    import torch
    cfg, ins = workloads.config_model_insect(512)
    n, L = cfg["n"], cfg["L"]
    u0 = workloads.shear_waves(n, L, mean=cfg["u_inf"]).astype(np.float32)
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    del u0
    rng = np.random.default_rng(512)
    pts = np.column_stack([rng.integers(0, 512, 4000) for _ in range(3)])
    # the insect sits at the box centre: body |x - 2| <= 0.5, wings |y - 2| <= 1.15
    near = np.column_stack([rng.integers(lo, hi, 4000)
                            for lo, hi in ((192, 320), (128, 384), (236, 276))])
    pts = np.vstack([pts, near])
    f = sim.debug_fields()
    vals = f[:, pts[:, 2], pts[:, 1], pts[:, 0]].double().cpu().numpy()
    del f
    torch.cuda.empty_cache()
    exact = workloads.shear_waves(n, L, mean=cfg["u_inf"], points=pts)
    assert np.abs(vals[0:3] - exact).max() <= 2e-5
    dx = L[0] / n[0]
    h = dx
    for i, (ix, iy, iz) in enumerate(pts):
        chi, col, us = oracle.solid_at(ins, 0.0, h, (ix * dx, iy * dx, iz * dx))
        assert abs(vals[6, i] - chi) <= 2e-5
        if chi > 1e-3 and vals[7, i] == col:
            assert np.abs(vals[8:11, i] - us).max() <= 1e-4
    assert (vals[6] > 0.5).sum() > 20
    # vorticity and nonlinear term at t = 0 against the closed-form curl of the waves
    om = shear_waves_curl(n, L, pts)
    assert np.abs(vals[3:6] - om).max() <= 1e-4 * np.abs(om).max()
    nl = np.cross(exact.T, om.T).T
    solid_pts = np.zeros(len(pts), bool)
    for i, (ix, iy, iz) in enumerate(pts):
        chi, col, us = oracle.solid_at(ins, 0.0, h, (ix * dx, iy * dx, iz * dx))
        if chi > 0:
            solid_pts[i] = True
            nl[:, i] -= chi / cfg["eta"] * (exact[:, i] - np.asarray(us))
    fluid = ~solid_pts
    assert np.abs(vals[11:14, fluid] - nl[:, fluid]).max() <= 1e-4 * np.abs(nl[:, fluid]).max()
    assert np.abs(vals[11:14, solid_pts] - nl[:, solid_pts]).max() <= 1e-4 * np.abs(nl[:, solid_pts]).max()
    sim.step(1)
    rows, _ = sim.forces()
    ek = workloads.shear_waves_energy(L, mean=cfg["u_inf"])
    assert abs(rows[0, 20] - ek) <= 1e-5 * ek
    assert rows[0, 1] == pytest.approx(min(0.1 * dx / rows[0, 21], cfg["eta"]), rel=1e-12)
    # properties of the stepped state at full size: solenoidal, 2/3-rule
    # truncated, the mean held at u_inf
    uh = sim.get_spectrum()
    mx = np.arange(n[0] // 2 + 1)
    my = np.fft.fftfreq(n[1], 1.0 / n[1])
    mz = np.fft.fftfreq(n[2], 1.0 / n[2])
    div = np.zeros(uh.shape[1:], complex)
    for c, (m, ax) in enumerate(((mx, 2), (my, 1), (mz, 0))):
        shape = [1, 1, 1]
        shape[ax] = -1
        div += (2 * np.pi / L[c]) * m.reshape(shape) * uh[c]
    kmax = 2 * np.pi * (n[0] // 3) / L[0] * np.sqrt(3)
    assert np.abs(div).max() <= 1e-6 * kmax * np.abs(uh).max()
    del div
    drop = (np.abs(mz)[:, None, None] > n[2] // 3) | (np.abs(my)[None, :, None] > n[1] // 3) | \
           (mx[None, None, :] > n[0] // 3)
    assert np.abs(uh[:, drop]).max() == 0.0
    assert np.allclose(uh[:, 0, 0, 0], cfg["u_inf"], rtol=0, atol=1e-7)
    del uh, drop
    sim.close()
    _check_first_force_row(cfg, ins, rows[0], (176, 92, 220), (336, 420, 292),
                           lambda pts: workloads.shear_waves(n, L, mean=cfg["u_inf"], points=pts))


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_single_wing_first_row_at_256(fl, prec):
    """The 256^3 single-wing configuration (C1: nx = 256, the nh = 2R^2 x pass
    with R = 8) from rest: its first force row is minus the penalized solid
    velocity, sum -chi u_s dV / C_eta and its moment about the pivot, against
    the oracle's mask over a sub-box that holds the whole wing."""
    cfg, ins = workloads.config_single_wing(256)
    n = cfg["n"]
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(np.zeros((3,) + tuple(reversed(n)), np.float32 if prec == "fp32" else np.float64))
    sim.step(1)
    rows, _ = sim.forces()
    sim.close()
    assert rows[0, 20] == 0.0
    _check_first_force_row(cfg, ins, rows[0], (104, 116, 104), (152, 212, 152),
                           lambda pts: np.zeros((3, len(pts))), parts=(1,),
                           tol=1e-10 if prec == "fp64" else 2e-4)


def test_turbulent_configuration_at_the_largest_size(fl):
    """The 1024^3 FP32 turbulent-inflow workload (the largest grid, the nh = 2R^2
    x pass, split TMA boxes, radix-16 y stages) in the benchmark's launch
    shape: the state after set_state at sampled points against the sum of its
    modes, the first force row's kinetic energy against its closed form, the
    adaptive step against the CFL rule, and a finite state after three steps."""
    import torch
    cfg, ins = workloads.config_turbulent_insect(1024)
    n, L = cfg["n"], cfg["L"]
    u0 = workloads.turbulent_field(n, L, mean=cfg["u_inf"], seed=cfg["init"][1], device="cuda")
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    del u0
    torch.cuda.empty_cache()
    rng = np.random.default_rng(1024)
    pts = np.column_stack([rng.integers(0, 1024, 3000) for _ in range(3)])
    out = torch.empty((3, 1024, 1024, 1024), dtype=torch.float32, device="cuda")
    sim.get_state_device(out)
    idx = [torch.as_tensor(pts[:, a], device="cuda") for a in (2, 1, 0)]
    vals = out[:, idx[0], idx[1], idx[2]].double().cpu().numpy()
    del out, idx
    torch.cuda.empty_cache()
    m, a = workloads.turbulent_modes(L, seed=cfg["init"][1])
    X = pts * (L[0] / n[0])
    k = 2 * np.pi * m / np.asarray(L)
    phase = np.exp(1j * (X @ k.T))                       # (points, modes)
    exact = np.asarray(cfg["u_inf"])[:, None] + 2 * np.real(a.T @ phase.T)
    assert np.abs(vals - exact).max() <= 2e-6
    sim.step(1)
    rows, _ = sim.forces()
    vol = L[0] * L[1] * L[2]
    ek = 0.5 * vol * (sum(c * c for c in cfg["u_inf"]) + 2 * np.sum(np.abs(a) ** 2))
    assert abs(rows[0, 20] - ek) <= 1e-5 * ek
    dx = L[0] / n[0]
    assert rows[0, 1] == pytest.approx(min(0.1 * dx / rows[0, 21], cfg["eta"]), rel=1e-12)
    sim.step(2)
    rows2, _ = sim.forces()
    assert rows2.shape[0] == 2 and np.isfinite(rows2).all()
    sim.close()


def _check_first_force_row(cfg, ins, row, lo, hi, u_at, parts=(0, 1, 2), tol=2e-4):
    """Force and moment of the given parts in the first row of a full-size step
    (the register-resident x pass the benchmark times), against the oracle's
    mask over the sub-box [lo, hi) of grid indices (x, y, z) that holds the
    whole insect and the closed-form initial field u_at(points):
    F = sum chi (u - u_s) dV / C_eta, M = sum r x chi (u - u_s) dV / C_eta
    (no unsteady correction on the first step)."""
    n, L = cfg["n"], cfg["L"]
    dx = L[0] / n[0]
    nsub = tuple(h - l for l, h in zip(lo, hi))
    off = np.array(lo) * dx
    sub = {"n": nsub, "L": tuple(m * dx for m in nsub), "nu": cfg["nu"], "eta": cfg["eta"]}
    shifted = dict(ins, x_cntr=tuple(np.asarray(ins["x_cntr"]) - off))
    chi, col, us = oracle.mask_grid(sub, shifted, 0.0)
    # the sub-box holds the whole insect: nothing on its faces
    for face in (chi[0], chi[-1], chi[:, 0], chi[:, -1], chi[:, :, 0], chi[:, :, -1]):
        assert face.max() == 0.0
    z, y, x = np.meshgrid(*(np.arange(lo[a], hi[a]) for a in (2, 1, 0)), indexing="ij")
    pts = np.column_stack([x.ravel(), y.ravel(), z.ravel()])
    u = u_at(pts)
    X = pts.T * dx
    pen = chi.ravel() * (u - us.reshape(3, -1)) * dx ** 3 / cfg["eta"]
    fr = oracle.frames(ins, 0.0)
    refs = [np.asarray(ins["x_cntr"]), fr["pivot_g"][0], fr["pivot_g"][1]]
    for c in parts:
        sel = col.ravel() == c + 1
        F = pen[:, sel].sum(axis=1)
        M = np.cross((X[:, sel] - refs[c][:, None]).T, pen[:, sel].T).sum(axis=0)
        got_F, got_M = row[2 + 6 * c: 5 + 6 * c], row[5 + 6 * c: 8 + 6 * c]
        assert np.abs(got_F - F).max() <= tol * np.abs(F).max(), c
        assert np.abs(got_M - M).max() <= tol * np.abs(M).max(), c
        assert np.abs(F).max() > 1e-3


WIDE = {"x512": ((512, 16, 12), (8.0, 1.0, 0.75)), "x128": ((128, 24, 16), (4.0, 0.75, 0.5)),
        "x1024": ((1024, 12, 8), (16.0, 1.0, 0.75)), "x256": ((256, 18, 16), (8.0, 0.75, 0.75)),
        "x96": ((96, 18, 12), (4.0, 0.75, 0.5)), "x64": ((64, 18, 12), (4.0, 1.125, 0.75))}
# nx of the register-resident x pass (nh = R^2 or 2 R^2 with R = 16 or 8;
# nh = 4 R with R = 12 or 8, the rectangular form)
SQUARE_NX = (64, 96, 128, 256, 512, 1024)


@pytest.mark.parametrize("name", sorted(WIDE))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_square_half_length_x_pass(fl, name, prec):
    """Grids with nx = 512 and 128 take the x pass whose half-length transform
    is two register-resident radix-16 (radix-8) passes, nx = 1024 and 256 the
    one with a radix-2 step between lane pairs after them, nx = 96 and 64 the
    rectangular one (radix 12 or 8 in registers, then radix 4 across four
    lanes; 216 rows, ragged against 16-row tiles); full steps with a
    sphere, adaptive dt and a mean flow against the oracle."""
    n, L = WIDE[name]
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0)}
    ins = workloads.sphere((L[0] / 2, L[1] / 2, L[2] / 2), 0.35 * min(L[1], L[2]), profile="cos")
    u0 = workloads.random_smooth_field(n, 7, mean=(0.3, 0.0, 0.0))
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    sim.step(5)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    sim.close()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(5)
    tol_u, tol_f = (1e-11, 1e-9) if prec == "fp64" else (2e-5, 1e-4)
    check_state(u, ref.get_state(), tol_u)
    assert rows_err(rows, ref_rows) <= tol_f


WAKE = {"generic_48x36x24": ((48, 36, 24), (4.0, 3.0, 2.0)),
        "square_512x16x12": ((512, 16, 12), (8.0, 1.0, 0.75)),
        "square_128x24x16": ((128, 24, 16), (4.0, 0.75, 0.5)),
        "square_1024x12x8": ((1024, 12, 8), (16.0, 1.0, 0.75)),
        "square_256x18x16": ((256, 18, 16), (8.0, 0.75, 0.75)),
        "rect_96x18x12": ((96, 18, 12), (4.0, 0.75, 0.5)),
        "rect_64x18x12": ((64, 18, 12), (4.0, 1.125, 0.75))}


@pytest.mark.parametrize("name", sorted(WAKE))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_sponge_and_dirichlet_layer(fl, name, prec):
    """Vorticity sponge and Dirichlet inflow layer (Sec. 2.3) with a sphere and
    a mean flow: physical fields at t = 0 and 5 full steps against the oracle,
    on the generic x pass, the square ones and the rectangular ones."""
    n, L = WAKE[name]
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0), "sponge_c": 0.1,
           "sponge_width": (L[0] / 6, L[1] / 8, 0.0), "layer_width": (L[0] / 16, 0.0, L[2] / 8)}
    ins = workloads.sphere((L[0] / 2, L[1] / 2, L[2] / 2), 0.3 * min(L[1], L[2]), profile="cos")
    u0 = workloads.random_smooth_field(n, 9, mean=(0.3, 0.0, 0.0))
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    got = sim.debug_fields().double().cpu().numpy()
    exp = oracle.Spectral(cfg).physical_fields(ref.uh, 0.0, ins)
    tol_f = 1e-11 if prec == "fp64" else 2e-5
    check_state(got[11:14], exp[11:14], tol_f)
    assert fl.flusi_kernels_per_step(sim.h) == (8 if n[0] in SQUARE_NX else 9)
    sim.step(5)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    sim.close()
    ref_rows = ref.step(5)
    tol_u, tol_r = (1e-11, 1e-9) if prec == "fp64" else (3e-5, 1e-4)
    check_state(u, ref.get_state(), tol_u)
    assert rows_err(rows, ref_rows) <= tol_r


RK4_CASES = {"insect_32": None, "square_512x16x12_wake": ((512, 16, 12), (8.0, 1.0, 0.75))}


@pytest.mark.parametrize("name", sorted(RK4_CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_rk4_matches_oracle(fl, name, prec):
    """RK4 with explicit diffusion: four right-hand sides per step with the
    mask at the stage times, adaptive dt with the diffusion cap; the flapping
    model insect, and a sphere with the wake terms on the square x pass."""
    if name == "insect_32":
        cfg, ins = CASES["insect_32"]()
        u0 = _initial(cfg)
    else:
        n, L = RK4_CASES[name]
        cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
               "u_inf": (0.3, 0.0, 0.0), "sponge_c": 0.1, "sponge_width": (L[0] / 6, 0.0, 0.0),
               "layer_width": (L[0] / 16, 0.0, 0.0)}
        ins = workloads.sphere((L[0] / 2, L[1] / 2, L[2] / 2), 0.3 * min(L[1], L[2]), profile="cos")
        u0 = workloads.random_smooth_field(n, 9, mean=(0.3, 0.0, 0.0))
    cfg = dict(cfg, time_scheme="rk4")
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    sim.step(5)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    prof = sim.profile(1)
    sim.close()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(5)
    tol_u, tol_r = (1e-11, 1e-9) if prec == "fp64" else (3e-5, 1e-4)
    check_state(u, ref.get_state(), tol_u)
    assert rows_err(rows, ref_rows) <= tol_r
    assert np.abs(rows[:, 1] - ref_rows[:, 1]).max() <= 1e-6 * ref_rows[:, 1].max()
    assert "update.4" in prof and "kinematics.3" in prof and "scalars" in prof


# Thin slabs whose y or z length is the bench's (512) or the largest one's
# (1024): the default TMA-staged y and z kernels at those lengths (two boxes
# per inverse tile, n/256 boxes forward, split boxes at 1024, the L2 hints
# of the inverse z pass), stepped against the oracle.  Spacing 1/128 as at
# 512^3 over a 4-long box; a sphere in a mean flow, adaptive dt.
BENCH_LENGTHS = {"y512_z512": ((16, 512, 512), (0.125, 4.0, 4.0)),
                 "z1024": ((16, 16, 1024), (0.125, 0.125, 8.0)),
                 "y1024": ((16, 1024, 16), (0.125, 8.0, 0.125))}
_BENCH_REF = {}


def _bench_length_reference(name):
    """The oracle's state and rows after 3 steps (computed once per slab)."""
    if name not in _BENCH_REF:
        n, L = BENCH_LENGTHS[name]
        cfg = {"n": n, "L": L, "nu": 0.004, "eta": 1e-3, "cfl": 0.1, "mean_mode": "fixed",
               "u_inf": (0.25, 0.0, 0.0)}
        ins = workloads.sphere((L[0] / 2, L[1] / 2, L[2] / 2), 0.04, profile="cos")
        u0 = workloads.random_smooth_field(n, 13, amplitude=0.5, mean=(0.25, 0.0, 0.0))
        ref = oracle.Simulation(cfg, ins)
        ref.set_state(u0)
        rows = ref.step(3)
        _BENCH_REF[name] = (cfg, ins, u0, ref.get_state(), rows)
    return _BENCH_REF[name]


@pytest.mark.parametrize("name", sorted(BENCH_LENGTHS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_default_y_and_z_kernels_at_the_bench_lengths(fl, name, prec):
    """Three adaptive steps on slabs with y and z = 512, z = 1024 and y = 1024
    through the default kernels (TMA tiles, unpaired y kernel) against the
    oracle: FP64 state <= 1e-11 and rows <= 1e-10, FP32 3e-5 and 1e-4, with
    the pointwise bound beside the relative L2."""
    cfg, ins, u0, u_ref, rows_ref = _bench_length_reference(name)
    sim = fl.Solver(cfg, ins, precision=prec)
    tune = sim.tuning()
    assert tune["y_pair"] == 0 and tune["y_paired"] == 0
    sim.set_state(u0)
    sim.step(3)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    sim.close()
    tol_u, tol_r = (1e-11, 1e-10) if prec == "fp64" else (3e-5, 1e-4)
    l2, mx = check_state(u, u_ref, tol_u, name)
    print(f"{name} {prec}: u rel L2 {l2:.2e}, pointwise {mx:.2e}, rows {rows_err(rows, rows_ref):.2e}")
    assert rows_err(rows, rows_ref) <= tol_r
    assert np.abs(rows_ref[:, 2:5]).max() > 0   # the sphere meets the grid


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_device_divergence_reduction(fl, prec):
    """flusi_divergence: max |k . u_hat| and max |k| |u_hat| reduced in FP64 on
    the device, against the same maxima taken on the host from the spectrum
    the handle returns; after three flapping-insect steps the state is
    solenoidal to the precision's round-off (the Leray projection of
    Eq. PNST_UP_pressure_poisson_eqn)."""
    cfg, ins = CASES["insect_32"]()
    u0 = _initial(cfg)
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    sim.step(3)
    d, ku = sim.divergence()
    uh = sim.get_spectrum()
    sim.close()
    nx, ny, nz = cfg["n"]
    Lx, Ly, Lz = cfg["L"]
    mx = np.arange(nx // 2 + 1)
    my = np.fft.fftfreq(ny, 1.0 / ny)
    mz = np.fft.fftfreq(nz, 1.0 / nz)
    kz, ky, kx = np.meshgrid(2 * np.pi * mz / Lz, 2 * np.pi * my / Ly, 2 * np.pi * mx / Lx, indexing="ij")
    div = np.abs(kx * uh[0] + ky * uh[1] + kz * uh[2])
    scale = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2) * np.sqrt((np.abs(uh) ** 2).sum(axis=0))
    assert abs(ku - scale.max()) <= 1e-14 * scale.max()
    assert abs(d - div.max()) <= 1e-14 * scale.max()
    assert d <= (1e-14 if prec == "fp64" else 1e-6) * ku


def test_energy_budget_at_the_largest_size(fl):
    """1024^3 FP32 turbulent-inflow insect: the kinetic-energy budget of the
    first step (Sec. 2.1, Eq. PNST_org_momentum with u x omega orthogonal to
    u): dE/dt = sum (u - u_mean) . (u x omega - chi/C_eta (u - u_s)) dV
    - nu sum |omega|^2 dV at t = 0, the mean held fixed.  The right-hand side
    comes from the solver's own physical fields; dE/dt from the force rows'
    E_kin of first steps of two fixed sizes, extrapolated (Richardson) to
    remove the O(dt) term of the finite difference."""
    import torch
    cfg0, ins = workloads.config_turbulent_insect(1024)
    n, L = cfg0["n"], cfg0["L"]
    dV = L[0] * L[1] * L[2] / (n[0] * n[1] * n[2])
    fd, pred = [], None
    for dt in (2e-5, 1e-5):
        cfg = dict(cfg0, dt_fixed=dt)
        u0 = workloads.turbulent_field(n, L, mean=cfg["u_inf"], seed=cfg["init"][1], device="cuda")
        sim = fl.Solver(cfg, ins, precision="fp32")
        sim.set_state(u0)
        del u0
        torch.cuda.empty_cache()
        if pred is None:
            f = sim.debug_fields()            # u, omega, chi, colour, u_s, NL at t = 0
            um = [float(f[c].double().mean()) for c in range(3)]
            work, visc = 0.0, 0.0
            for z0 in range(0, n[2], 128):    # FP64 sums slab by slab
                sl = slice(z0, z0 + 128)
                for c in range(3):
                    work += float(((f[c, sl].double() - um[c]) * f[11 + c, sl].double()).sum())
                    visc += float((f[3 + c, sl].double() ** 2).sum())
            del f
            torch.cuda.empty_cache()
            pred = (work - cfg["nu"] * visc) * dV
        sim.step(2)
        rows, _ = sim.forces()
        sim.close()
        torch.cuda.empty_cache()
        assert rows[0, 1] == dt and rows[1, 1] == dt
        fd.append((rows[1, 20] - rows[0, 20]) / dt)
    dEdt = 2 * fd[1] - fd[0]
    print(f"1024^3 energy budget: predicted {pred:.6e}, measured {dEdt:.6e} "
          f"(first-order differences {fd[0]:.6e}, {fd[1]:.6e})")
    assert abs(pred) > 1e-3
    assert abs(dEdt - pred) <= 1e-2 * abs(pred)
