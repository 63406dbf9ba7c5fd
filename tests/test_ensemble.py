"""Ensembles of independent runs (flusi_ensemble_*): host-side argument checks,
and on the GPU, members stepped together equal the same members stepped one
by one, bit for bit."""
import ctypes as C

import numpy as np
import pytest

import workloads


@pytest.fixture(scope="module")
def fl():
    from conftest import build_flusi
    return build_flusi()


def test_ensemble_arguments_checked_on_host(fl):
    out = C.c_void_p()
    h = fl.flusi_create((16, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
    arr = (C.c_void_p * 2)(h.value, h.value)
    assert fl.lib.flusi_ensemble_create(arr, 2, None, None) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_ensemble_create(None, 1, None, C.byref(out)) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_ensemble_create(arr, 0, None, C.byref(out)) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_ensemble_create(arr, 2, None, C.byref(out)) == fl.FLUSI_EINVAL
    assert "repeats" in fl.flusi_last_error(None)
    null = (C.c_void_p * 1)(None)
    assert fl.lib.flusi_ensemble_create(null, 1, None, C.byref(out)) == fl.FLUSI_EINVAL
    # a member without a workspace
    assert fl.lib.flusi_ensemble_create(arr, 1, None, C.byref(out)) == fl.FLUSI_ESTATE
    assert "flusi_bind" in fl.flusi_last_error(None)
    assert out.value is None
    assert fl.lib.flusi_ensemble_step(None, 1) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_ensemble_destroy(None) == fl.FLUSI_OK
    fl.flusi_destroy(h)


def test_ensemble_draws_are_seeded():
    a = workloads.config_ensemble(40, 1506)
    b = workloads.config_ensemble(40, 1506)
    assert [c["draw"] for c, _ in a] == [c["draw"] for c, _ in b]
    for cfg, ins in a:
        d = cfg["draw"]
        assert 40 <= d["phi0_deg"] <= 80 and 0.8 <= d["freq"] <= 1.2 and 50 <= d["re"] <= 400
        assert cfg["n"] in workloads.ENSEMBLE_GRIDS
        assert cfg["L"][2] == (8.0 if cfg["n"][2] == 192 else 4.0)
        U = workloads.mean_tip_speed(d["phi0_deg"] * np.pi / 180, d["freq"])
        assert cfg["nu"] == pytest.approx(U * 0.3 / d["re"], rel=1e-14)
        assert ins["x_cntr"] == tuple(0.5 * x for x in cfg["L"])


SMALL = [((16, 16, 16), (4.0, 4.0, 4.0), 55.0, 0.9, 120.0),
         ((24, 16, 12), (4.0, 4.0, 4.0), 70.0, 1.1, 300.0),
         ((16, 16, 32), (4.0, 4.0, 8.0), 45.0, 1.0, 80.0)]


def _member(n, L, phi_deg, f, re):
    phi = phi_deg * np.pi / 180
    cfg = {"n": n, "L": L, "nu": workloads.nu_from_re(re, workloads.mean_tip_speed(phi, f), 0.3),
           "eta": 2.5e-3, "cfl": 0.1, "mean_mode": "fixed"}
    return cfg, workloads.single_wing(L, n, phi_m=phi, freq=f)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_ensemble_equals_one_by_one(fl, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    members = [_member(*m) for m in SMALL]
    dt = np.float64 if prec == "fp64" else np.float32
    fields = [workloads.random_smooth_field(cfg["n"], 3 + i, amplitude=0.2).astype(dt)
              for i, (cfg, _) in enumerate(members)]
    solo = []
    for (cfg, ins), u0 in zip(members, fields):
        s = fl.Solver(cfg, ins, precision=prec)
        s.set_state(u0)
        s.step(6)
        solo.append((s.get_state(dt)[0], s.forces()[0]))
        s.close()
    solvers = [fl.Solver(cfg, ins, precision=prec) for cfg, ins in members]
    for s, u0 in zip(solvers, fields):
        s.set_state(u0)
    ens = fl.Ensemble(solvers)
    ens.step(2)
    ens.step(4)
    for s, (u, rows) in zip(solvers, solo):
        got, t, step = s.get_state(dt)
        assert step == 6
        assert np.array_equal(got, u)
        assert np.array_equal(s.forces()[0], rows)
    # a member whose options change invalidates the captured ensemble graph
    fl.flusi_set_options(solvers[1].h, fl.make_options(members[1][0]))
    with pytest.raises(fl.FlusiError) as e:
        ens.step(1)
    assert e.value.code == fl.FLUSI_ESTATE
    ens.close()
    # so does a member's new tuning; the asynchronous drain counts the
    # ensemble's steps
    ens = fl.Ensemble(solvers)
    ens.step(2)
    rows = torch.zeros((4, fl.FORCE_COLS), dtype=torch.float64).pin_memory().numpy()
    assert fl.flusi_forces_async(solvers[0].h, rows) == (2, 0)
    solvers[0].sync()
    assert np.isfinite(rows[:2]).all() and rows[1, 0] > rows[0, 0] > 0
    solvers[2].set_tuning(y_cols=8)
    with pytest.raises(fl.FlusiError) as e:
        ens.step(1)
    assert e.value.code == fl.FLUSI_ESTATE
    ens.close()
    for s in solvers:
        s.close()


# three groups of members that share their launches (same grid, box, options;
# different kinematics and Reynolds numbers) and one member on its own
SHARED = [((16, 16, 16), (4.0, 4.0, 4.0), 55.0, 0.9, 120.0),
          ((16, 16, 16), (4.0, 4.0, 4.0), 70.0, 1.1, 300.0),
          ((16, 16, 16), (4.0, 4.0, 4.0), 45.0, 1.0, 80.0),
          ((24, 16, 12), (4.0, 4.0, 4.0), 60.0, 0.8, 200.0),
          ((24, 16, 12), (4.0, 4.0, 4.0), 75.0, 1.2, 50.0),
          ((128, 16, 12), (8.0, 1.0, 0.75), 50.0, 1.0, 150.0),
          ((64, 16, 12), (4.0, 1.0, 0.75), 60.0, 1.0, 100.0),
          ((64, 16, 12), (4.0, 1.0, 0.75), 65.0, 0.9, 250.0)]


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_shared_launches_equal_one_by_one(fl, prec):
    """Members of the same grid step as one launch per kernel (gridDim.z =
    members, each block on its own member's buffers); each member's state and
    force rows equal its solo run's bit for bit after 7 adaptive steps (the
    register-resident x pass at nx = 128, its rectangular form at 64, the
    shared-memory one at 16 and 24)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    members = [_member(*m) for m in SHARED]
    members[5] = (members[5][0], dict(members[5][1], x_cntr=(4.0, 0.5, 0.375)))
    for i in (6, 7):
        members[i] = (members[i][0], dict(members[i][1], x_cntr=(2.0, 0.5, 0.375)))
    dt = np.float64 if prec == "fp64" else np.float32
    fields = [workloads.random_smooth_field(cfg["n"], 11 + i, amplitude=0.2).astype(dt)
              for i, (cfg, _) in enumerate(members)]
    solo = []
    for (cfg, ins), u0 in zip(members, fields):
        s = fl.Solver(cfg, ins, precision=prec)
        s.set_state(u0)
        s.step(7)
        solo.append((s.get_state(dt)[0], s.forces()[0]))
        s.close()
    solvers = [fl.Solver(cfg, ins, precision=prec) for cfg, ins in members]
    for s, u0 in zip(solvers, fields):
        s.set_state(u0)
    ens = fl.Ensemble(solvers)
    ens.step(3)
    assert ens.batches() == (3, 7)
    ens.step(4)
    for s, (u, rows) in zip(solvers, solo):
        got, t, step = s.get_state(dt)
        assert step == 7
        assert np.array_equal(got, u)
        assert np.array_equal(s.forces()[0], rows)
    ens.close()
    for s in solvers:
        s.close()
