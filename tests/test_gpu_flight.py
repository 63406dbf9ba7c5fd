"""Wing power (Sec. 3.5) and free flight (Sec. 3.6) on the GPU against the
oracle: the power columns of the force rows, the free-fall closed form, a
free-flying model insect step by step, a body held by its dof mask, and an
exact restart of a free flight."""
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


def rows_err(a, b):
    """max deviation of each column relative to its scale"""
    a, b = np.asarray(a), np.asarray(b)
    err = 0.0
    for j in range(b.shape[1]):
        scale = np.abs(b[:, j]).max()
        d = np.abs(a[:, j] - b[:, j]).max()
        err = max(err, d / scale if scale > 1e-12 else d)
    return err


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _oracle_body(sim):
    return {"x_cntr": np.array(sim.ins.x_cntr[:]), "u_cntr": np.array(sim.ins.u_cntr[:]),
            "quat": np.array(sim.ins.quat[:]), "Omega_body": np.array(sim.ins.Omega_body[:])}


def flying_insect(n=(32, 32, 32), L=(4.0, 4.0, 4.0)):
    """The model insect, pitched and rolled, spinning, heavy enough to stay
    near its start over a few steps (the impulsive start gives forces of ~1e3)."""
    ins = workloads.model_insect(L, n)
    ins["body_angles"] = (0.05, -0.4, 0.1)
    ins["J_wing"] = (2e-2, 1e-3, 2e-2, 1e-4, -3e-4, 2e-4)
    ins["free_flight"] = {"mass": 400.0, "gravity": 9.81, "J_body": (2.0, 5.0, 5.0),
                          "Omega_body": (0.3, -0.2, 0.5)}
    return ins


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_free_fall(fl, prec):
    """A body that covers no grid point falls under gravity alone: u_z = -g t
    and, after the Euler start, z = z0 - g t^2/2 + g dt^2/2; the force rows
    stay zero."""
    n, L = (16, 16, 16), (4.0, 4.0, 4.0)
    g, dt, steps = 9.81, 2e-3, 15
    d = L[0] / n[0]
    x0 = (2.0 + 0.5 * d, 2.0 + 0.5 * d, 2.0 + 0.5 * d)
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "dt_fixed": dt, "mean_mode": "fixed"}
    ins = {"body": "sphere", "nwings": 0, "profile": "cos", "c_smth": 0.1, "body_axes": (1e-6, 0.0),
           "x_cntr": x0, "free_flight": {"mass": 0.7, "gravity": g, "J_body": (1.0, 1.0, 1.0)}}
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(np.zeros((3,) + n[::-1]))
    sim.step(steps)
    rows, _ = sim.forces()
    b = sim.body()
    sim.close()
    t = steps * dt
    assert np.abs(rows[:, 2:26]).max() == 0.0
    assert abs(b["u_cntr"][2] + g * t) <= 1e-13
    assert abs(b["x_cntr"][2] - (x0[2] - 0.5 * g * t * t + 0.5 * g * dt * dt)) <= 1e-13
    assert b["x_cntr"][0] == x0[0] and b["x_cntr"][1] == x0[1]
    assert np.array_equal(b["quat"], [1.0, 0.0, 0.0, 0.0])


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_free_flight_matches_oracle(fl, prec):
    cfg = dict(workloads.config_model_insect(32)[0])
    ins = flying_insect()
    u0 = workloads.initial_field(cfg)
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    start = sim.body()
    sim.step(12)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    b = sim.body()
    sim.close()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    assert np.abs(start["quat"] - np.array(ref.ins.quat[:])).max() <= 1e-15
    ref_rows = ref.step(12)
    rb = _oracle_body(ref)
    tol_u, tol_r, tol_b = (1e-11, 1e-9, 1e-10) if prec == "fp64" else (3e-5, 2e-4, 2e-4)
    check_state(u, ref.get_state(), tol_u)
    assert rows_err(rows, ref_rows) <= tol_r
    # body state: its change over the run, relative to the change
    for key in ("x_cntr", "u_cntr", "quat", "Omega_body"):
        moved = rb[key] - start[key]
        assert np.abs((b[key] - start[key]) - moved).max() <= tol_b * np.abs(moved).max(), key
    assert abs(np.linalg.norm(b["quat"]) - 1.0) <= 1e-15


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_power_columns_tethered(fl, prec):
    """The inertial power depends on the kinematics alone (FP64 in both
    precisions); the aerodynamic power follows the wing moments."""
    cfg = dict(workloads.config_model_insect(32)[0])
    ins = workloads.model_insect(cfg["L"], cfg["n"])
    # with a deviation angle the wing roots swing towards the mirror plane,
    # where the two wings tie and either colour and velocity is valid: the
    # pivots move out so that their layers stay apart
    ins["kinematics"]["theta"] = (0.1, [0.2], [0.15])
    ins["pivot_l"], ins["pivot_r"] = (0.0, 0.3, 0.0), (0.0, -0.3, 0.0)
    ins["J_wing"] = (1e-3, 2e-4, 1.2e-3, 1e-5, -2e-5, 3e-5)
    u0 = workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"])
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    sim.step(6)
    rows, _ = sim.forces()
    sim.close()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(6)
    assert np.abs(rows[:, 24:26] - ref_rows[:, 24:26]).max() <= 1e-12 * np.abs(ref_rows[:, 24:26]).max()
    assert rows_err(rows[:, 22:24], ref_rows[:, 22:24]) <= (1e-9 if prec == "fp64" else 2e-4)
    assert (np.abs(ref_rows[:, 22:26]).max(axis=0) > 0).all()


def test_held_body_is_tethered(fl):
    """dof = 0 and no rotation: the free-flight path (quaternion frame, body
    ODE) reproduces the tethered run up to the rounding of the frame."""
    cfg = dict(workloads.config_model_insect(32)[0])
    ins = workloads.model_insect(cfg["L"], cfg["n"])
    ins["body_angles"] = (0.05, -0.4, 0.1)
    u0 = workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"])
    out = []
    for d in (ins, dict(ins, free_flight={"mass": 1.0, "gravity": 9.81, "J_body": (1.0, 1.0, 1.0),
                                          "dof": (0.0,) * 6})):
        sim = fl.Solver(cfg, d, precision="fp64")
        sim.set_state(u0)
        sim.step(5)
        out.append((sim.forces()[0], sim.get_state()[0], sim.body()))
        sim.close()
    (ra, ua, _), (rb, ub, bb) = out
    assert rows_err(rb, ra) <= 1e-11
    check_state(ub, ua, 1e-13)
    assert np.array_equal(bb["x_cntr"], ins["x_cntr"]) and np.array_equal(bb["u_cntr"], (0, 0, 0))


@pytest.mark.parametrize("graph", [0, 1])
def test_free_flight_restart_bit_for_bit(fl, graph):
    """save after 4 steps, load into a new solver with the same descriptor:
    the next 4 steps, the rows and the body state are those of one run."""
    cfg = dict(workloads.config_model_insect(32)[0], n=(32, 24, 16), L=(4.0, 3.0, 2.0),
               use_graph=graph)
    ins = flying_insect(cfg["n"], cfg["L"])
    ins["x_cntr"] = (2.0, 1.5, 1.0)
    u0 = workloads.initial_field(cfg)
    a = fl.Solver(cfg, ins, precision="fp32")
    a.set_state(u0)
    a.step(8)
    rows_a, _ = a.forces()
    ua = a.get_state()[0]
    ba = a.body()
    a.close()
    b = fl.Solver(cfg, ins, precision="fp32")
    b.set_state(u0)
    b.step(4)
    first, _ = b.forces()
    ck = b.save()
    b.close()
    c = fl.Solver(cfg, ins, precision="fp32")
    c.load(ck)
    c.step(4)
    rest, _ = c.forces()
    uc = c.get_state()[0]
    bc = c.body()
    c.close()
    assert np.array_equal(np.vstack([first, rest]), rows_a)
    assert np.array_equal(uc, ua)
    for key in ba:
        assert np.array_equal(bc[key], ba[key]), key
    assert not np.array_equal(ba["x_cntr"], ins["x_cntr"])


def test_get_body_needs_an_insect(fl):
    cfg = {"n": (16, 16, 16), "L": (1.0, 1.0, 1.0), "nu": 0.01, "eta": 1e-2}
    sim = fl.Solver(cfg, None, precision="fp64")
    with pytest.raises(fl.FlusiError) as e:
        sim.body()
    assert e.value.code == fl.FLUSI_ESTATE
    sim.close()
