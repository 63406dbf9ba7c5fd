"""FFT plans, tile shapes and the autotuner on the GPU.

Every setting of flusi_set_tuning computes the same transforms, so each must
meet the oracle at the tolerances of the default path (FP64: 1e-11 relative
L2 for the state, 1e-10 for force rows; FP32: 1e-5 per step).  The grid
128 x 256 x 16 makes every setting take a different path: nx = 128 has a
register-resident x kernel; ny = 256 is 8 8 4 (plans 0, 1) or 16 16 (plan 2);
nz = 16 is 4 4 (plan 0) or 16 (plans 1, 2) in the forward z pass.
"""
import numpy as np
import pytest

import oracle
from parity import check_state
import workloads

pytestmark = pytest.mark.gpu

N = (128, 256, 16)
L = (4.0, 8.0, 0.5)
STEPS = 3
SETTINGS = {
    "default": {},
    "plans_0": {"y_plan": 0, "zf_plan": 0},
    "plans_2": {"y_plan": 2, "zf_plan": 2},
    "narrow_tiles": {"y_cols": 8, "z_cols": 8},
    "narrowest_tiles": {"y_cols": 4, "z_cols": 4},
    "shared_memory_x_kernel": {"x_kernel": 1},
    "paired_y": {"y_pair": 1},
    "all_changed": {"y_plan": 2, "zf_plan": 0, "y_cols": 8, "z_cols": 16, "x_kernel": 1, "y_pair": 1},
}


@pytest.fixture(scope="module")
def fl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from conftest import build_flusi
    return build_flusi()


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _case():
    cfg = {"n": N, "L": L, "nu": 0.01, "eta": 1e-2, "dt_fixed": 2e-3, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0)}
    ins = workloads.sphere((2.0, 4.0, 0.25), 0.15, profile="cos")
    u0 = workloads.random_smooth_field(N, 7, mean=(0.3, 0.0, 0.0))
    return cfg, ins, u0


@pytest.fixture(scope="module")
def reference():
    cfg, ins, u0 = _case()
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    rows = ref.step(STEPS)
    return ref.get_state(), rows


@pytest.mark.parametrize("name", sorted(SETTINGS))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_setting_matches_the_oracle(fl, reference, name, prec):
    cfg, ins, u0 = _case()
    sim = fl.Solver(cfg, ins, precision=prec)
    if SETTINGS[name]:
        sim.set_tuning(**SETTINGS[name])
    t = sim.tuning()
    for k, v in SETTINGS[name].items():
        assert t[k] == v
    sim.set_state(u0)
    sim.step(STEPS)
    rows, lost = sim.forces()
    u = sim.get_state()[0]
    sim.close()
    u_ref, rows_ref = reference
    assert lost == 0 and rows.shape == rows_ref.shape
    tol_u, tol_f = (1e-11, 1e-10) if prec == "fp64" else (3e-5, 1e-4)
    check_state(u, u_ref, tol_u)
    assert rel_l2(rows[:, 2:20], rows_ref[:, 2:20]) <= tol_f


PAIR_GRIDS = [((16, 1024, 12), (1.0, 8.0, 0.75)),    # half 512 = 8 8 8
              ((24, 768, 8), (1.5, 6.0, 0.5)),       # half 384 = 3 16 8
              ((8, 96, 18), (0.5, 0.75, 1.125)),     # half 48 = 3 16
              ((16, 16, 16), (1.0, 1.0, 1.0))]       # half 8 = 8: one stage


@pytest.mark.parametrize("n,L", PAIR_GRIDS)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_paired_y_kernel_matches_the_oracle(fl, n, L, prec):
    """The two-CTA y kernel (y_pair 1; rows split by parity, joined by a
    radix-2 step through distributed shared memory) against the oracle, on
    grids with half lengths of one to three stages and a factor 3."""
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "dt_fixed": 1e-3, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0)}
    ins = workloads.sphere(tuple(0.5 * x for x in L), 0.3 * min(L), profile="cos")
    u0 = workloads.random_smooth_field(n, 5, mean=(0.3, 0.0, 0.0))
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    rows_ref = ref.step(2)
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_tuning(y_pair=1)
    assert sim.tuning()["y_paired"] == 1
    sim.set_state(u0)
    sim.step(2)
    rows, _ = sim.forces()
    u = sim.get_state()[0]
    sim.close()
    tol_u, tol_f = (1e-11, 1e-10) if prec == "fp64" else (3e-5, 1e-4)
    check_state(u, ref.get_state(), tol_u)
    assert rel_l2(rows[:, 2:20], rows_ref[:, 2:20]) <= tol_f


def test_retuning_a_running_handle_keeps_its_state(fl):
    """flusi_set_tuning between steps: the state (the kept modes) carries
    over, and the run continues as a handle that had the new setting from the
    start would after loading the same state (bit for bit).  Physical-space
    read-outs go through the new plans, so only the spectrum is compared
    across the change."""
    cfg, ins, u0 = _case()
    a = fl.Solver(cfg, ins, precision="fp64")
    a.set_state(u0)
    a.step(2)
    ck = a.save()
    before = a.get_spectrum()
    a.set_tuning(y_plan=2, zf_plan=0, y_cols=8, x_kernel=1)
    assert np.array_equal(a.get_spectrum(), before)
    a.step(2)
    ua, ta, sa = a.get_state()
    a.close()
    b = fl.Solver(cfg, ins, precision="fp64")
    b.set_tuning(y_plan=2, zf_plan=0, y_cols=8, x_kernel=1)
    b.set_state(u0)
    b.load(ck)
    b.step(2)
    ub, tb, sb = b.get_state()
    b.close()
    assert np.array_equal(ua, ub) and ta == tb and sa == sb == 4


def test_autotune_restores_the_state_and_uses_its_cache(fl, tmp_path):
    cfg, ins, u0 = _case()
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    sim.step(2)
    u_before, t_before, s_before = sim.get_state(np.float32)
    spec_before = sim.get_spectrum()
    cache = str(tmp_path / "tuning.txt")
    chosen = sim.autotune(steps=2, cache_path=cache)
    assert sim.tuning() == chosen
    _, t_after, s_after = sim.get_state(np.float32)
    assert np.array_equal(sim.get_spectrum(), spec_before)
    assert t_after == t_before and s_after == s_before == 2
    assert sim.forces()[0].shape[0] == 0          # rows of the timed steps are dropped
    lines = open(cache).read().splitlines()
    assert len(lines) == 1
    key, *vals = lines[0].split()
    assert "128x256x16|fp32|ab2" in key
    assert [int(v) for v in vals] == [chosen[k] for k in fl.TUNING_SETTINGS]
    # the run goes on exactly as a handle given the chosen settings would
    sim.step(2)
    u_tuned = sim.get_state()[0]
    ck_state = (u_before, t_before)
    sim.close()
    other = fl.Solver(cfg, ins, precision="fp32")
    other.set_state(u0)
    other.step(2)
    assert np.array_equal(other.get_state(np.float32)[0], ck_state[0])
    # a cached key is applied without timing: nothing is appended
    again = other.autotune(steps=2, cache_path=cache)
    assert again == chosen and len(open(cache).read().splitlines()) == 1
    assert other.get_state()[1] == t_before
    other.step(2)
    assert np.array_equal(other.get_state()[0], u_tuned)
    other.close()


def test_autotune_rejects_bad_arguments(fl):
    cfg, ins, u0 = _case()
    sim = fl.Solver(cfg, ins, precision="fp32")
    with pytest.raises(fl.FlusiError) as e:
        sim.autotune(steps=2)                     # no state yet
    assert e.value.code == fl.FLUSI_ESTATE
    sim.set_state(u0)
    for steps in (0, 1001):
        with pytest.raises(fl.FlusiError) as e:
            sim.autotune(steps=steps)
        assert e.value.code == fl.FLUSI_EINVAL
    sim.close()


@pytest.mark.parametrize("kind", ["rk4_wake", "free_flight"])
def test_autotune_restores_every_kind_of_state(fl, kind):
    """RK4 with the wake terms (stage-suffixed kernel names, the separate
    sponge pass of the shared-memory x kernel) and free flight (the body state
    lives on the device): after flusi_autotune the spectrum, time, step count
    and body state are those before it, and the run continues exactly as a
    handle given the same settings from a checkpoint would."""
    import test_gpu_flight as tf
    n, L = (128, 64, 32), (4.0, 2.0, 1.0)
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0)}
    if kind == "rk4_wake":
        cfg.update(time_scheme="rk4", sponge_c=0.1, sponge_width=(L[0] / 8, 0.0, 0.0),
                   layer_width=(L[0] / 16, 0.0, 0.0))
        ins = workloads.sphere((2.0, 1.0, 0.5), 0.3, profile="cos")
    else:
        ins = tf.flying_insect(n, L)
        ins["x_cntr"] = (2.0, 1.0, 0.5)
    u0 = workloads.random_smooth_field(n, 5, mean=(0.3, 0.0, 0.0))
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    sim.step(3)
    ck = sim.save()
    spec, (t0, s0) = sim.get_spectrum(), sim.get_state()[1:]
    body = sim.body() if kind == "free_flight" else None
    chosen = sim.autotune(steps=1)
    assert np.array_equal(sim.get_spectrum(), spec) and sim.get_state()[1:] == (t0, s0)
    if body is not None:
        after = sim.body()
        for k in body:
            assert np.array_equal(after[k], body[k]), k
    sim.step(2)
    u_a = sim.get_state()[0]
    sim.close()
    other = fl.Solver(cfg, ins, precision="fp32")
    other.set_tuning(**{k: chosen[k] for k in fl.TUNING_SETTINGS})
    other.load(ck)
    other.step(2)
    assert np.array_equal(other.get_state()[0], u_a)
    other.close()
