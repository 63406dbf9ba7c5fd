"""The asynchronous paths of the C-ABI on the GPU: insect descriptors
uploaded from the handle's page-locked slots while earlier steps run, and
force rows drained without waiting (flusi_forces_async).  Both must give the
rows and states of the synchronous calls bit for bit."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fl():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from conftest import build_flusi
    return build_flusi()


def _pinned_rows(fl, n):
    import torch
    return torch.zeros((n, fl.FORCE_COLS), dtype=torch.float64).pin_memory().numpy()


def _case(ring=4096):
    cfg = dict(workloads.config_model_insect(32)[0], n=(48, 32, 32), force_ring=ring)
    ins = workloads.model_insect((4.0, 4.0, 4.0), (48, 32, 32))
    u0 = workloads.initial_field(cfg)
    return cfg, ins, u0


def _moved(fl, ins, k):
    """The insect with its body centre moved by k small steps (same mask shape)."""
    d = dict(ins, x_cntr=(2.0 + 0.01 * k, 2.0 - 0.005 * k, 2.0 + 0.003 * k))
    return fl.make_insect(d)


@pytest.mark.parametrize("graph", [1, 0])
def test_async_rows_and_descriptors_equal_the_synchronous_ones(fl, graph):
    """12 steps, a new descriptor before each (more than the 8 staging slots
    are reused): one run waits after every step and drains synchronously, the
    other queues all steps, uploads and row copies and waits once."""
    cfg, ins, u0 = _case()
    cfg = dict(cfg, use_graph=graph)
    steps = 12
    a = fl.Solver(cfg, ins, precision="fp32")
    a.set_state(u0)
    rows_a = []
    for k in range(steps):
        fl.flusi_set_kinematics(a.h, _moved(fl, ins, k))
        a.step(1)
        r, _ = a.forces()
        rows_a.append(r)
    rows_a = np.vstack(rows_a)
    ua = a.get_state()[0]
    a.close()
    b = fl.Solver(cfg, ins, precision="fp32")
    b.set_state(u0)
    buf = _pinned_rows(fl, steps)
    got = 0
    for k in range(steps):
        fl.flusi_set_kinematics(b.h, _moved(fl, ins, k))
        b.step(1)
        cnt, lost = fl.flusi_forces_async(b.h, buf, got)
        assert cnt == 1 and lost == 0
        got += cnt
    ub = b.get_state()[0]            # synchronizes: the row copies have run
    assert b.forces()[0].shape[0] == 0
    b.close()
    assert np.array_equal(buf, rows_a)
    assert np.array_equal(ub, ua)
    assert len(set(rows_a[:, 2])) == steps          # the moving body changes every row


def test_async_drain_counts_lost_rows(fl):
    """force_ring 4, 10 steps queued, one asynchronous drain: the last 4 rows,
    6 lost; a drain right after finds nothing; mixed with the synchronous
    drain no row comes twice."""
    cfg, ins, u0 = _case(ring=4)
    ref = fl.Solver(dict(cfg, force_ring=64), ins, precision="fp32")
    ref.set_state(u0)
    ref.step(13)
    all_rows = ref.forces()[0]
    ref.close()
    sim = fl.Solver(cfg, ins, precision="fp32")
    sim.set_state(u0)
    sim.step(10)
    buf = _pinned_rows(fl, 8)
    cnt, lost = fl.flusi_forces_async(sim.h, buf)
    assert (cnt, lost) == (4, 6)
    assert fl.flusi_forces_async(sim.h, buf, 4) == (0, 0)
    sim.sync()
    assert np.array_equal(buf[:4], all_rows[6:10])
    sim.step(2)
    r, lost = sim.forces()
    assert lost == 0 and np.array_equal(r, all_rows[10:12])
    sim.step(1)
    cnt, lost = fl.flusi_forces_async(sim.h, buf, 4)
    assert (cnt, lost) == (1, 0)
    sim.sync()
    assert np.array_equal(buf[4], all_rows[12])
    sim.close()


def test_async_drain_arguments(fl):
    cfg, ins, u0 = _case()
    sim = fl.Solver(cfg, ins, precision="fp32")
    buf = _pinned_rows(fl, 4)
    with pytest.raises(fl.FlusiError) as e:
        fl.flusi_forces_async(sim.h, buf)                   # no state yet
    assert e.value.code == fl.FLUSI_ESTATE
    sim.set_state(u0)
    with pytest.raises(ValueError):
        fl.flusi_forces_async(sim.h, np.zeros((4, 3)))
    sim.step(2)
    assert fl.flusi_forces_async(sim.h, buf, 4) == (0, 0)    # no room: nothing taken
    assert fl.flusi_forces_async(sim.h, buf, 3) == (1, 0)
    sim.sync()
    sim.close()
