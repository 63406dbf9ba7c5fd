"""Checkpoint and exact restart (flusi_checkpoint_bytes / flusi_save /
flusi_load): host-side argument checks, and on the GPU a run restarted from
a checkpoint continues bit for bit."""
import ctypes as C

import numpy as np
import pytest

import workloads


@pytest.fixture(scope="module")
def fl():
    from conftest import build_flusi
    return build_flusi()


def test_checkpoint_size_and_host_checks(fl):
    h = fl.flusi_create((16, 12, 8), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
    nbytes = fl.flusi_checkpoint_bytes(h)
    # header + step state + body state + u_hat and the history over the kept modes
    Mx, My, Mz = 16 // 3 + 1, 2 * (12 // 3) + 1, 2 * (8 // 3) + 1
    Mxp = (Mx + 3) // 4 * 4
    spec = 3 * Mz * My * Mxp * 8
    assert nbytes > 2 * spec and nbytes - 2 * spec < 1024
    buf = np.zeros(nbytes, np.uint8)
    ptr = C.c_void_p(buf.ctypes.data)
    # no state yet
    assert fl.lib.flusi_save(h, ptr, nbytes) == fl.FLUSI_ESTATE
    assert fl.lib.flusi_save(h, ptr, nbytes - 1) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_load(h, ptr, nbytes) == fl.FLUSI_EINVAL        # no magic
    assert "checkpoint" in fl.flusi_last_error(h)
    assert fl.lib.flusi_load(h, None, nbytes) == fl.FLUSI_EINVAL
    fl.flusi_destroy(h)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_restart_continues_bit_for_bit(fl, prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    cfg, ins = workloads.config_model_insect(32)
    cfg = dict(cfg, n=(32, 24, 16), L=(4.0, 3.0, 2.0))
    ins = workloads.model_insect(cfg["L"], cfg["n"])
    dt = np.float64 if prec == "fp64" else np.float32
    u0 = workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"]).astype(dt)
    a = fl.Solver(cfg, ins, precision=prec)
    a.set_state(u0)
    a.step(7)
    rows_a, _ = a.forces()
    ua, ta, na = a.get_state(dt)
    a.close()

    b = fl.Solver(cfg, ins, precision=prec)
    b.set_state(u0)
    b.step(4)
    first, _ = b.forces()
    ck = b.save()
    b.close()
    c = fl.Solver(cfg, ins, precision=prec)
    c.load(ck)
    c.step(3)
    rest, lost = c.forces()
    uc, tc, nc = c.get_state(dt)
    assert (nc, lost) == (7, 0) and tc == ta
    assert np.array_equal(uc, ua)
    assert np.array_equal(np.vstack([first, rest]), rows_a)
    # a checkpoint of another grid is refused before anything is touched
    other = fl.Solver(dict(cfg, n=(32, 24, 24)), ins, precision=prec)
    with pytest.raises(fl.FlusiError) as e:
        other.load(ck)
    assert e.value.code == fl.FLUSI_EINVAL
    other.close()
    c.close()
