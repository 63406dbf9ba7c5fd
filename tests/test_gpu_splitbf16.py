"""The split-BF16 forms (FLUSI_FP32_SPLITBF16, FLUSI_FP32_SPLITBF16X3):
FP32 state whose physical x pass takes its DFT stages on the tensor cores
(tcgen05) as BF16 products of operands split into two or three pieces.
Full steps through the C-ABI against the FP64 oracle (Sec. 2.4; Algorithm 1).

Error budget.  A product of two pieces-split operands keeps about 16 (two
pieces, the lo*lo term dropped) or 24 (three pieces) significant bits, so a
transformed line carries a relative error of about 2^-16 ~ 1.5e-5 (bf16x2)
or the FP32 rounding level (bf16x3).  That error enters the state only
through the nonlinear term, scaled by dt |N| / |u| (a step moves the state by
a small fraction of itself), so one step stays within the stated 1e-5 per
step; five steps within 5e-5 (bf16x2) and the FP32 bar 2e-5 (bf16x3).  Force
rows are sums over the solid of chi (u - u_s) / C_eta, where u ~ u_s: the
line error of u appears there relative to |u - u_s| and is bounded by 1e-3
(bf16x2) and 2e-4 (bf16x3) of each column's scale.
"""
import math

import numpy as np
import pytest

import oracle
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


def max_rel(a, b):
    """largest pointwise deviation relative to the largest value"""
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / np.abs(np.asarray(b)).max())


def rows_err(a, b):
    a, b = np.asarray(a), np.asarray(b)
    err = 0.0
    for j in range(b.shape[1]):
        scale = np.abs(b[:, j]).max()
        if scale > 1e-12:
            err = max(err, np.abs(a[:, j] - b[:, j]).max() / scale)
    return err


# nx = 512 (16 x 16 stages, 8 grid rows per tile) and 256 (8 x 16 / 16 x 8,
# 16 rows per tile); the second grid of each leaves a ragged last tile
GRIDS = {"x512": ((512, 16, 12), (8.0, 1.0, 0.75)), "x512_ragged": ((512, 18, 9), (8.0, 1.125, 0.5625)),
         "x256": ((256, 24, 16), (8.0, 0.75, 0.5)), "x256_ragged": ((256, 18, 9), (8.0, 0.5625, 0.28125))}
TOL = {"bf16x2": {"u1": 1e-5, "u5": 5e-5, "max5": 2e-4, "rows": 1e-3},
       "bf16x3": {"u1": 2e-6, "u5": 2e-5, "max5": 5e-5, "rows": 2e-4}}


def _run(fl, cfg, ins, u0, prec, steps):
    sim = fl.Solver(cfg, ins, precision=prec)
    sim.set_state(u0)
    names = list(sim.profile(1))   # kernel names of one (uncaptured) step
    sim.set_state(u0)
    out = []
    for s in steps:
        sim.step(s)
        out.append(sim.get_state()[0])
    rows, _ = sim.forces()
    sim.close()
    return out, rows, names


@pytest.mark.parametrize("name", sorted(GRIDS))
@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_split_forms_match_the_oracle(fl, name, prec):
    """A sphere in a mean flow with adaptive dt: the state after 1 and 5 steps
    (relative L2 and the largest pointwise deviation) and the force rows
    against the oracle; the tensor-core kernel is the one that ran."""
    n, L = GRIDS[name]
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0)}
    ins = workloads.sphere((L[0] / 2, L[1] / 2, L[2] / 2), 0.35 * min(L[1], L[2]), profile="cos")
    u0 = workloads.random_smooth_field(n, 7, mean=(0.3, 0.0, 0.0))
    (u1, u5), rows, names = _run(fl, cfg, ins, u0, prec, (1, 4))
    assert "xpass_tc" in names and "xpass_phys" not in names
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(1)
    r1 = ref.get_state()
    ref_rows = np.vstack([ref_rows, ref.step(4)])
    r5 = ref.get_state()
    t = TOL[prec]
    e1, e5, m5, er = rel_l2(u1, r1), rel_l2(u5, r5), max_rel(u5, r5), rows_err(rows, ref_rows)
    print(f"{prec} {name}: u rel L2 {e1:.2e} (1 step) {e5:.2e} (5 steps), max {m5:.2e}, rows {er:.2e}")
    assert e1 <= t["u1"] and e5 <= t["u5"] and m5 <= t["max5"] and er <= t["rows"]


@pytest.mark.parametrize("prec", ["bf16x2", "bf16x3"])
def test_split_forms_flapping_wing(fl, prec):
    """A flapping plate wing crossing many tiles at nx = 256 with the
    Dirichlet layer on (the layer's term is formed in the same per-point
    pass): 6 adaptive steps against the oracle."""
    n, L = (256, 36, 24), (4.0, 3.0, 2.0)
    cfg = {"n": n, "L": L, "nu": 0.0125664, "eta": 2.5e-3, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.2, 0.0, 0.0), "layer_width": (0.25, 0.0, 0.0)}
    ins = dict(workloads.single_wing(L, n), x_cntr=(2.0, 1.5, 1.0))
    u0 = workloads.random_smooth_field(n, 5, mean=(0.2, 0.0, 0.0))
    (u6,), rows, names = _run(fl, cfg, ins, u0, prec, (6,))
    assert "xpass_tc" in names
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(6)
    t = TOL[prec]
    e, er = rel_l2(u6, ref.get_state()), rows_err(rows, ref_rows)
    print(f"{prec} flapping wing 256x36x24: u rel L2 {e:.2e} after 6 steps, rows {er:.2e}")
    assert e <= t["u5"] and er <= t["rows"]


def test_split_form_needs_a_supported_length(fl):
    for nx in (128, 1024, 96):
        with pytest.raises(fl.FlusiError) as e:
            fl.flusi_create((nx, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32_SPLITBF16)
        assert e.value.code == fl.FLUSI_EINVAL


WIDE_SPLIT = ((512, 16, 12), (8.0, 1.0, 0.75))


@pytest.mark.parametrize("scheme", ["ab2_wake", "rk4_wake"])
def test_split_form_with_the_wake_terms_and_rk4(fl, scheme):
    """bf16x2 with the vorticity sponge and the Dirichlet layer (the sponge's
    extra x round trip on the FP32 kernel, the layer's term in the tensor-core
    pass), with AB2 and with RK4 (four tensor-core x passes per step): five
    adaptive steps against the oracle."""
    n, L = WIDE_SPLIT
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0), "sponge_c": 0.1, "sponge_width": (L[0] / 6, 0.0, 0.0),
           "layer_width": (L[0] / 16, 0.0, 0.0)}
    if scheme == "rk4_wake":
        cfg["time_scheme"] = "rk4"
    ins = workloads.sphere((L[0] / 2, L[1] / 2, L[2] / 2), 0.3 * min(L[1], L[2]), profile="cos")
    u0 = workloads.random_smooth_field(n, 9, mean=(0.3, 0.0, 0.0))
    (u5,), rows, names = _run(fl, cfg, ins, u0, "bf16x2", (5,))
    assert "xpass_tc" in names and "sponge_x" in names
    if scheme == "rk4_wake":
        assert "xpass_tc.4" in names
    ref = oracle.Simulation(cfg, ins)
    ref.set_state(u0)
    ref_rows = ref.step(5)
    t = TOL["bf16x2"]
    e, er = rel_l2(u5, ref.get_state()), rows_err(rows, ref_rows)
    print(f"bf16x2 {scheme} 512x16x12: u rel L2 {e:.2e} after 5 steps, rows {er:.2e}")
    assert e <= t["u5"] and max_rel(u5, ref.get_state()) <= t["max5"] and er <= t["rows"]


def test_split_form_restarts_bit_for_bit(fl):
    """A checkpoint of a bf16x2 run (state, history, step state in FP32, the
    same layout as FLUSI_FP32) continues bit for bit, and cannot be loaded into
    a handle of another precision."""
    import ctypes as C
    n, L = WIDE_SPLIT
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 1e-2, "cfl": 0.1, "mean_mode": "fixed",
           "u_inf": (0.3, 0.0, 0.0)}
    ins = workloads.sphere((L[0] / 2, L[1] / 2, L[2] / 2), 0.35 * min(L[1], L[2]), profile="cos")
    u0 = workloads.random_smooth_field(n, 7, mean=(0.3, 0.0, 0.0))
    a = fl.Solver(cfg, ins, precision="bf16x2")
    a.set_state(u0)
    a.step(7)
    ua, rows_a = a.get_state(np.float32)[0], a.forces()[0]
    a.close()
    b = fl.Solver(cfg, ins, precision="bf16x2")
    b.set_state(u0)
    b.step(4)
    nbytes = C.c_size_t()
    assert fl.lib.flusi_checkpoint_bytes(b.h, C.byref(nbytes)) == fl.FLUSI_OK
    buf = (C.c_char * nbytes.value)()
    assert fl.lib.flusi_save(b.h, buf, nbytes) == fl.FLUSI_OK
    rows_b = b.forces()[0]
    b.close()
    c = fl.Solver(cfg, ins, precision="bf16x2")
    assert fl.lib.flusi_load(c.h, buf, nbytes) == fl.FLUSI_OK
    c.step(3)
    uc, rows_c = c.get_state(np.float32)[0], c.forces()[0]
    c.close()
    assert np.array_equal(uc, ua)
    assert np.array_equal(np.vstack([rows_b, rows_c]), rows_a)
    d = fl.Solver(cfg, ins, precision="fp32")
    assert fl.lib.flusi_load(d.h, buf, nbytes) == fl.FLUSI_EINVAL
    d.close()
