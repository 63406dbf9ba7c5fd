"""The allocation-free sums entry point, flusi_penalization_sums_noalloc.

It serves callers that cannot allocate device memory (their memory belongs to
another allocator's pool, or a cudaMalloc/cudaFree with its device
synchronization is not acceptable where they run): it takes a velocity field
they already hold and returns the force, moment, energy and CFL sums, with its
scratch in a fixed device array of the library.  Here its output is checked
against the force rows the time step itself produces, on two calls in a row
(the second reuses the array the first one left behind).  This file is named
to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

import workloads


@pytest.fixture(scope="module")
def fl():
    from conftest import build_flusi
    return build_flusi()


def _close(a, b, tol):
    a, b = np.asarray(a, float), np.asarray(b, float)
    scale = max(np.abs(b).max(), 1e-300)
    return np.abs(a - b).max() <= tol * scale


@pytest.mark.gpu
def test_noalloc_sums_match_step_force_rows(fl):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    cfg, ins = workloads.config_model_insect(32)
    insect = workloads.model_insect(cfg["L"], cfg["n"])
    u0 = workloads.initial_field(cfg) + 0.05 * workloads.random_smooth_field(cfg["n"], 1)
    nx, ny, nz = cfg["n"]
    sim = fl.Solver(cfg, insect, precision="fp64")
    sim.set_state(u0)
    u_t0 = torch.empty((3, nz, ny, nx), dtype=torch.float64, device="cuda")
    sim.get_state_device(u_t0)
    sim.step(1)
    u_t1 = torch.empty_like(u_t0)
    t1, _ = sim.get_state_device(u_t1)
    sim.step(1)
    rows, _ = sim.forces()
    sim.close()
    assert rows.shape[0] == 2 and rows[1, 0] == t1

    desc = fl.make_insect(insect)
    torch.cuda.synchronize()
    s0 = fl.flusi_penalization_sums_noalloc(cfg["n"], cfg["L"], cfg["eta"], desc, 0.0,
                                            u_t0.data_ptr())
    s1 = fl.flusi_penalization_sums_noalloc(cfg["n"], cfg["L"], cfg["eta"], desc, t1,
                                            u_t1.data_ptr())
    dt0 = rows[0, 1]
    for c in range(3):
        F0, M0 = s0[12 * c: 12 * c + 3], s0[12 * c + 3: 12 * c + 6]
        I0, J0 = s0[12 * c + 6: 12 * c + 9], s0[12 * c + 9: 12 * c + 12]
        F1, M1 = s1[12 * c: 12 * c + 3], s1[12 * c + 3: 12 * c + 6]
        I1, J1 = s1[12 * c + 6: 12 * c + 9], s1[12 * c + 9: 12 * c + 12]
        # first row: no unsteady correction; second: backward difference over dt0
        assert _close(F0, rows[0, 2 + 6 * c: 5 + 6 * c], 1e-10)
        assert _close(M0, rows[0, 5 + 6 * c: 8 + 6 * c], 1e-10)
        assert _close(F1 + (I1 - I0) / dt0, rows[1, 2 + 6 * c: 5 + 6 * c], 1e-9)
        assert _close(M1 + (J1 - J0) / dt0, rows[1, 5 + 6 * c: 8 + 6 * c], 1e-9)
    for s, r in ((s0, rows[0]), (s1, rows[1])):
        assert abs(s[36] - r[20]) <= 1e-12 * r[20]
        assert abs(s[37] - r[21]) <= 1e-14 * r[21]
    assert np.abs(s0[:12]).max() > 0 and np.abs(s0[12:24]).max() > 0   # body and a wing hit


def _oracle_sums(cfg, insect, u, t):
    """The oracle's force, moment, solid-integral, energy and max|u| sums of
    the physical field u (Sec. 2.2, Eqs. force_with_unst_corrections,
    moment_of_love): its right-hand side evaluated on the spectrum of u."""
    import oracle
    sp = oracle.Spectral(cfg)
    return sp.rhs(sp.forward(u), t, insect)[1], sp.inverse(sp.forward(u))


@pytest.mark.gpu
def test_noalloc_sums_match_the_oracle_at_the_cta_cap(fl):
    """128 x 64 x 48 points (more than 1 024 CTAs of 256 points, so the grid
    is capped and every CTA strides over several blocks), a flapping insect at
    two times: each colour's F, M, sum chi u_s, sum r x chi u_s, the energy
    and max |u| against the CPU oracle, on two calls in a row."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    n, L = (128, 64, 48), (4.0, 2.0, 1.5)
    assert n[0] * n[1] * n[2] > 1024 * 256
    cfg = {"n": n, "L": L, "nu": 0.01, "eta": 2.5e-3}
    insect = dict(workloads.model_insect(L, n), x_cntr=(2.0, 1.0, 0.75))
    desc = fl.make_insect(insect)
    for seed, t in ((3, 0.13), (4, 0.41)):
        u = workloads.random_smooth_field(n, seed, amplitude=0.7, mean=(0.25, 0.0, 0.0))
        ref, u_band = _oracle_sums(cfg, insect, u, t)
        u_dev = torch.from_numpy(np.ascontiguousarray(u_band)).cuda()
        torch.cuda.synchronize()
        got = fl.flusi_penalization_sums_noalloc(n, L, cfg["eta"], desc, t, u_dev.data_ptr())
        for c in range(3):
            blk, rb = got[12 * c: 12 * c + 12], ref[12 * c: 12 * c + 12]
            assert np.abs(rb).max() > 0, c   # every part meets the grid
            for q in range(4):
                assert _close(blk[3 * q: 3 * q + 3], rb[3 * q: 3 * q + 3], 1e-10), (c, q)
        assert abs(got[36] - ref[36]) <= 1e-12 * ref[36]
        assert abs(got[37] - ref[37]) <= 1e-13 * ref[37]


@pytest.mark.gpu
def test_noalloc_without_an_insect(fl):
    """No insect: all 36 force and moment sums exactly zero; the energy and
    max |u| against a direct host computation."""
    import torch
    if not torch.cuda.is_available():
        pytest.fail("GPU test needs a CUDA device")
    n, L = (96, 48, 64), (3.0, 1.5, 2.0)
    u = workloads.random_field(n, 11, amplitude=0.5)
    u_dev = torch.from_numpy(np.ascontiguousarray(u)).cuda()
    torch.cuda.synchronize()
    got = fl.flusi_penalization_sums_noalloc(n, L, 1e-2, None, 0.0, u_dev.data_ptr())
    assert np.all(np.asarray(got[:36]) == 0.0)
    dV = L[0] * L[1] * L[2] / (n[0] * n[1] * n[2])
    e = 0.5 * float((u * u).sum()) * dV
    umax = float(np.sqrt((u * u).sum(axis=0)).max())
    assert abs(got[36] - e) <= 1e-12 * e
    assert abs(got[37] - umax) <= 1e-14 * umax


def test_noalloc_rejects_oversized_grids(fl):
    dummy = 0x100000
    with pytest.raises(fl.FlusiError) as e:
        fl.flusi_penalization_sums_noalloc((1025, 1024, 1024), (1.0, 1.0, 1.0), 1e-3, None, 0.0,
                                           dummy)
    assert e.value.code == fl.FLUSI_EINVAL
    assert "FLUSI_NOALLOC_MAX_POINTS" in fl.flusi_last_error(None)
    with pytest.raises(fl.FlusiError):
        fl.flusi_penalization_sums_noalloc((8, 8, 8), (1.0, 1.0, 1.0), 0.0, None, 0.0, dummy)
