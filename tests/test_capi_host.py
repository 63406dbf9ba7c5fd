"""Host-side checks of the C-ABI (no GPU): the library loads, exports every
entry point declared in include/flusi.h, and rejects bad arguments before any
device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fl():
    from conftest import build_flusi
    return build_flusi()


def _declared():
    src = open(os.path.join(ROOT, "include", "flusi.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(flusi_[a-z_]+)\s*\(", src)))


def test_header_symbols_exported(fl):
    names = _declared()
    assert "flusi_create" in names and "flusi_step" in names and len(names) >= 15
    lib = C.CDLL(fl.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), f"{n} declared in flusi.h but not exported"


def test_create_validates_sizes(fl):
    L = (1.0, 1.0, 1.0)
    for n in [(7, 8, 8), (8, 10, 8), (9, 8, 8), (2048, 8, 8), (4, 8, 8), (8, 8, 5)]:
        with pytest.raises(fl.FlusiError) as e:
            fl.flusi_create(n, L, 0.1, 1e-2, fl.FLUSI_FP64)
        assert e.value.code == fl.FLUSI_EINVAL
    with pytest.raises(fl.FlusiError):
        fl.flusi_create((8, 8, 8), (1.0, -1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP64)
    with pytest.raises(fl.FlusiError):
        fl.flusi_create((8, 8, 8), L, 0.1, 0.0, fl.FLUSI_FP64)
    with pytest.raises(fl.FlusiError):
        fl.flusi_create((8, 8, 8), L, 0.1, 1e-2, 7)
    h = fl.flusi_create((96, 12, 1024), L, 0.1, 1e-2, fl.FLUSI_FP32)
    fl.flusi_destroy(h)


def test_workspace_size_scales_with_grid_and_precision(fl):
    L = (1.0, 1.0, 1.0)
    sizes = {}
    for prec in (fl.FLUSI_FP32, fl.FLUSI_FP64):
        for n in (32, 64):
            h = fl.flusi_create((n, n, n), L, 0.1, 1e-2, prec)
            sizes[(prec, n)] = fl.flusi_workspace_bytes(h)
            fl.flusi_destroy(h)
    assert sizes[(fl.FLUSI_FP64, 64)] > 1.6 * sizes[(fl.FLUSI_FP32, 64)]
    assert sizes[(fl.FLUSI_FP32, 64)] > 4 * sizes[(fl.FLUSI_FP32, 32)]
    # 512^3 FP32: state, history and the six-field work buffer of pruned rows
    h = fl.flusi_create((512, 512, 512), (4.0, 4.0, 4.0), 0.1, 1e-3, fl.FLUSI_FP32)
    b = fl.flusi_workspace_bytes(h)
    fl.flusi_destroy(h)
    spec = 3 * 341 * 341 * 172 * 8
    work = 6 * 512 * 512 * 172 * 8
    assert spec * 2 + work <= b <= spec * 2 + work + 64 * 2 ** 20


def test_options_validation(fl):
    h = fl.flusi_create((16, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP64)
    o = fl.flusi_default_options()
    assert o.cfl == 0.1 and o.force_ring == 4096 and o.use_graph == 1
    fl.flusi_set_options(h, o)
    for field, bad in (("cfl", 0.0), ("dt_fixed", -1.0), ("force_ring", 0), ("mean_mode", 2)):
        b = fl.flusi_default_options()
        setattr(b, field, bad)
        with pytest.raises(fl.FlusiError) as e:
            fl.flusi_set_options(h, b)
        assert e.value.code == fl.FLUSI_EINVAL
    fl.flusi_destroy(h)


def test_calls_before_bind_fail_cleanly(fl):
    h = fl.flusi_create((16, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP64)
    u = np.zeros((3, 16, 16, 16))
    for call in (lambda: fl.flusi_set_state(h, u, fl.FLUSI_HOST_FP64),
                 lambda: fl.flusi_step(h, 1), lambda: fl.flusi_forces(h, 4),
                 lambda: fl.flusi_sync(h)):
        with pytest.raises(fl.FlusiError) as e:
            call()
        assert e.value.code == fl.FLUSI_ESTATE
    assert "bind" in fl.flusi_last_error(h)
    # bind with a NULL, misaligned or short workspace is rejected on the host
    assert fl.lib.flusi_bind(h, None, 10, None) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_bind(h, C.c_void_p(0x1001), 1 << 40, None) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_bind(h, C.c_void_p(0x100000), 16, None) == fl.FLUSI_ENOMEM
    assert fl.flusi_destroy(h) == fl.FLUSI_OK
    assert fl.lib.flusi_destroy(None) == fl.FLUSI_OK


def test_insect_descriptor_validation(fl):
    import workloads
    h = fl.flusi_create((16, 16, 16), (4.0, 4.0, 4.0), 0.1, 1e-2, fl.FLUSI_FP64)
    good = fl.make_insect(workloads.model_insect((4.0, 4.0, 4.0), (16, 16, 16)))
    fl.flusi_set_kinematics(h, good)
    fl.flusi_set_kinematics(h, None)
    for field, bad in (("nwings", 3), ("body_type", 5), ("c_smth", 0.0), ("nfourier", 9),
                       ("body_type", 3)):   # a curved thorax without its arc
        ins = fl.make_insect(workloads.model_insect((4.0, 4.0, 4.0), (16, 16, 16)))
        setattr(ins, field, bad)
        with pytest.raises(fl.FlusiError):
            fl.flusi_set_kinematics(h, ins)
    curved = fl.make_insect(workloads.curved_insect((4.0, 4.0, 4.0), (16, 16, 16)))
    fl.flusi_set_kinematics(h, curved)
    for arc in ((0.1, 0.0, -1.0), (1.0, 0.0, 0.0), (0.1, 0.0, -0.05)):
        bad = fl.make_insect(dict(workloads.curved_insect((4.0, 4.0, 4.0), (16, 16, 16)), body_arc=arc))
        with pytest.raises(fl.FlusiError):
            fl.flusi_set_kinematics(h, bad)
    fl.flusi_destroy(h)


def test_struct_layouts_match_header(fl):
    """The ctypes mirrors have the sizes the C compiler gives the structs."""
    assert C.sizeof(fl.Options) == 3 * 8 + 3 * 8 + 4 * 4 + 7 * 8 + 2 * 4
    assert C.sizeof(fl.Insect) == (4 * 4 + 8 * (1 + 3 + 3 + 6 + 2 + 3 + 3 + 1 + 4 + 1 + 3 * 17)
                                   + 8 * (3 + 1 + 3 + 1) + 2 * 4 + 8 * (3 + 2 * 32)
                                   + 8 * 6 + 2 * 4 + 8 * (2 + 3 + 6 + 4 + 3) + 8 * 3)
    assert fl.FORCE_COLS == 26


def test_free_flight_descriptor_checks(fl):
    """Free flight needs a positive mass and moments of inertia and the AB2
    scheme, whichever of options and kinematics comes first."""
    L, n = (4.0, 4.0, 4.0), (16, 16, 16)
    ff = {"mass": 0.2, "gravity": 9.81, "J_body": (1e-3, 2e-3, 2e-3)}
    h = fl.flusi_create(n, L, 0.1, 1e-2, fl.FLUSI_FP64)
    fl.flusi_set_kinematics(h, fl.make_insect(dict(workloads.model_insect(L, n), free_flight=ff)))
    with pytest.raises(fl.FlusiError):
        fl.flusi_set_options(h, fl.make_options({"time_scheme": "rk4"}))
    for bad in ({"mass": 0.0}, {"J_body": (1e-3, 0.0, 2e-3)}, {"gravity": float("nan")}):
        with pytest.raises(fl.FlusiError):
            fl.flusi_set_kinematics(h, fl.make_insect(dict(workloads.model_insect(L, n),
                                                           free_flight=dict(ff, **bad))))
    ins = fl.make_insect(dict(workloads.model_insect(L, n), free_flight=ff))
    ins.free_flight = 2
    with pytest.raises(fl.FlusiError):
        fl.flusi_set_kinematics(h, ins)
    fl.flusi_destroy(h)
    h = fl.flusi_create(n, L, 0.1, 1e-2, fl.FLUSI_FP64)
    fl.flusi_set_options(h, fl.make_options({"time_scheme": "rk4"}))
    with pytest.raises(fl.FlusiError):
        fl.flusi_set_kinematics(h, fl.make_insect(dict(workloads.model_insect(L, n), free_flight=ff)))
    # tethered kinematics stay allowed with RK4
    fl.flusi_set_kinematics(h, fl.make_insect(workloads.model_insect(L, n)))
    fl.flusi_destroy(h)


def test_kernels_per_step(fl):
    h = fl.flusi_create((16, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP64)
    assert fl.flusi_kernels_per_step(h) == 8
    before = fl.flusi_workspace_bytes(h)
    fl.flusi_set_options(h, fl.make_options({"time_scheme": "rk4"}))
    # four right-hand sides of seven kernels, one scalar kernel; one more state buffer
    assert fl.flusi_kernels_per_step(h) == 4 * 7 + 1
    spec = 3 * 11 * 11 * 8 * 16
    assert fl.flusi_workspace_bytes(h) - before == (spec + 255) // 256 * 256
    bad = fl.make_options({})
    bad.time_scheme = 2
    with pytest.raises(fl.FlusiError):
        fl.flusi_set_options(h, bad)
    fl.flusi_destroy(h)


def _prod(rs):
    p = 1
    for r in rs:
        p *= r
    return p


@pytest.mark.parametrize("n", [16, 48, 96, 128, 192, 256, 384, 512, 768, 1024])
def test_radix_plans(fl, n):
    """The three plan modes of the y and forward z passes: every plan
    factors n; mode 1 differs from mode 0 only for 2^(3q+1) (one 16 for 4 4),
    mode 2 from mode 1 only for 2^(3q+2) with q >= 2 (16 16 for 8 8 4); the
    inverse z pass keeps mode 0."""
    h = fl.flusi_create((16, n, n), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
    plans = {}
    for mode in (0, 1, 2):
        fl.flusi_set_tuning(h, y_plan=mode, zf_plan=mode)
        t = fl.flusi_get_tuning(h)
        assert t["y_radix"] == t["zf_radix"]
        assert _prod(t["y_radix"]) == n and _prod(t["zi_radix"]) == n
        plans[mode] = t["y_radix"]
        zi = t["zi_radix"]
    fl.flusi_destroy(h)
    b = 0
    while n % 3 ** (b + 1) == 0:
        b += 1
    a = (n // 3 ** b).bit_length() - 1          # n = 2^a 3^b
    assert zi == plans[0] and 16 not in plans[0]
    assert all(r in (2, 3, 4, 8) for r in plans[0])
    if a % 3 == 1 and a >= 4:
        assert plans[1].count(16) == 1 and len(plans[1]) == len(plans[0]) - 1
    else:
        assert plans[1] == plans[0]
    if a % 3 == 2 and a >= 8:
        assert plans[2].count(16) == 2 and len(plans[2]) == len(plans[0]) - 1
    else:
        assert plans[2] == plans[1]
    for p in plans.values():                      # the factors 3 come first
        assert p[:b] == [3] * b and 3 not in p[b:]


def test_named_plans(fl):
    h = fl.flusi_create((16, 256, 1024), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP64)
    t = fl.flusi_get_tuning(h)
    assert (t["y_radix"], t["zf_radix"], t["zi_radix"]) == ([8, 8, 4], [16, 8, 8], [8, 8, 4, 4])
    fl.flusi_set_tuning(h, y_plan=2, zf_plan=0)
    t = fl.flusi_get_tuning(h)
    assert (t["y_radix"], t["zf_radix"]) == ([16, 16], [8, 8, 4, 4])
    fl.flusi_destroy(h)


def test_tuning_is_validated(fl):
    """Bad settings are FLUSI_EINVAL and leave the handle's tuning unchanged;
    tile caps bound the tiles the passes take."""
    h = fl.flusi_create((512, 64, 64), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
    before = fl.flusi_get_tuning(h)
    assert before["y_plan"] == 1 and before["zf_plan"] == 1 and before["x_line_kernel"] == 1
    for bad in ({"y_plan": 3}, {"zf_plan": -1}, {"y_cols": 3}, {"y_cols": 2}, {"z_cols": 512},
                {"z_cols": -4}, {"x_kernel": 2}, {"y_pair": 2}, {"y_pair": -1}):
        with pytest.raises(fl.FlusiError) as e:
            fl.flusi_set_tuning(h, **bad)
        assert e.value.code == fl.FLUSI_EINVAL
        assert fl.flusi_get_tuning(h) == before
    with pytest.raises(ValueError):
        fl.flusi_set_tuning(h, y_radix=4)
    for cap in (4, 8, 16):
        fl.flusi_set_tuning(h, y_cols=cap, z_cols=cap)
        t = fl.flusi_get_tuning(h)
        assert t["y_tile_cols"] <= cap and t["z_tile_cols"] <= cap
    fl.flusi_set_tuning(h, x_kernel=1)
    assert fl.flusi_get_tuning(h)["x_line_kernel"] == 0
    fl.flusi_destroy(h)
    h = fl.flusi_create((64, 64, 64), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP64)
    fl.flusi_set_tuning(h, y_cols=2, z_cols=2)   # 32 bytes of FP64 complex values
    t = fl.flusi_get_tuning(h)
    # nx = 64 and 96 take the rectangular register-resident x pass; 48 the generic one
    assert t["y_tile_cols"] == 2 and t["z_tile_cols"] == 2 and t["x_line_kernel"] == 1
    fl.flusi_destroy(h)
    for nx, kind in ((96, 1), (48, 0), (72, 0)):
        h = fl.flusi_create((nx, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
        assert fl.flusi_get_tuning(h)["x_line_kernel"] == kind, nx
        fl.flusi_destroy(h)


def test_autotune_needs_a_bound_handle(fl):
    h = fl.flusi_create((32, 32, 32), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
    with pytest.raises(fl.FlusiError) as e:
        fl.flusi_autotune(h, 2)
    assert e.value.code == fl.FLUSI_ESTATE
    fl.flusi_destroy(h)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_paired_y_kernel_choice(fl, prec):
    """y_pair 1 takes the paired y kernel wherever ny is even (at least 16),
    with the half length's plan and a tile of 128-byte rows or wider; 0 (the
    default) never."""
    P = fl.FLUSI_FP32 if prec == "fp32" else fl.FLUSI_FP64
    row = 128 // (8 if prec == "fp32" else 16)       # complex values in 128 bytes
    for ny in (512, 768, 1024, 96, 16, 27):
        h = fl.flusi_create((16, ny, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, P)
        t = fl.flusi_get_tuning(h)
        assert t["y_pair"] == 0 and t["y_paired"] == 0 and _prod(t["y_radix"]) == ny
        fl.flusi_set_tuning(h, y_pair=1)
        t = fl.flusi_get_tuning(h)
        assert t["y_paired"] == (ny % 2 == 0)
        if ny % 2 == 0:
            assert _prod(t["y_radix"]) == ny // 2 and t["y_tile_cols"] >= min(row, 8192 // 8)
        else:
            assert _prod(t["y_radix"]) == ny
        fl.flusi_destroy(h)


def test_async_drain_needs_a_state(fl):
    """flusi_forces_async checks its handle before any device work."""
    h = fl.flusi_create((16, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
    rows = np.zeros((4, fl.FORCE_COLS))
    with pytest.raises(fl.FlusiError) as e:
        fl.flusi_forces_async(h, rows)
    assert e.value.code == fl.FLUSI_ESTATE
    with pytest.raises(ValueError):
        fl.flusi_forces_async(h, rows, 5)
    fl.flusi_destroy(h)


def test_header_is_plain_c(fl, tmp_path):
    """include/flusi.h compiles as C99 and a C program links against the
    library and calls it (no device work: defaults, creation, sizes, tuning)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text(r"""
#include <stdio.h>
#include "flusi.h"
int main(void)
{
    flusi_options o;
    flusi_default_options(&o);
    double L[3] = {1.0, 1.0, 1.0};
    flusi_t h = 0;
    if (flusi_create(64, 48, 32, L, 0.01, 1e-2, FLUSI_FP32, &h) != FLUSI_OK) return 1;
    size_t bytes = 0;
    if (flusi_workspace_bytes(h, &bytes) != FLUSI_OK || bytes == 0) return 2;
    flusi_tuning t;
    if (flusi_get_tuning(h, &t) != FLUSI_OK || t.y_plan != 1) return 3;
    t.y_cols = 3;
    if (flusi_set_tuning(h, &t) != FLUSI_EINVAL) return 4;
    if (flusi_step(h, 1) != FLUSI_ESTATE) return 5;
    printf("%zu %d\n", bytes, t.y_tile_cols);
    return flusi_destroy(h);
}
""")
    exe = tmp_path / "use"
    libdir = os.path.dirname(fl.LIB_PATH)
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-lflusi", f"-Wl,-rpath,{libdir}"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert int(r.stdout.split()[0]) > 0


def test_build_id_is_the_source_hash(fl):
    """The loaded library was built from the sources present (the import
    refuses any other); the hash changes with the flags."""
    from paper_1506_06513_gb300 import _build
    assert fl.flusi_build_id() == _build.source_hash() == _build.built_hash()
    assert _build.source_hash(("-DX=1",)) != _build.source_hash()
    assert len(fl.flusi_build_id()) == 32


def test_fma_peak_validates_arguments(fl):
    f = C.c_double()
    for fp64, ms in ((2, 10.0), (0, 0.0), (1, -1.0), (0, 1e5)):
        assert fl.lib.flusi_fma_peak(fp64, ms, C.byref(f), None) == fl.FLUSI_EINVAL
    assert fl.lib.flusi_fma_peak(0, 10.0, None, None) == fl.FLUSI_EINVAL


def test_debug_inject_needs_a_state(fl):
    h = fl.flusi_create((16, 16, 16), (1.0, 1.0, 1.0), 0.1, 1e-2, fl.FLUSI_FP32)
    assert fl.lib.flusi_debug_inject(h, 0, 1, 1, 1, 0.0, 0.0) == fl.FLUSI_ESTATE
    assert fl.lib.flusi_debug_inject(None, 0, 1, 1, 1, 0.0, 0.0) == fl.FLUSI_EINVAL
    fl.flusi_destroy(h)
