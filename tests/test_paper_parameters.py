"""The Reynolds-number and boundary-layer helpers reproduce the parameter
values the paper prints (tests/golden/paper_parameters.json, each with its
section)."""
import json
import math
import os

import workloads

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden",
                                   "paper_parameters.json")))


def _round_to(x, ref):
    """x rounded to as many significant digits as the printed value has."""
    digits = len(repr(ref).replace("0.", "").lstrip("0").replace(".", ""))
    return float(f"{x:.{digits}g}")


def test_suzuki_wing():
    g = GOLD["suzuki_flapping_wing"]
    U = workloads.peak_tip_speed(g["phi_m_deg"] * math.pi / 180)
    nu = workloads.nu_from_re(g["Re"], U, g["B"])
    assert _round_to(nu, g["nu_printed"]) == g["nu_printed"]
    K = workloads.boundary_layer_points(nu, g["C_eta"], g["L"] / g["n"])
    assert _round_to(K, g["K_printed"]) == g["K_printed"]


def test_fruit_fly():
    g = GOLD["fruit_fly_hover"]
    U = workloads.mean_tip_speed(g["Phi_rad"] / 2)   # 2 Phi R f with Phi = 2 phi_m
    nu = workloads.nu_from_re(g["Re"], U, g["c_m"])
    K = workloads.boundary_layer_points(nu, g["C_eta"], g["L"] / g["n"])
    assert _round_to(K, g["K_printed"]) == g["K_printed"]


def test_butterfly():
    g = GOLD["butterfly_free_flight"]
    nu = workloads.nu_from_re(g["Re"], g["U_tip"], g["R"])
    K = workloads.boundary_layer_points(nu, g["C_eta"], g["L"] / g["n"])
    assert _round_to(K, g["K_printed"]) == g["K_printed"]


def test_falling_sphere_constant_K():
    g = GOLD["falling_sphere"]
    for n, eta in g["grids"]:
        K = workloads.boundary_layer_points(g["nu"], eta, g["Lx"] / n)
        assert _round_to(K, g["K_printed"]) == g["K_printed"]


def test_config_reynolds_numbers():
    """The single-wing and model-insect configurations use Re = U c / nu with
    the mean tip speed U = 4 phi_m f R and chord c = 0.3, and keep K inside the
    paper's recommended range 0.1 - 0.4 (Sec. 2.1)."""
    for make, re in ((workloads.config_single_wing, 100.0), (workloads.config_model_insect, 300.0)):
        cfg, ins = make()
        U = workloads.mean_tip_speed(60 * math.pi / 180)
        assert abs(U * 0.3 / cfg["nu"] - re) <= 1e-9 * re
        K = workloads.boundary_layer_points(cfg["nu"], cfg["eta"], cfg["L"][0] / cfg["n"][0])
        assert 0.1 <= K <= 0.4
