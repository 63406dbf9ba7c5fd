"""Pins of the oracle's realistic shapes (Sec. 3.2, 3.4): contour wings
R(theta) (Eq. Fourier_radious_wing) and a body with head and eye spheres
(Eq. DELTA_body_jerry), by closed forms of area, centroid and volume."""
import math

import numpy as np

import workloads


def _still(ins):
    ins["kinematics"] = {"phi": (0.0, [], []), "alpha": (0.0, [], []), "theta": (0.0, [], [])}
    return ins


def _contour_wing(L, n, contour, h=0.25):
    ins = _still(workloads.single_wing(L, n))
    ins["wing"] = (0.0, 0.0, 0.0, h)
    ins["contour"] = contour
    return ins


def test_disc_contour_is_a_disc_plate(orc):
    ins = _contour_wing((4.0,) * 3, (32,) * 3, {"center": (0.1, 0.4), "a0": 0.8}, h=0.1)
    rng = np.random.default_rng(4)
    for _ in range(200):
        xw = rng.uniform(-0.8, 0.8, 3) + np.array([0.1, 0.4, 0.0])
        r = math.hypot(xw[0] - 0.1, xw[1] - 0.4)
        expect = max(abs(xw[2]) - 0.05, r - 0.4)
        assert abs(orc.wing_distance(ins, xw) - expect) <= 1e-15


def _wing_frame_points(orc, cfg, ins):
    """Wing-frame coordinates of every grid point of a still wing."""
    fr = orc.frames(ins, 0.0)
    nx, ny, nz = cfg["n"]
    L = cfg["L"]
    z, y, x = np.meshgrid(np.arange(nz) * L[2] / nz, np.arange(ny) * L[1] / ny,
                          np.arange(nx) * L[0] / nx, indexing="ij")
    X = np.stack([x, y, z]) - np.asarray(ins["x_cntr"])[:, None, None, None]
    xb = np.einsum("ij,jzyx->izyx", fr["M_body"], X) - np.asarray(ins["pivot_l"])[:, None, None, None]
    return np.einsum("ij,jzyx->izyx", fr["M_wing"][0] @ fr["M_stroke"][0], xb)


def test_contour_area_and_orientation(orc):
    """Area of a polar curve: (1/2) int R^2 = pi (a0/2)^2 + (pi/2) sum (a_i^2 + b_i^2);
    R = c + b sin(theta) puts the centroid at y = pi (c^2 b + b^3/4) / A towards +y^(w)."""
    h = 0.25
    contour = {"center": (0.2, 0.6), "a0": 1.0, "a": [0.1, 0.0], "b": [0.08, 0.05]}
    c = 0.5
    area = math.pi * c * c + 0.5 * math.pi * (0.1 ** 2 + 0.08 ** 2 + 0.05 ** 2)
    errs = []
    for n in (48, 96):
        cfg = {"n": (n,) * 3, "L": (4.0,) * 3, "nu": 0.0, "eta": 1.0}
        ins = _contour_wing(cfg["L"], cfg["n"], contour, h)
        chi, col, us = orc.mask_grid(cfg, ins, 0.0)
        vol = chi.sum() * (4.0 / n) ** 3
        errs.append(abs(vol - area * h) / (area * h))
        assert set(np.unique(col)) == {0, 2}
    assert errs[0] / errs[1] > 2.0 and errs[1] < 0.03
    # centroid of a pure sine contour
    b = 0.1
    contour = {"center": (0.0, 0.0), "a0": 2 * c, "b": [b]}
    A = math.pi * c * c + 0.5 * math.pi * b * b
    cfg = {"n": (96,) * 3, "L": (4.0,) * 3, "nu": 0.0, "eta": 1.0}
    ins = _contour_wing(cfg["L"], cfg["n"], contour, h)
    chi, _, _ = orc.mask_grid(cfg, ins, 0.0)
    xw = _wing_frame_points(orc, cfg, ins)
    yc = (chi * xw[1]).sum() / chi.sum()
    xc = (chi * xw[0]).sum() / chi.sum()
    assert abs(yc - math.pi * (c * c * b + b ** 3 / 4) / A) <= 3e-3
    assert abs(xc) <= 3e-3


def test_head_and_eyes_join_the_thorax(orc):
    """Thorax (a, b) + head sphere + two eye spheres, disjoint: the body volume
    converges to the sum of the four volumes; the eyes mirror in y^(b)."""
    a, b, rh, re = 0.5, 0.12, 0.12, 0.06
    vol = 4 / 3 * math.pi * (a * b * b + rh ** 3 + 2 * re ** 3)
    errs = []
    for n in (48, 96):
        L = (2.0,) * 3
        cfg = {"n": (n,) * 3, "L": L, "nu": 0.0, "eta": 1.0}
        ins = {"body": "ellipsoid", "nwings": 0, "profile": "cos", "c_smth": 1.0,
               "x_cntr": (1.0, 1.0, 1.0), "body_axes": (a, b),
               "head": ((0.65, 0.0, 0.0), rh), "eyes": ((0.2, 0.3, 0.0), re)}
        chi, col, _ = orc.mask_grid(cfg, ins, 0.0)
        errs.append(abs(chi.sum() * (2.0 / n) ** 3 - vol) / vol)
        assert set(np.unique(col)) == {0, 1}
        # mirror y -> 2 - y maps grid row j to (n - j) mod n
        mirror = chi[:, (-np.arange(n)) % n, :]
        assert np.abs(mirror - chi).max() <= 1e-12
    assert errs[0] / errs[1] > 2.5 and errs[1] < 0.03
    # at the head's centre the body distance is -r_head, at an eye's centre -r_eye
    assert abs(orc.body_distance(ins, (0.65, 0.0, 0.0)) + rh) <= 1e-15
    assert abs(orc.body_distance(ins, (0.2, -0.3, 0.0)) + re) <= 1e-15


def _curved(a=0.5, b=0.12, arc=(0.6, -0.2, -0.7), x_cntr=(1.0, 1.0, 1.0)):
    return {"body": "curved", "nwings": 0, "profile": "cos", "c_smth": 1.0, "x_cntr": x_cntr,
            "body_axes": (a, b), "body_arc": arc}


def _arc_point(arc, s):
    """Centre-line point at arc length s from the point nearest the body
    origin's direction, and the in-plane unit normal there."""
    rc, xc, zc = arc
    th = math.atan2(-xc, -zc) + s / rc
    nrm = np.array([math.sin(th), 0.0, math.cos(th)])
    return np.array([xc, 0.0, zc]) + rc * nrm, nrm


def test_curved_thorax_surface_points(orc):
    """Points built on the tube (centre line plus the local radius along any
    normal) are at distance 0; the centre line is at minus the local radius;
    beyond the ends the distance is that to the end point."""
    a, b, arc = 0.5, 0.12, (0.6, -0.2, -0.7)
    ins = _curved(a, b, arc)
    rng = np.random.default_rng(7)
    for _ in range(100):
        s = rng.uniform(-0.98 * a, 0.98 * a)
        phi = rng.uniform(0, 2 * math.pi)
        c, nrm = _arc_point(arc, s)
        rho = b * math.sqrt(1 - (s / a) ** 2)
        p = c + rho * (math.cos(phi) * nrm + math.sin(phi) * np.array([0.0, 1.0, 0.0]))
        assert abs(orc.body_distance(ins, p)) <= 1e-14
        assert abs(orc.body_distance(ins, c) + rho) <= 1e-14
        assert abs(orc.body_distance(ins, p * [1, -1, 1]) - orc.body_distance(ins, p)) <= 1e-15
    end, nrm = _arc_point(arc, a)
    tangent = np.array([nrm[2], 0.0, -nrm[0]])      # direction of growing s
    for d in (0.01, 0.1, 0.3):
        assert abs(orc.body_distance(ins, end + d * tangent) - d) <= 1e-14


def test_curved_thorax_straightens_for_a_large_radius(orc):
    """A centre-line circle of radius R through the origin tends to the x
    axis: the distance tends to the straight thorax's, at O(|x|^2 / R)."""
    a, b = 0.5, 0.12
    rng = np.random.default_rng(8)
    pts = rng.uniform(-0.7, 0.7, (200, 3)) * [1, 0.3, 0.3]
    straight = {"body": "ellipsoid", "nwings": 0, "x_cntr": (0, 0, 0), "body_axes": (a, b)}
    for R in (1e2, 1e4):
        curved = _curved(a, b, (R, 0.0, -R), (0, 0, 0))
        err = max(abs(orc.body_distance(curved, p) - orc.body_distance(straight, p)) for p in pts)
        assert err <= 2.0 / R
    assert err <= 2e-4


def test_curved_thorax_volume_and_centroid(orc):
    """Circular cross-sections centred on the arc.  In polar coordinates about
    the circle's centre the volume element is (1 + u/r_c) ds du dy, u the
    outward offset from the centre line, so the volume is int A(s) ds =
    (4/3) pi a b^2, the straight ellipsoid's (Pappus), and the first moment is
    int (A(s) C(s) + (pi rho^4 / 4) n(s) / r_c) ds with n the outward normal
    (quadrature along the arc)."""
    from scipy.integrate import quad
    a, b, arc = 0.5, 0.12, (0.6, -0.2, -0.7)
    vol = 4 / 3 * math.pi * a * b * b
    area = lambda s: math.pi * b * b * (1 - (s / a) ** 2)

    def moment(s, i):
        c, nrm = _arc_point(arc, s)
        return area(s) * c[i] + area(s) ** 2 / (4 * math.pi) * nrm[i] / arc[0]
    cen = np.array([quad(moment, -a, a, args=(i,))[0] for i in range(3)]) / vol
    errs = []
    for n in (48, 96):
        L = (2.0,) * 3
        cfg = {"n": (n,) * 3, "L": L, "nu": 0.0, "eta": 1.0}
        chi, col, _ = orc.mask_grid(cfg, _curved(a, b, arc), 0.0)
        dv = (2.0 / n) ** 3
        errs.append(abs(chi.sum() * dv - vol) / vol)
        assert set(np.unique(col)) == {0, 1}
        z, y, x = np.meshgrid(*(np.arange(n) * 2.0 / n,) * 3, indexing="ij")
        got = np.array([(chi * q).sum() / chi.sum() for q in (x, y, z)]) - 1.0
        assert np.abs(got - cen).max() <= (6e-4 if n == 48 else 1.2e-4)
        mirror = chi[:, (-np.arange(n)) % n, :]
        assert np.abs(mirror - chi).max() <= 1e-12
    assert errs[0] / errs[1] > 2.0 and errs[1] < 0.03
