"""Error of the reduced-precision forms of the step against the FP64 step on
the same input: FP32, and FP32 with the x pass's DFT stages as split-BF16
tensor-core products (bf16x2: hi + lo pieces; bf16x3: hi + mid + lo).

    python -m paper_1506_06513_gb300.accuracy --config single_wing --grid 256 --stroke
    python -m paper_1506_06513_gb300.accuracy --config model_insect --grid 512 --stroke
    python -m paper_1506_06513_gb300.accuracy --config model_insect --grid 512 --steps 1

All runs start from the same state and use the same fixed time step (the
CFL step at the peak wing-tip speed, below C_eta), so their time grids
coincide.  Reported per form: relative L2 error of u over all points and
components after the first step and after the last, and of the force/moment
history (the columns of the colours present).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_1506_06513_gb300 as fl  # noqa: E402
import workloads  # noqa: E402


def rel_l2(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run_form(cfg, insect, u0, steps, prec, chunk=1000):
    sim = fl.Solver(cfg, insect, precision=prec)
    sim.set_state(u0)
    sim.step(1)
    u1, _, _ = sim.get_state()
    rows = [sim.forces()[0]]
    done = 1
    t0 = time.perf_counter()
    while done < steps:
        k = min(chunk, steps - done)
        sim.step(k)
        rows.append(sim.forces()[0])
        done += k
    elapsed = time.perf_counter() - t0
    uN, t, n = sim.get_state()
    sim.close()
    return {"u1": u1, "uN": uN, "rows": np.vstack(rows), "t": t, "n": n, "s": elapsed}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--config", default="single_wing", choices=["single_wing", "model_insect"])
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--stroke", action="store_true", help="run one wingbeat")
    ap.add_argument("--forms", default="fp32,bf16x2,bf16x3",
                    help="comma-separated forms compared with fp64 (forms a grid cannot run are skipped)")
    args = ap.parse_args()

    make = workloads.config_single_wing if args.config == "single_wing" else workloads.config_model_insect
    cfg, ins = make(args.grid)
    dx = min(cfg["L"][i] / cfg["n"][i] for i in range(3))
    peak = workloads.peak_tip_speed(60 * math.pi / 180)
    dt = min(cfg.get("cfl", 0.1) * dx / peak, cfg["eta"])
    cfg = dict(cfg, dt_fixed=dt)
    steps = int(math.ceil(1.0 / dt)) if args.stroke else args.steps
    if cfg["init"][0] == "uniform" and cfg.get("u_inf", (0, 0, 0)) != (0, 0, 0):
        u0 = workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"])
    else:
        u0 = workloads.initial_field(cfg)
    ref = run_form(cfg, ins, u0, steps, "fp64")
    cols = [j for j in range(2, 20) if np.abs(ref["rows"][:, j]).max() > 0]
    res = {"config": f"{args.config} {args.grid}^3", "steps": steps, "dt": dt, "t_end": ref["t"],
           "seconds": {"fp64": ref["s"]}, "forms": {}}
    for prec in [f for f in args.forms.split(",") if f]:
        try:
            a = run_form(cfg, ins, u0, steps, prec)
        except fl.FlusiError as exc:
            res["forms"][prec] = {"unavailable": str(exc)}
            continue
        res["forms"][prec] = {
            "u_rel_l2_after_1_step": rel_l2(a["u1"], ref["u1"]),
            "u_rel_l2_after_last_step": rel_l2(a["uN"], ref["uN"]),
            "force_history_rel_l2": rel_l2(a["rows"][:, cols], ref["rows"][:, cols]),
            "energy_rel_diff_last": float(abs(a["rows"][-1, 20] - ref["rows"][-1, 20]) / ref["rows"][-1, 20])
            if ref["rows"][-1, 20] else None,
            "seconds": a["s"]}
        del a
    print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
