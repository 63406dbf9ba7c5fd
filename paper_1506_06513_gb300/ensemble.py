"""Batched ensemble of independent runs against the same runs one by one.

    python -m paper_1506_06513_gb300.ensemble [--count 40] [--steps 200]

The members (workloads.config_ensemble: uneven grids, flapping amplitudes,
frequencies and Reynolds numbers, FP32) are stepped twice from the same
state: one after another, each to the end with its own step graph, and
together, with one graph per ensemble step holding a step of every member
(flusi_ensemble_*), in which members of the same grid share one launch per
kernel.  Throughput is the sum over members of grid points times
steps, divided by the wall time between two device synchronizations.  The two
runs use the same kernels in the same order per member, so their final states
are compared bit for bit.  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import paper_1506_06513_gb300 as fl  # noqa: E402
import workloads  # noqa: E402


def _zero_states(solvers, fields):
    for s, u in zip(solvers, fields):
        s.set_state(u)


def run(count=40, steps=200, warmup=3, precision="fp32", seed=1506):
    import torch
    members = workloads.config_ensemble(count, seed)
    solvers = [fl.Solver(cfg, ins, precision=precision) for cfg, ins in members]
    fields = [workloads.initial_field(cfg, np.float32 if precision == "fp32" else np.float64)
              for cfg, _ in members]
    points = [int(np.prod(cfg["n"])) for cfg, _ in members]
    _zero_states(solvers, fields)
    ens = fl.Ensemble(solvers)

    def sync_all():
        for s in solvers:
            s.stream.synchronize()
        ens.sync()

    # warm-up: capture every member's own graph and the ensemble graph
    for s in solvers:
        s.step(warmup)
    ens.step(warmup)
    sync_all()
    groups, grouped = ens.batches()

    # one by one
    _zero_states(solvers, fields)
    sync_all()
    t0 = time.perf_counter()
    for s in solvers:
        s.step(steps)
        s.stream.synchronize()
    seq_s = time.perf_counter() - t0
    seq_states = [s.get_state(np.float32)[0] for s in solvers]
    seq_rows = [s.forces(cap=steps + 8)[0] for s in solvers]

    # batched
    _zero_states(solvers, fields)
    sync_all()
    t0 = time.perf_counter()
    ens.step(steps)
    ens.sync()
    bat_s = time.perf_counter() - t0
    identical = True
    for i, s in enumerate(solvers):
        u, _, nstep = s.get_state(np.float32)
        rows = s.forces(cap=steps + 8)[0]
        identical &= nstep == steps and np.array_equal(u, seq_states[i]) and np.array_equal(rows, seq_rows[i])
    work = float(sum(points)) * steps
    ens.close()
    for s in solvers:
        s.close()
    torch.cuda.synchronize()
    grids = {}
    for cfg, _ in members:
        k = "x".join(map(str, cfg["n"]))
        grids[k] = grids.get(k, 0) + 1
    return {"workload": f"{count} single-wing runs, uneven grids {grids}, {steps} steps each, "
                        f"{precision.upper()}, seed {seed}",
            "unit": "grid-point steps/s", "steps": steps,
            "batched": work / bat_s, "sequential": work / seq_s,
            "speedup": seq_s / bat_s, "batched_s": bat_s, "sequential_s": seq_s,
            "identical_to_one_by_one": bool(identical),
            "shared_launch_groups": groups, "members_in_groups": grouped}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--count", type=int, default=40)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    args = ap.parse_args()
    print(json.dumps(run(args.count, args.steps, precision=args.precision)), flush=True)


if __name__ == "__main__":
    main()
