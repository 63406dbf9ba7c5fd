#!/usr/bin/env python
"""Benchmark of the penalized pseudo-spectral Navier-Stokes AB2 step on GB300.

Workload: the model insect (ellipsoidal body + two flapping plates, Re 300,
inflow 0.25, C_eta = 1e-3, CFL 0.1 adaptive dt) on a 512^3 grid over a 4^3
box, FP32 state; the same step in FP64 is timed beside it.  Reported: grid-point
steps/s of the whole job, the dominant kernel against the measured HBM peak,
the stage-model fraction, an end-to-end figure through the C-ABI with host
buffers, and the CPU oracle timed on a bounded sample.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs an independent replica on its own GPU
(one step has no exchange between replicas: each is a whole simulation) and
rank 0 prints one JSON line.  The solver's FFT plans and tile shapes are
autotuned first (flusi_autotune; --no-autotune keeps the defaults).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "AB2 grid-point steps/s at 512³, FP32 vs FP64 on 1 GB300; % of HBM roofline"
UNIT = "grid-point steps/s"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="flusi", choices=["flusi", "reference"])
    ap.add_argument("--workload", default="model_insect", choices=["model_insect", "turbulent_insect"],
                    help="model insect in uniform inflow plus waves (512^3 by default), or the "
                         "model insect in seeded isotropic turbulent inflow (1024^3 by default)")
    ap.add_argument("--grid", type=int, default=None)
    ap.add_argument("--rk4", action="store_true",
                    help="time the RK4 scheme (explicit diffusion, four right-hand sides per step)")
    ap.add_argument("--wake", action="store_true",
                    help="add the wake-removal terms: a vorticity sponge (C_sp 0.1) 32 grid "
                         "points deep at the x and y ends and a Dirichlet layer 4 points deep at the x end")
    ap.add_argument("--insect", default="model", choices=["model", "realistic", "curved"],
                    help="model: ellipsoid thorax and plate wings; realistic: thorax, head, eyes and "
                         "16-harmonic contour wings; curved: the realistic insect on a curved thorax")
    ap.add_argument("--flight", action="store_true",
                    help="free flight (Sec. 3.6) with the power columns: the body state advances "
                         "every step (mass 400, J_body (2, 5, 5), g 9.81, wing J set)")
    ap.add_argument("--shape", default=None,
                    help="nx,ny,nz: a reduced grid of the same box and insect (profiling)")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16x2", "bf16x3"],
                    help="the timed leg's form: FP32, or FP32 with the x pass's DFT stages as split-BF16 "
                         "tensor-core products (two or three pieces)")
    ap.add_argument("--no-split", action="store_true",
                    help="skip the split-BF16 legs timed beside the FP32 one")
    ap.add_argument("--split-steps", type=int, default=50)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=None,
                    help="steps of the end-to-end job (default: --steps, the device-timed job's length)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default FFT plans and tiles instead of flusi_autotune's choice")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-grid", type=int, default=256,
                    help="grid of the all-cores oracle sample of the CPU baseline (512: the bench's own)")
    ap.add_argument("--cpu-steps", type=int, default=2)
    ap.add_argument("--oracle-time", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-yardstick", action="store_true",
                    help="skip timing cuFFT on the step's nine 3-D transforms")
    ap.add_argument("--no-ensemble", action="store_true",
                    help="skip the 40-run uneven ensemble, batched against one by one")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": FALLBACK_HBM_GBS}, "fallback"


# ------------------------------------------------------------------ workload

def cutoff(n):
    return n // 3


def spectral_sizes(n):
    nx, ny, nz = n
    Mx, My, Mz = cutoff(nx) + 1, 2 * cutoff(ny) + 1, 2 * cutoff(nz) + 1
    return Mx, My, Mz


def kernel_bytes(n, s, wake=False):
    """Algorithmic bytes per launch of each kernel: every input it must read
    and every output it must write once, complex values of 2s bytes over the
    kept modes (x: Mx of nx/2+1; y: My of ny; z: Mz of nz).  With the wake
    terms the vorticity makes a second x round trip and three more fields
    go through the forward y and z passes and the update."""
    nx, ny, nz = n
    Mx, My, Mz = spectral_sizes(n)
    c = 2 * s
    A = nz * My * Mx * c          # one field after the z transform
    B = nz * ny * Mx * c          # one field after the y transform
    S = Mz * My * Mx * c          # one state field
    f = 6 if wake else 3          # fields of the forward y and z passes
    out = {
        "zinv_curl": 3 * S + 6 * A,
        "yinv": 6 * A + 6 * B,
        "xpass_phys": 6 * B + 3 * B,
        "xpass_tc": 6 * B + 3 * B,
        "yfwd": f * B + f * A,
        "zfwd": f * A + f * S,
        "update": f * S + 2 * 3 * S + 2 * 3 * S,
        "kinematics": 0,
        "scalars": 0,
    }
    if wake:
        out["sponge_x"] = 3 * B + 3 * B
    return out


# Nominal FP32 rate: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def xpass_flops(n, wake=False):
    """Algorithmic FP32 flops of one physical x pass: per row, the 6 inverse
    and 3 forward real transforms as half-length complex FFTs at the
    conventional 5 m log2 m flops (m = nx/2), their mirror steps (one complex
    multiply and three complex adds, 14 flops, per output), and per point the
    Lamb vector, energy and max |u| (15 flops).  The penalization of masked
    rows is left out (its share depends on the insect)."""
    nx, ny, nz = n
    m = nx // 2
    lines = 9 + (6 if wake else 0)
    per_row = lines * (5 * m * math.log2(m) + 14 * m) + 15 * nx
    return ny * nz * per_row


def xpass_tc_flops(n, pieces):
    """Tensor-core flops of one split-BF16 x pass (2 M N K per product of an
    M x K and a K x N matrix): per tile of 128/Q rows (nx = 32 Q), the six
    inverse and three forward line transforms take a 16-row stage of Q-point
    DFTs (16/Q products of 128 x 2Q x 2Q) and a Q-row stage of 16-point DFTs
    (one product of 128 x 32 x 32), each product taken P(P+1)/2 times over
    the operand pieces."""
    nx, ny, nz = n
    Q = nx // 32
    rows_per_tile = 128 // Q
    tiles = -(-(ny * nz) // rows_per_tile)
    per_line = (16 // Q) * 128 * (2 * Q) ** 2 + 128 * 32 * 32
    return 2 * tiles * 9 * per_line * pieces * (pieces + 1) // 2


def kernel_flops(n, wake=False):
    """Algorithmic flops per launch of each kernel: every 1-D complex FFT of m
    points at the conventional 5 m log2 m (the x pass as xpass_flops), the
    curl, projection and IF-AB2 update at 60 flops per kept mode (three
    components).  The FP64 path's arithmetic roofline divides by these."""
    nx, ny, nz = n
    Mx, My, Mz = spectral_sizes(n)
    f = 6 if wake else 3
    fft = lambda m: 5 * m * math.log2(m)
    out = {"zinv_curl": 5 * My * Mx * fft(nz) + 12 * Mz * My * Mx,
           "yinv": 6 * nz * Mx * fft(ny),
           "xpass_phys": xpass_flops(n, wake),
           "yfwd": f * nz * Mx * fft(ny),
           "zfwd": f * My * Mx * fft(nz),
           "update": 60 * Mz * My * Mx,
           "kinematics": 0, "scalars": 0}
    out["xpass_tc"] = out["xpass_phys"]
    return out


def stage_model_bytes(n, s):
    """Stage-model bytes per step: 6 inverse + 3 forward full FFTs read and
    written once, the physical pass and the spectral pass over the full half
    spectrum: B = 24 F_c + 18 F_r."""
    nx, ny, nz = n
    Fr = s * nx * ny * nz
    Fc = 2 * s * (nx // 2 + 1) * ny * nz
    return 24 * Fc + 18 * Fr


def workload_setup(args):
    if args.workload == "turbulent_insect":
        cfg, ins = workloads.config_turbulent_insect(args.grid or 1024)
    else:
        cfg, ins = workloads.config_model_insect(args.grid or 512)
    if args.shape:
        shape = tuple(int(v) for v in args.shape.split(","))
        cfg = dict(cfg, n=shape)
        ins = workloads.model_insect(cfg["L"], shape)
    if args.insect != "model":
        make = workloads.realistic_insect if args.insect == "realistic" else workloads.curved_insect
        ins = dict(make(cfg["L"], cfg["n"]), kinematics=ins["kinematics"])
    if args.rk4:
        cfg = dict(cfg, time_scheme="rk4")
    if args.flight:
        if args.rk4:
            raise SystemExit("free flight runs with the AB2 scheme only")
        ins = in_free_flight(ins)
    if args.wake:
        d = [cfg["L"][i] / cfg["n"][i] for i in range(3)]
        cfg = dict(cfg, sponge_c=0.1, sponge_width=(32 * d[0], 32 * d[1], 0.0),
                   layer_width=(4 * d[0], 0.0, 0.0))
    return cfg, ins


def bench_field(cfg, device):
    """The workload's initial velocity in float32: uniform inflow plus
    band-limited divergence-free waves (host numpy), or the seeded turbulent
    inflow (built on the device, a torch tensor)."""
    if cfg["init"][0] == "turbulent":
        return workloads.turbulent_field(cfg["n"], cfg["L"], mean=cfg["u_inf"], seed=cfg["init"][1],
                                         device=f"cuda:{device}")
    return workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"]).astype(np.float32)


# ------------------------------------------------------------------- clocks

class Clocks:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd[1:1] = ["-i", self.uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# --------------------------------------------------------------- CPU oracle

def in_free_flight(ins):
    """The insect in free flight (Sec. 3.6) with a wing tensor of inertia for
    the power columns; heavy enough that the impulsive start in the inflow
    moves it by a fraction of its length over a few hundred steps."""
    return dict(ins, J_wing=(2e-2, 1e-3, 2e-2, 1e-4, 0.0, 0.0),
                free_flight={"mass": 400.0, "gravity": 9.81, "J_body": (2.0, 5.0, 5.0)})


def oracle_workload(workload, n, flight=False, insect="model"):
    """The workload at a reduced grid n^3 for the oracle: (cfg, insect, u0 FP64)."""
    if workload == "turbulent_insect":
        cfg, ins = workloads.config_turbulent_insect(n)
        u0 = workloads.turbulent_field(cfg["n"], cfg["L"], mean=cfg["u_inf"], seed=cfg["init"][1])
    else:
        cfg, ins = workloads.config_model_insect(n)
        u0 = workloads.shear_waves(cfg["n"], cfg["L"], mean=cfg["u_inf"])
    if insect != "model":
        make = workloads.realistic_insect if insect == "realistic" else workloads.curved_insect
        ins = dict(make(cfg["L"], cfg["n"]), kinematics=ins["kinematics"])
    return cfg, in_free_flight(ins) if flight else ins, u0


def host_cpu():
    """CPU model and logical core count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        import platform
        model = platform.processor() or platform.machine()
    return {"cpu_model": model, "nproc": os.cpu_count()}


def oracle_time(workload, n, steps, threads, flight=False, insect="model"):
    """One oracle timing in a fresh process (the single-threaded build, or the
    OpenMP build on `threads` threads): set_state untimed, then `steps` steps."""
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    cmd = [sys.executable, os.path.abspath(__file__), "--oracle-time",
           f"{workload},{n},{steps},{int(threads > 1)},{int(flight)},{insect}"]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        raise RuntimeError(f"oracle timing failed: {r.stderr[-500:]}")
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_time_main(spec):
    import oracle
    workload, n, steps, omp, flight, insect = spec.split(",")
    n, steps = int(n), int(steps)
    if int(omp) and not oracle.use_openmp():
        raise SystemExit("the OpenMP build of the oracle is not available on this host")
    cfg, ins, u0 = oracle_workload(workload, n, bool(int(flight)), insect)
    sim = oracle.Simulation(cfg, ins)
    sim.set_state(u0)
    t0 = time.perf_counter()
    sim.step(steps)
    el = time.perf_counter() - t0
    print(json.dumps({"n": n, "steps": steps, "seconds": el, "threads": oracle.threads(),
                      "value": n ** 3 * steps / el}))


def oracle_sample(workload, flight=False, insect="model", n_all=256, steps_all=2, n_one=128, steps_one=2):
    """The oracle (C, FP64) as it stands on the same workload at reduced grids:
    the OpenMP build on every host core (the reported value) and the plain
    build on one core beside it; grid-point steps/s."""
    host = host_cpu()
    cores = host["nproc"] or 1
    one = oracle_time(workload, n_one, steps_one, 1, flight, insect)
    try:
        alls = oracle_time(workload, n_all, steps_all, cores, flight, insect)
    except RuntimeError:
        alls = None
    main = alls or one
    what = (f"the same workload at {main['n']}^3 (same box, body, wings, Re, C_eta, inflow), "
            f"{main['steps']} steps, FP64 C oracle on {main['threads']} thread(s), {main['seconds']:.1f} s")
    return {"value": main["value"], "unit": UNIT, "cores": main["threads"], "kind": "oracle",
            "sample": what, "host": host,
            "single_thread": {"value": one["value"], "grid": one["n"], "steps": one["steps"],
                              "seconds": round(one["seconds"], 2)},
            "all_cores": None if alls is None else {"value": alls["value"], "grid": alls["n"],
                                                    "steps": alls["steps"], "threads": alls["threads"],
                                                    "seconds": round(alls["seconds"], 2)}}


class Ranks:
    """Replicas, one process per GPU: a barrier and the maximum over ranks of
    a host number.  No data moves between ranks; `dist` is torch.distributed
    (NCCL between GPUs, gloo in the CPU tests) or None for one process."""

    def __init__(self, dist, device):
        self.dist, self.device = dist, device

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x):
        if self.dist is None:
            return x
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


def whole_job_rate(points, steps, world, ms_max):
    """Grid-point steps/s of all replicas: every rank runs `steps` steps of a
    `points`-point grid; the job takes the slowest rank's time."""
    return points * steps * world / (ms_max * 1e-3)


# ------------------------------------------------------------------ own arm

def run_flusi(args):
    import torch
    import paper_1506_06513_gb300 as fl

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    ranks = Ranks(dist, torch.device("cuda", local))
    barrier, allmax = ranks.barrier, ranks.max

    cfg, ins = workload_setup(args)
    N = int(np.prod(cfg["n"]))
    u0 = bench_field(cfg, local)
    peaks, peak_src = measured_peaks()
    hbm = float(peaks.get("hbm_gbs", FALLBACK_HBM_GBS))

    # ---- measured FMA peaks (dependent-FMA chains on every SM, CUDA events)
    fp32_peak, _ = fl.flusi_fma_peak(0, 30.0)
    fp64_peak, _ = fl.flusi_fma_peak(1, 30.0)
    alu_src = "measured: flusi_fma_peak (independent chains of dependent FMAs, every SM, best of 3)"

    # ---- FP32, device-resident timed region
    sim = fl.Solver(cfg, ins, precision=args.precision, device=local)
    sim.set_state(u0)
    # plans and tile shapes timed on this GPU; the state is left as it was
    tuning = sim.tuning() if args.no_autotune else sim.autotune(steps=3)
    sim.step(args.warmup)
    sim.sync()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
        if uuid and not uuid.startswith("GPU-"):
            uuid = "GPU-" + uuid
    except Exception:
        uuid = None
    clocks = Clocks(uuid)
    clocks.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    ev0.record(sim.stream)
    sim.step(args.steps)
    ev1.record(sim.stream)
    torch.cuda.synchronize()
    barrier()
    ms = ev0.elapsed_time(ev1)
    # the last force row of the timed steps (t, dt, ..., E_kin, max|u| at its start)
    rows_t, _ = sim.forces()
    last_row = None
    if len(rows_t):
        lr = rows_t[-1]
        last_row = {"rows": int(len(rows_t)), "t": float(lr[0]), "dt": float(lr[1]),
                    "E_kin": float(lr[20]), "u_max": float(lr[21]), "finite": bool(np.isfinite(rows_t).all())}
    # the step timed again: median of 5 repeats of 50 graph steps
    reps = []
    for _ in range(5):
        k = 50
        torch.cuda.synchronize()
        ev0.record(sim.stream)
        sim.step(k)
        ev1.record(sim.stream)
        torch.cuda.synchronize()
        reps.append(ev0.elapsed_time(ev1) / k)
    clk = clocks.stop()
    sim.sync()
    ms_max = allmax(ms)
    value = whole_job_rate(N, args.steps, world, ms_max)
    ms_per_step = ms_max / args.steps
    repeats = {"ms_per_step": [round(r, 4) for r in reps], "steps_each": 50,
               "median_ms_per_step": round(statistics.median(reps), 4),
               "median_value": N * 1e3 / statistics.median(reps) * world}
    kps = fl.flusi_kernels_per_step(sim.h)

    # ---- per-kernel durations (CUDA events on the solver stream)
    prof = sim.profile(10)
    kb = kernel_bytes(cfg["n"], 4, wake=args.wake)
    dom = max(prof, key=prof.get)
    ach = kb[dom.split(".")[0]] / (prof[dom] * 1e-3) / 1e9
    traffic = None
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            tr = json.load(f)
        ent = tr.get(f"{dom}@{'x'.join(map(str, cfg['n']))}/{args.precision}")
        if ent and ent.get("source_hash") == source_hash(ent.get("sources")):
            traffic = ent["bytes_per_launch"]
    except (OSError, ValueError):
        pass
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(ach, 1), "peak": hbm,
                "unit": "GB/s", "frac": round(ach / hbm, 4), "traffic": traffic,
                "algorithmic_bytes": kb[dom.split(".")[0]], "peak_source": f"{peak_src} (hbm_gbs, copy)"}
    if dom.split(".")[0] == "xpass_tc":
        pieces = 2 if args.precision == "bf16x2" else 3
        tfl = xpass_tc_flops(cfg["n"], pieces)
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        tf = tfl / (prof[dom] * 1e-3) / 1e12
        roofline["tensor"] = {"achieved": round(tf, 2), "peak": bf16, "unit": "TFLOP/s",
                              "frac": round(tf / bf16, 4), "flop_per_launch": tfl,
                              "peak_source": f"{peak_src} (bf16_tflops, cuBLAS burst)"}
    if dom.split(".")[0] == "xpass_phys":
        # the same kernel against the FP32 arithmetic roofline (it is bound by
        # instruction issue, between the two)
        fl_x = xpass_flops(cfg["n"], args.wake)
        tf = fl_x / (prof[dom] * 1e-3) / 1e12
        peak32 = fp32_peak / 1e12
        roofline["alu"] = {"achieved": round(tf, 2), "peak": round(peak32, 2), "unit": "TFLOP/s",
                           "frac": round(tf / peak32, 4), "flop_per_launch": fl_x, "peak_source": alu_src,
                           "nominal_peak": round(FP32_PEAK_TFLOPS, 1)}
    base = lambda k: k.split(".")[0]    # RK4 stages 2..4 carry a ".q" suffix
    kernels = {k: {"ms": round(v, 4),
                   "GB_s": round(kb[base(k)] / (v * 1e-3) / 1e9, 1) if kb[base(k)] else None}
               for k, v in prof.items()}
    stage = stage_model_bytes(cfg["n"], 4)
    step_bytes = sum(kb[k.split(".")[0]] for k in prof)   # every launch of the step

    # ---- end to end through the C-ABI with pinned host buffers
    e2e_steps = args.e2e_steps if args.e2e_steps else args.steps
    if isinstance(u0, np.ndarray):
        host_in = torch.from_numpy(u0).pin_memory().numpy()
    else:
        host_in = u0.cpu().pin_memory().numpy()
    host_out = torch.empty(tuple(u0.shape), dtype=torch.float32).pin_memory().numpy()
    host_rows = torch.zeros((e2e_steps, fl.FORCE_COLS), dtype=torch.float64).pin_memory().numpy()
    rows_total = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fl.flusi_set_state(sim.h, host_in, fl.FLUSI_HOST_FP32)
    for _ in range(e2e_steps):
        if not args.flight:      # in free flight the body state lives on the device
            fl.flusi_set_kinematics(sim.h, sim.insect)
        fl.flusi_step(sim.h, 1)
        cnt, _ = fl.flusi_forces_async(sim.h, host_rows, rows_total)
        rows_total += cnt
    fl.flusi_get_state(sim.h, host_out, fl.FLUSI_HOST_FP32)   # waits for the steps and the row copies
    e2e_s = time.perf_counter() - t0
    assert rows_total == e2e_steps and np.isfinite(host_out[:, ::64, ::64, ::64]).all()
    assert np.isfinite(host_rows).all() and (host_rows[:, 1] > 0).all() and np.all(np.diff(host_rows[:, 0]) > 0)
    e2e_s = allmax(e2e_s)
    state_bytes = host_in.nbytes
    e2e = {"value": whole_job_rate(N, e2e_steps, world, e2e_s * 1e3), "unit": UNIT, "steps": e2e_steps,
           "h2d_bytes_per_step": (state_bytes + (0 if args.flight else e2e_steps * ctypes.sizeof(fl.Insect)))
                                 / e2e_steps,
           "d2h_bytes_per_step": (state_bytes + e2e_steps * fl.FORCE_COLS * 8) / e2e_steps,
           "what": "set_state from pinned host FP32, per step set_kinematics (H2D) + step + "
                   "force-row drain (D2H into pinned rows, flusi_forces_async: no per-step wait), "
                   "get_state to pinned host FP32"}
    sim.close()
    del host_in, host_out

    # ---- the split-BF16 forms beside it: same workload, the FP32 leg's tuning
    split = None
    if not args.no_split and args.precision == "fp32":
        split = {}
        bf16 = float(peaks.get("bf16_tflops", 1900.0))
        for form, pieces in (("bf16x2", 2), ("bf16x3", 3)):
            try:
                s2 = fl.Solver(cfg, ins, precision=form, device=local)
            except fl.FlusiError as exc:   # grids whose nx has no tensor-core x pass
                split[form] = {"unavailable": str(exc)}
                continue
            s2.set_state(u0)
            fl.flusi_set_tuning(s2.h, **{k: tuning[k] for k in fl.TUNING_SETTINGS})
            s2.step(3)
            s2.sync()
            barrier()
            torch.cuda.synchronize()
            ev0.record(s2.stream)
            s2.step(args.split_steps)
            ev1.record(s2.stream)
            torch.cuda.synchronize()
            ms2 = allmax(ev0.elapsed_time(ev1)) / args.split_steps
            prof2 = s2.profile(5)
            s2.close()
            tc_ms = prof2.get("xpass_tc")
            tfl = xpass_tc_flops(cfg["n"], pieces)
            split[form] = {"value": whole_job_rate(N, args.split_steps, world, ms2 * args.split_steps),
                           "unit": UNIT, "ms_per_step": ms2, "steps": args.split_steps,
                           "vs_fp32": ms_per_step / ms2,
                           "kernels_ms": {k: round(v, 3) for k, v in prof2.items()},
                           "xpass_tc": None if tc_ms is None else {
                               "ms": round(tc_ms, 4),
                               "GB_s": round(kb["xpass_phys"] / (tc_ms * 1e-3) / 1e9, 1),
                               "tensor_TFLOP_s": round(tfl / (tc_ms * 1e-3) / 1e12, 2),
                               "tensor_frac": round(tfl / (tc_ms * 1e-3) / 1e12 / bf16, 4),
                               "flop_per_launch": tfl}}

    # ---- FP64 beside it
    fp64 = None
    if not args.no_fp64:
        sim64 = fl.Solver(cfg, ins, precision="fp64", device=local)
        sim64.set_state(u0)
        tuning64 = sim64.tuning() if args.no_autotune else sim64.autotune(steps=1)
        sim64.step(2)
        sim64.sync()
        barrier()
        torch.cuda.synchronize()
        ev0.record(sim64.stream)
        sim64.step(args.fp64_steps)
        ev1.record(sim64.stream)
        torch.cuda.synchronize()
        ms64 = allmax(ev0.elapsed_time(ev1))
        sim64.sync()
        prof64 = sim64.profile(2)
        sim64.close()
        v64 = whole_job_rate(N, args.fp64_steps, world, ms64)
        # the FP64 path against max(bytes / HBM, flops / FP64 peak), per kernel and per step
        kb64, kf = kernel_bytes(cfg["n"], 8, wake=args.wake), kernel_flops(cfg["n"], wake=args.wake)
        dom64 = max(prof64, key=prof64.get)
        b64, f64 = kb64[dom64.split(".")[0]], kf[dom64.split(".")[0]]
        t64 = prof64[dom64] * 1e-3
        step_b64 = sum(kb64[k.split(".")[0]] for k in prof64)
        step_f64 = sum(kf[k.split(".")[0]] for k in prof64)
        step_s = ms64 / args.fp64_steps * 1e-3
        fp64 = {"value": v64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps,
                "steps": args.fp64_steps, "fp32_speedup": value / v64,
                "kernels_ms": {k: round(v, 3) for k, v in prof64.items()}, "tuning": tuning64,
                "roofline": {"kernel": dom64, "bound": "fp64" if f64 / fp64_peak > b64 / (hbm * 1e9) else "hbm",
                             "achieved": round(f64 / t64 / 1e12, 3), "peak": round(fp64_peak / 1e12, 3),
                             "unit": "TFLOP/s", "frac": round(f64 / t64 / fp64_peak, 4),
                             "flop_per_launch": f64, "bytes_per_launch": b64,
                             "fp64_floor_ms": round(f64 / fp64_peak * 1e3, 3),
                             "hbm_floor_ms": round(b64 / (hbm * 1e9) * 1e3, 3),
                             "peak_source": alu_src},
                "step_roofline": {"flop_per_step": step_f64, "bytes_per_step": step_b64,
                                  "floor_ms": round(max(step_f64 / fp64_peak, step_b64 / (hbm * 1e9)) * 1e3, 3),
                                  "frac": round(max(step_f64 / fp64_peak, step_b64 / (hbm * 1e9)) / step_s, 4)}}
    del u0

    yardstick = None
    if not args.no_yardstick:
        from paper_1506_06513_gb300.yardstick import run as run_yardstick
        yardstick = run_yardstick(cfg["n"][0]) if len(set(cfg["n"])) == 1 else None
        if yardstick:
            yardstick["step_ms_over_cufft_ms"] = ms_per_step / yardstick["ms"]
        torch.cuda.empty_cache()

    ensemble = None
    if not args.no_ensemble:
        from paper_1506_06513_gb300.ensemble import run as run_ensemble
        ensemble = run_ensemble(40, 200)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = oracle_sample(args.workload, flight=args.flight, insect=args.insect, n_all=args.cpu_grid,
                            steps_all=args.cpu_steps)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": dict(workload_config(cfg["n"], world, args.workload, args.wake, args.flight, args.insect),
                       precision=args.precision),
        "roofline": roofline,
        "repeats": repeats,
        "last_row": last_row,
        "stage_model": {"bytes_per_step": stage, "frac_of_peak": round(stage / (ms_per_step * 1e-3) / 1e9 / hbm, 4),
                        "frac_of_nominal_8TBs": round(stage / (ms_per_step * 1e-3) / 8e12, 4),
                        "kernel_bytes_per_step": step_bytes,
                        "kernel_bytes_frac_of_peak": round(step_bytes / (ms_per_step * 1e-3) / 1e9 / hbm, 4)},
        "kernels_ms": kernels,
        "tuning": dict(tuning, autotuned=not args.no_autotune),
        "fp64": fp64,
        "split_bf16": split,
        "alu_peaks": {"fp32_tflops": round(fp32_peak / 1e12, 2), "fp64_tflops": round(fp64_peak / 1e12, 3),
                      "source": alu_src},
        "ensemble": ensemble,
        "cufft_yardstick": yardstick,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": kps * args.steps,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def source_hash(sources=None):
    """Hash of the CUDA sources a kernel's counters were taken from (all of
    csrc/ when no list is given): a counter whose sources changed since is
    not reported."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1506_06513_gb300", "csrc")
    for name in sorted(sources or os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def workload_config(n, world, workload="model_insect", wake=False, flight=False, insect="model"):
    """The `config` object of both arms: the workload as the GPU arm runs it."""
    step_bytes = sum(kernel_bytes(n, 4, wake).values())
    if insect == "model":
        parts = ("ellipsoid body (0.5, 0.12) + 2 flapping plates (c 0.3, R 1, 4dx thick, "
                 "phi 60deg sin, alpha 45deg cos)")
    else:
        parts = ("ellipsoid thorax (0.5, 0.12)" + (" bent on a centre-line circle of radius 1"
                                                   if insect == "curved" else "")
                 + " with head and eyes + 2 flapping 16-harmonic contour wings (R 1, 4dx thick, "
                   "phi 60deg sin, alpha 45deg cos)")
    if workload == "turbulent_insect":
        what = (f"model insect {'x'.join(map(str, n))} FP32 in turbulent inflow: {parts}, Re 1000, "
                "u_inf (0.25,0,0), C_eta 5e-4, CFL 0.1 adaptive dt")
        init = ("inflow + seeded isotropic divergence-free field, E(k) ~ k^-5/3 on 2 <= |k| <= 8, "
                "u_rms 0.1 (seed 6513)")
    else:
        what = (f"model insect {'x'.join(map(str, n))} FP32: {parts}, Re 300, u_inf (0.25,0,0), "
                "C_eta 1e-3, CFL 0.1 adaptive dt")
        init = "inflow + band-limited divergence-free waves"
    if wake:
        what += ("; vorticity sponge C_sp 0.1, 32 points deep at the x and y ends, Dirichlet layer "
                 "4 points deep at the x end")
    if flight:
        what += "; free flight (mass 400, J_body (2, 5, 5), g 9.81) with wing power"
    return {"workload": what, "grid": list(n), "box": [4.0, 4.0, 4.0], "precision": "fp32",
            "initial": init,
            "l2": f"inputs larger than L2: {step_bytes / 1e9:.1f} GB moved per step",
            "parallelism": "replicas" if world > 1 else "single GPU"}


# ----------------------------------------------------------- reference arm

def run_reference(args):
    """The oracle as it stands, on the host cores (its OpenMP build, every
    core): each step is one oracle step of the same workload at the largest
    grid of a ladder that keeps the whole run near two minutes."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    host = host_cpu()
    cores = host["nproc"] or 1
    pick, probe = 32, None
    for n in (32, 48, 64, 96, 128, 192, 256):
        probe = oracle_time(args.workload, n, 1, cores, args.flight, args.insect)
        if probe["seconds"] * (args.steps + args.warmup) > 120.0:
            break
        pick = n
    # the timed run: warm-up steps are untimed inside the same process
    r = oracle_time(args.workload, pick, args.steps, cores, args.flight, args.insect)
    value = r["value"]
    el = r["seconds"]
    sample = (f"the same workload at {pick}^3 (same box, body, wings, Re, C_eta, inflow), FP64 C "
              f"oracle on {r['threads']} thread(s) of {host['cpu_model']} ({host['nproc']} logical cores), "
              f"{args.steps} steps in {el:.1f} s; value in grid-point steps/s of that sample")
    cfg = workload_config((pick, pick, pick), world, args.workload, args.wake, args.flight, args.insect)
    cfg["sample_of"] = list(workload_setup(args)[0]["n"])
    cfg["precision"] = "fp64"
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "impl": "reference", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": r["threads"], "kind": "oracle",
                            "sample": sample, "host": host},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.oracle_time:
        oracle_time_main(args.oracle_time)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_flusi(args)


if __name__ == "__main__":
    main()
