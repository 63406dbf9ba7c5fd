"""cuFFT (through torch.fft) on the transforms of one step, as a yardstick.

    python -m paper_1506_06513_gb300.yardstick [--grid 512]

One step of the method needs six inverse (c2r) and three forward (r2c) 3-D
transforms.  This times exactly those with cuFFT on full half spectra in FP32
(no 2/3-rule pruning, no fusion), batched three fields per call, with CUDA
events after warm-up.  It is a yardstick for the project's own pruned
transforms, which run inside the step's kernels together with the curl, the
mask, the nonlinear term and the update; it is not part of the solver.
Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json


def run(n=512, reps=10):
    import torch
    dev = torch.device("cuda")
    spec = torch.randn((3, n, n, n // 2 + 1), dtype=torch.complex64, device=dev)
    phys = torch.randn((3, n, n, n), dtype=torch.float32, device=dev)
    out_r = torch.empty((3, n, n, n), dtype=torch.float32, device=dev)
    out_c = torch.empty((3, n, n, n // 2 + 1), dtype=torch.complex64, device=dev)

    def one_step():
        # velocity and vorticity back to the grid, the nonlinear term forward
        torch.fft.irfftn(spec, s=(n, n, n), dim=(1, 2, 3), out=out_r)
        torch.fft.irfftn(spec, s=(n, n, n), dim=(1, 2, 3), out=out_r)
        torch.fft.rfftn(phys, dim=(1, 2, 3), out=out_c)

    for _ in range(3):
        one_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        one_step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    bytes_moved = 2 * (3 * n ** 3 * 4 + 3 * n * n * (n // 2 + 1) * 8) * 3   # read + write per call, 3 calls
    return {"what": f"cuFFT via torch.fft: 6 c2r + 3 r2c 3-D transforms of {n}^3 FP32 "
                    "(full half spectra, batched 3 fields per call)",
            "ms": ms, "grid": n, "min_bytes_per_step": bytes_moved}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=512)
    args = ap.parse_args()
    print(json.dumps(run(args.grid)), flush=True)


if __name__ == "__main__":
    main()
