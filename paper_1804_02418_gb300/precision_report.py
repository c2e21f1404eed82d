"""Error of the reduced-precision paths against the FP64 path on one workload.

    python -m paper_1804_02418_gb300.precision_report [--nx 4096 --ny 2048 --steps 10000]
        [--precs f64,f32,f16dev,bf16dev] [--no-tune]

Runs the graphene-like sample (walls, two 32-wide contacts 256 apart on the
y = 0 edge, uniform force 1e-6 along x, tau = 1, from rest) with FP64, FP32,
FP16-deviation and BF16-deviation storage for the same number of steps and
prints one JSON line per precision with the relative L2 and L-infinity errors
of n, u (vector field) and T against the FP64 run:
    L2   = ||x - x64||_2 / ||x64||_2,   Linf = max|x - x64| / max|x64|,
plus the deviation fields' relative errors (n - 1, T - 1), which carry the
physics at these small drives.  The FP64 run itself matches the CPU oracle
to 1e-12 (tests/test_gpu_parity.py).  Each context first picks its launch
shape with rlbm_autotune (not timed; the state does not advance; --no-tune
keeps the single-sample kernel, one block per tile); the line names the
shape.  Without f64 among the precisions the lines carry the timings only.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def errors(x, r):
    d = x - r
    return {"L2": float(np.linalg.norm(d) / max(np.linalg.norm(r), 1e-300)),
            "Linf": float(np.abs(d).max() / max(np.abs(r).max(), 1e-300))}


def run(nx, ny, steps, precs, tune=True):
    import torch

    from . import rlbm, workloads as W
    s = W.graphene_sample(nx=nx, ny=ny)
    out = {}
    for prec in precs:
        with rlbm.Solver(s, prec=prec) as sv:
            sv.init(0)
            shape = sv.autotune() if tune else (0, 0, 0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sv.step(steps)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            n, ux, uy, T = sv.moments()
            sv.check()
        out[prec] = (n, ux, uy, T, dt, shape)
    return s, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--precs", default="f64,f32,f16dev,bf16dev")
    ap.add_argument("--no-tune", action="store_true")
    args = ap.parse_args()
    precs = args.precs.split(",")
    s, out = run(args.nx, args.ny, args.steps, precs, tune=not args.no_tune)
    for prec in precs:
        n, ux, uy, T, dt, shape = out[prec]
        line = {
            "precision": prec, "nx": args.nx, "ny": args.ny, "steps": args.steps,
            "seconds": dt, "GLUPS": s.sites * args.steps / dt / 1e9,
            "launch_shape": {"sites_per_block": shape[0] or 128, "blocks": shape[1] or "one per tile",
                             "staged": shape[2], "kernel": "single-sample" if shape[0] == 0 else "batched"},
        }
        if "f64" in out:
            n0, ux0, uy0, T0 = out["f64"][:4]
            u0, u = np.stack([ux0, uy0]), np.stack([ux, uy])
            du = np.sqrt(((u - u0) ** 2).sum(0))
            umag = np.sqrt((u0 ** 2).sum(0))
            line.update({
                "n": errors(n, n0), "T": errors(T, T0),
                "u": {"L2": float(np.linalg.norm(du) / np.linalg.norm(umag)),
                      "Linf": float(du.max() / umag.max())},
                "n_minus_1": errors(n - 1.0, n0 - 1.0), "T_minus_1": errors(T - 1.0, T0 - 1.0),
                "max_u": float(umag.max()),
            })
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
