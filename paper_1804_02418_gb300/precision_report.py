"""Error of the reduced-precision paths against the FP64 path on one workload.

    python -m paper_1804_02418_gb300.precision_report [--nx 4096 --ny 2048 --steps 10000]

Runs the graphene-like sample (walls, two 32-wide contacts 256 apart on the
y = 0 edge, uniform force 1e-6 along x, tau = 1, from rest) with FP64, FP32,
FP16-deviation and BF16-deviation storage for the same number of steps and
prints one JSON line per precision with the relative L2 and L-infinity errors
of n, u (vector field) and T against the FP64 run:
    L2   = ||x - x64||_2 / ||x64||_2,   Linf = max|x - x64| / max|x64|,
plus the deviation fields' relative errors (n - 1, T - 1), which carry the
physics at these small drives.  The FP64 run itself matches the CPU oracle
to 1e-12 (tests/test_gpu_parity.py).
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


def run(nx, ny, steps, precs):
    import torch

    from . import rlbm, workloads as W
    s = W.graphene_sample(nx=nx, ny=ny)
    out = {}
    for prec in precs:
        with rlbm.Solver(s, prec=prec) as sv:
            sv.init(0)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sv.step(steps)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            n, ux, uy, T = sv.moments()
            sv.check()
        out[prec] = (n, ux, uy, T, dt)
    return s, out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=4096)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--steps", type=int, default=10000)
    args = ap.parse_args()
    precs = ["f64", "f32", "f16dev", "bf16dev"]
    s, out = run(args.nx, args.ny, args.steps, precs)
    n0, ux0, uy0, T0, _ = out["f64"]
    u0 = np.stack([ux0, uy0])
    for prec in precs:
        n, ux, uy, T, dt = out[prec]
        u = np.stack([ux, uy])
        du = np.sqrt(((u - u0) ** 2).sum(0))
        umag = np.sqrt((u0 ** 2).sum(0))
        line = {
            "precision": prec, "nx": args.nx, "ny": args.ny, "steps": args.steps,
            "seconds": dt, "GLUPS": s.sites * args.steps / dt / 1e9,
            "n": errors(n, n0), "T": errors(T, T0),
            "u": {"L2": float(np.linalg.norm(du) / np.linalg.norm(umag)),
                  "Linf": float(du.max() / umag.max())},
            "n_minus_1": errors(n - 1.0, n0 - 1.0), "T_minus_1": errors(T - 1.0, T0 - 1.0),
            "max_u": float(umag.max()),
        }
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
