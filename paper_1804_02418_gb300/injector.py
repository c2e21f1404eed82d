"""Potential near a current injector (Sec. 3, Eq. phi-approx-inlet).

In the Stokes regime, the electrochemical potential near a point injector on
a no-slip edge of a half-plane falls off as

    Phi(r, theta) ~ (2 I eta / (pi n^2 e^2)) cos(2 theta) / r^2,

with I the injected current, eta the shear viscosity, n the equilibrium
density, r, theta polar coordinates about the injector (theta from the
edge).  The paper shows that r^2 Phi, normalised to its value at r = 40,
theta = 0, collapses onto one curve at several r.

Reading for this solver: in slow steady flow the force per particle that
the viscous stress balances is -grad(P)/n + F_E = -grad U with
    U = (P - P0) / n0 + (e^2 / C_g) (n - n0)
(pressure P = n T of the massless gas, F_E the local-capacitance force), so
U plays the role of e Phi.  Stokes flow from a source of volume flux
Q = I / n on a no-slip wall (stream function (Q / pi)(theta - sin(2 theta)/2))
has the pressure P = P_inf - (2 eta Q / pi) cos(2 theta) / r^2, hence
    U = -(2 I eta / (pi n^2)) cos(2 theta) / r^2 + const,
the printed law with the pressure's sign (electrons carry -e).  The current
I = sum over a cut of n u_y (per unit length: the length unit of c = 1 is 5
sites), eta = (3/4) n T (tau - 1/2) (viscosity of the lattice), r in sites.

    python -m paper_1804_02418_gb300.injector --tau 0.8
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import rlbm, workloads as W


def geometry(nx=2000, ny=500, width=8, v_in=1e-5, n0=1.5, T0=1.25, tau=0.8, inv_cg=0.1):
    """Injector on the lower edge (centre x = nx/2), collector on the upper
    edge opposite it (u_n is along the inward normal: the collector draws
    the same flux out); the rest of the boundary is a no-slip wall."""
    x0 = nx // 2 - width // 2
    C = W.Contact
    return W.Sample(nx, ny, tau=tau, inv_cg=inv_cg,
                    contacts=[C(0, x0, width, u_n=v_in, n=n0, T=T0),
                              C(1, x0, width, u_n=-v_in, n=n0, T=T0)])


def steady(s, n0, T0, prec="f64", tol=1e-9, max_steps=400000, chunk=2000, log=None):
    """Runs from uniform (n0, u = 0, T0) until the per-step residual <= tol."""
    shape = (s.ny, s.nx)
    with rlbm.Solver(s, prec=prec, graph_steps=100) as sv:
        z = np.zeros(shape)
        sv.init(0, np.full(shape, n0), z, z.copy(), np.full(shape, T0))
        sv.autotune()
        r, t0 = 1.0, time.perf_counter()
        while r > tol and sv.steps_done < max_steps:
            sv.step(chunk)
            r = sv.step(2, residual=True)
            if log:
                log(f"step {sv.steps_done} residual {r:.3e} ({time.perf_counter() - t0:.1f} s)")
        fields = sv.moments(0)
        sv.check()
        return fields, sv.steps_done, r


def bilinear(a, x, y):
    """a[y, x] at fractional (x, y) (clamped to the grid)."""
    x = np.clip(x, 0, a.shape[1] - 1.000001)
    y = np.clip(y, 0, a.shape[0] - 1.000001)
    i, j = np.floor(x).astype(int), np.floor(y).astype(int)
    fx, fy = x - i, y - j
    return ((1 - fx) * (1 - fy) * a[j, i] + fx * (1 - fy) * a[j, i + 1]
            + (1 - fx) * fy * a[j + 1, i] + fx * fy * a[j + 1, i + 1])


def potential(s, fields, n0, T0):
    """U = (n T - n0 T0) / n0 + (e^2 / C_g)(n - n0), and the injected current
    I (flux through the row 40 sites above the injector, per length unit)."""
    n, ux, uy, T = fields
    U = (n * T - n0 * T0) / n0 + s.inv_cg * (n - n0)
    I = float((n[40] * uy[40]).sum()) / 5.0
    return U, I


def hop_average(a, h=5):
    """Mean over h x h boxes centred on every site (edge rows / columns use
    the part of the box inside the grid): removes structure finer than a hop,
    which the lattice does not resolve."""
    k = h // 2
    c = np.cumsum(np.cumsum(np.pad(a, ((1, 0), (1, 0))), 0), 1)
    ny, nx = a.shape
    y0 = np.clip(np.arange(ny) - k, 0, ny); y1 = np.clip(np.arange(ny) + k + 1, 0, ny)
    x0 = np.clip(np.arange(nx) - k, 0, nx); x1 = np.clip(np.arange(nx) + k + 1, 0, nx)
    tot = c[y1][:, x1] - c[y0][:, x1] - c[y1][:, x0] + c[y0][:, x0]
    cnt = (y1 - y0)[:, None] * (x1 - x0)[None, :]
    return tot / cnt


def analyse(s, U, I, n0, T0, radii=(20, 40, 60, 80), thetas=None, y_src=-0.5, smooth=True):
    """U on circles of radius r (sites) about the injector, fitted per circle
    as A(r) cos(2 theta) + B(r) (B: the potential of the far field, not part
    of the law).  Returns the angles, U per radius, the fits (A, B, rms
    misfit), eta and the predicted r^2 A = -2 I eta / (pi n0^2) (r in the
    length unit of c = 1, 5 sites)."""
    if smooth:
        U = hop_average(U)
    if thetas is None:
        thetas = np.linspace(0.12 * np.pi, 0.88 * np.pi, 39)
    xc = s.contacts[0].x0 + s.contacts[0].length / 2.0 - 0.5
    eta = 0.75 * n0 * T0 * (s.tau - 0.5)
    pred = -2.0 * I * eta / (np.pi * n0 ** 2)
    M = np.stack([np.cos(2 * thetas), np.ones_like(thetas)], axis=1)
    prof, fits = {}, {}
    for r in radii:
        u = bilinear(U, xc + r * np.cos(thetas), y_src + r * np.sin(thetas))
        (A, B), *_ = np.linalg.lstsq(M, u, rcond=None)
        rms = float(np.sqrt(np.mean((M @ np.array([A, B]) - u) ** 2)) / abs(A))
        prof[r], fits[r] = u, (float(A), float(B), rms)
    return thetas, prof, fits, eta, pred


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--tau", type=float, default=0.8)
    ap.add_argument("--nx", type=int, default=2000)
    ap.add_argument("--ny", type=int, default=500)
    ap.add_argument("--width", type=int, default=8)
    ap.add_argument("--v-in", type=float, default=1e-5)
    ap.add_argument("--cg", type=float, default=10.0, help="C_g (0: infinite)")
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--prec", default="f64")
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--save", default=None, help="write U and I to this .npz file")
    args = ap.parse_args()
    n0, T0 = 1.5, 1.25
    s = geometry(args.nx, args.ny, args.width, args.v_in, n0, T0, args.tau,
                 0.0 if args.cg == 0 else 1.0 / args.cg)
    log = lambda m: print(m, flush=True)
    t0 = time.perf_counter()
    fields, steps, r = steady(s, n0, T0, args.prec, args.tol, max_steps=args.max_steps,
                              chunk=10000)
    U, I = potential(s, fields, n0, T0)
    if args.save:
        np.savez(args.save, U=U - U.mean(), I=I, steps=steps, res=r)
    th, prof, fits, eta, pred = analyse(s, U, I, n0, T0, radii=(20, 40, 60, 80, 120))
    res = {"tau": args.tau, "C_g": args.cg, "steps": steps, "residual": r,
           "seconds": time.perf_counter() - t0, "current": I, "eta": eta,
           "predicted_r2A": pred,
           "r2A_over_prediction": {str(k): (k / 5.0) ** 2 * f[0] / pred for k, f in fits.items()},
           "fit_rms_over_A": {str(k): f[2] for k, f in fits.items()},
           "r2U_minus_B_over_r40_A": {str(k): ((k / 40.0) ** 2 * (prof[k] - fits[k][1]) / fits[40][0]).round(4).tolist() for k in fits},
           "theta_over_pi": (th / np.pi).round(4).tolist()}
    log(json.dumps(res))


if __name__ == "__main__":
    main()
