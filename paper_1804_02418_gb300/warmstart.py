"""Learned warm start of the relativistic LBM with the spectral neural operator.

    python -m paper_1804_02418_gb300.warmstart [--samples 2000] [--epochs 40] ...

1. Dataset: ensemble-style samples (walled rectangles, two contacts on the
   y = 0 edge, uniform force along x, seeded per sample) are run to steady
   state (per-sample residual <= 1e-6) by the batched FP32 solver and
   resampled onto an N x N canvas.
2. Training: the operator (fno.FNO) learns (mask, drive, tau, x, y) ->
   normalised (n, u_x, u_y, T) with its own forward / backward / Adam kernels.
3. Evaluation: held-out samples are converged from rest (cold) and from the
   operator's prediction (warm, f = f^eq of the predicted fields); steps and
   wall time to residual <= 1e-6 are compared.
4. `--bound K`: on K held-out samples, the steps to residual <= 1e-6 from
   seeds built out of the exact steady fields (as f^eq, partly, with the
   first-order Chapman-Enskog non-equilibrium part), and the late decay rate
   of the residual against the damping of the longest sound mode: what any
   macroscopic seed could gain.

Normalisation (from the linear Stokes response to a uniform force): with
nu = 25 (tau - 1/2) / 4 sites^2 / step and the short side W, velocities are
scaled by F W^2 / nu and density / temperature deviations by F L / 5 (the
pressure gradient balancing the force over the long side L).
"""
from __future__ import annotations

import argparse
import json
import math
import time
from dataclasses import dataclass

import numpy as np

from . import fno, rlbm, workloads as W

TOL = 1e-6


def nu_lattice(tau):
    return 25.0 * (tau - 0.5) / 4.0


def dataset_samples(count, seed0, w_lo=16, w_hi=48, max_aspect=4.0):
    """Ensemble-style samples small enough to converge in a few thousand steps."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        Wd = int(rng.integers(w_lo, w_hi + 1))
        a = float(rng.uniform(1.0, max_aspect))
        L = max(Wd, int(round(a * Wd)))
        tau = float(rng.uniform(0.6, 2.0))
        cw = int(rng.integers(4, max(5, Wd // 3) + 1))
        F = float(10.0 ** rng.uniform(-7.0, -5.0))
        spacing = max(cw + 2 * W.HOP_RADIUS, L // 4)
        spacing = min(spacing, L - cw - 2)
        out.append(W.graphene_sample(nx=L, ny=Wd, contact_width=cw, contact_spacing=spacing,
                                     force=F, tau=tau))
    return out


def scales(s):
    u = s.Fx * s.ny ** 2 / nu_lattice(s.tau)
    d = s.Fx * s.nx / 5.0
    return d, u


def canvas_inputs(s, N):
    """Input channels on the canvas [N, N, 5] and the mask [N, N].  The
    sample (nx x ny) is scaled by N / max(nx, ny) and placed at the origin;
    rows are y, columns x."""
    M = max(s.nx, s.ny)
    wc, hc = max(1, round(N * s.nx / M)), max(1, round(N * s.ny / M))
    x = np.zeros((N, N, 5), dtype=np.float32)
    mask = np.zeros((N, N), dtype=np.float32)
    mask[:hc, :wc] = 1.0
    geo = mask.copy()
    rows = max(1, round(N / M))                      # canvas rows of the contact edge
    for c in s.contacts:
        lo, hi = round(N * c.x0 / M), round(N * (c.x0 + c.length) / M)
        geo[:rows, lo:hi] = 2.0
    x[..., 0] = geo
    x[..., 1] = mask * (math.log10(abs(s.Fx)) + 6.0)
    x[..., 2] = mask * (s.tau - 1.3) / 0.7
    jj, ii = np.meshgrid(np.arange(N), np.arange(N))
    x[..., 3] = jj / N
    x[..., 4] = ii / N
    return x, mask, (hc, wc)


class Resampler:
    """Bilinear resampling between sample grids and the canvas (library kernel)."""

    def __init__(self):
        import torch
        self.torch = torch
        self.lib = fno._lib()

    def __call__(self, planes, dh, dw):
        t = self.torch
        src = planes.contiguous().float()
        nch, sh, sw = src.shape
        dst = t.empty((nch, dh, dw), dtype=t.float32, device=src.device)
        fno._ok(self.lib.rlbm_resample_bilinear(fno._p(src), nch, sh, sw, fno._p(dst), dh, dw,
                                                ctypes_stream(t)), "resample")
        return dst


def ctypes_stream(torch):
    import ctypes
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def converge(samples, prec, init=None, check=100, max_steps=40000, graph_steps=20, ref=None,
             ce=False, history=None):
    """Runs every sample to residual <= TOL; returns (steps per sample, wall seconds,
    final fields per sample, distances).  init: optional list of (n, ux, uy, T)
    host arrays, set as f^eq (rlbm_init) or, with ce, as the Chapman-Enskog
    seed (rlbm_init_ce).  ref: optional reference steady fields; then `distances` holds,
    per check and sample, ||u(t) - u_ref|| / ||u_ref|| (else None).  history:
    optional list that receives the per-sample residuals of every check."""
    import torch
    stream = torch.cuda.Stream()
    dist = [] if ref is not None else None
    with torch.cuda.stream(stream):
        sv = rlbm.Solver(samples, prec=prec, stream=stream, graph_steps=graph_steps)
        for i in range(len(samples)):
            if init is None:
                sv.init(i)
            else:
                f = [np.ascontiguousarray(a, dtype=np.float64) for a in init[i]]
                (sv.init_ce if ce else sv.init)(i, *f)
        sv.autotune()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        done = np.full(len(samples), -1, dtype=np.int64)
        steps = 0
        while steps < max_steps and (done < 0).any():
            sv.step(check, residual=True)
            steps += check
            r = sv.sample_residuals()
            if history is not None:
                history.append(r.copy())
            newly = (done < 0) & (r <= TOL)
            done[newly] = steps
            if ref is not None:
                row = []
                for i in range(len(samples)):
                    _, ux, uy, _ = sv.moments(i)
                    rx, ry = ref[i][1], ref[i][2]
                    row.append(float(np.sqrt(((ux - rx) ** 2 + (uy - ry) ** 2).sum()
                                             / max((rx ** 2 + ry ** 2).sum(), 1e-300))))
                dist.append(row)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        fields = [sv.moments(i) for i in range(len(samples))]
        sv.close()
    done[done < 0] = max_steps
    return done, wall, fields, (np.array(dist) if dist is not None else None)


def steps_to(dist, level, check=100):
    """First check (in steps) at which each sample's distance is <= level."""
    out = np.full(dist.shape[1], dist.shape[0] * check)
    for i in range(dist.shape[1]):
        hit = np.nonzero(dist[:, i] <= level)[0]
        if hit.size:
            out[i] = (hit[0] + 1) * check
    return out


@dataclass
class Data:
    x: np.ndarray        # [S, N, N, 5]
    y: np.ndarray        # [S, N, N, 4] normalised targets
    m: np.ndarray        # [S, N, N]


def build_dataset(samples, fields, N):
    import torch
    rs = Resampler()
    S = len(samples)
    X = np.zeros((S, N, N, 5), np.float32)
    Y = np.zeros((S, N, N, 4), np.float32)
    Mk = np.zeros((S, N, N), np.float32)
    for k, (s, f) in enumerate(zip(samples, fields)):
        x, mask, (hc, wc) = canvas_inputs(s, N)
        d, u = scales(s)
        n, ux, uy, T = f
        planes = torch.tensor(np.stack([(n - 1) / d, ux / u, uy / u, (T - 1) / d]),
                              dtype=torch.float32, device="cuda")
        r = rs(planes, hc, wc).cpu().numpy()
        X[k] = x
        Mk[k] = mask
        Y[k, :hc, :wc] = np.moveaxis(r, 0, -1)
    return Data(X, Y, Mk)


def canvas_to_fields(rs, y, s, N, use=("n", "u", "T"), chan=None):
    """Normalised canvas fields y (tensor [N, N, 4]) -> (n, u_x, u_y, T) host
    arrays on the sample grid [ny][nx].  chan: per-channel standard scales the
    targets were divided by (None: 1).  Fields not in `use` are set to their
    rest values (n = T = 1, u = 0)."""
    M = max(s.nx, s.ny)
    wc, hc = max(1, round(N * s.nx / M)), max(1, round(N * s.ny / M))
    planes = y[:hc, :wc].permute(2, 0, 1).contiguous()
    r = rs(planes, s.ny, s.nx).double().cpu().numpy()
    if chan is not None:
        r = r * np.asarray(chan, dtype=np.float64)[:, None, None]
    d, u = scales(s)
    n = 1.0 + d * r[0]
    T = 1.0 + d * r[3]
    ux, uy = u * r[1], u * r[2]
    sp = np.sqrt(ux * ux + uy * uy)
    lim = 0.3
    fac = np.where(sp > lim, lim / np.maximum(sp, 1e-300), 1.0)
    if "n_anchor" in use:
        # the contacts hold n = 1: shift the predicted density so that the
        # sites beside the contacts sit at the contact value
        vals = [n[0, c.x0:c.x0 + c.length] for c in s.contacts if c.edge == 0]
        if vals:
            n = n - np.concatenate(vals).mean() + 1.0
    elif "n" not in use:
        n = np.ones_like(n)
    if "T" not in use:
        T = np.ones_like(T)
    if "u" not in use:
        ux, uy, fac = np.zeros_like(ux), np.zeros_like(uy), 1.0
    return (np.clip(n, 0.5, 1.5), ux * fac, uy * fac, np.clip(T, 0.5, 1.5))


def predict_fields(net, samples, N, use=("n", "u", "T"), chan=None):
    """Operator prediction -> (n, u_x, u_y, T) on every sample's own grid."""
    import torch
    rs = Resampler()
    out = []
    B = net.B
    for k0 in range(0, len(samples), B):
        chunk = samples[k0:k0 + B]
        X = np.zeros((B, N, N, 5), np.float32)
        for j, s in enumerate(chunk):
            X[j] = canvas_inputs(s, N)[0]
        y = net.forward(torch.tensor(X.reshape(-1, 5), dtype=torch.bfloat16, device="cuda"))
        y = y.view(B, N, N, 4)
        for j, s in enumerate(chunk):
            out.append(canvas_to_fields(rs, y[j], s, N, use, chan))
    return out


def train(data, cfg, epochs, batch, lr=2e-3, seed=0, log=None):
    import torch
    net = fno.FNO(cfg, batch=batch, seed=seed)
    S = data.x.shape[0]
    rng = np.random.default_rng(seed)
    N = cfg.N
    X = torch.tensor(data.x.reshape(S, N * N, 5), dtype=torch.bfloat16, device="cuda")
    Y = torch.tensor(data.y.reshape(S, N * N, 4), dtype=torch.float32, device="cuda")
    Mk = torch.tensor(data.m.reshape(S, N * N), dtype=torch.float32, device="cuda")
    steps_per_epoch = max(1, S // batch)
    total = epochs * steps_per_epoch
    it = 0
    history = []
    t0 = time.perf_counter()
    for ep in range(epochs):
        perm = rng.permutation(S)
        acc = 0.0
        for k in range(steps_per_epoch):
            idx = torch.tensor(perm[k * batch:(k + 1) * batch], device="cuda")
            net.forward(X[idx].reshape(-1, 5))
            loss = net.loss(Y[idx].reshape(-1, 4).contiguous(), Mk[idx].reshape(-1).contiguous())
            net.backward()
            it += 1
            cur = lr * 0.5 * (1.0 + math.cos(math.pi * it / total))     # cosine decay
            net.adam(lr=cur)
            acc += float(loss)
        history.append(acc / steps_per_epoch)
        if log:
            log(f"epoch {ep + 1}/{epochs} loss {history[-1]:.4e} ({time.perf_counter() - t0:.1f} s)")
    torch.cuda.synchronize()
    return net, history, time.perf_counter() - t0


def evaluate(net, data, batch):
    """Masked MSE of the operator on a dataset (normalised units)."""
    import torch
    S = data.x.shape[0]
    N = net.cfg.N
    tot, cnt = 0.0, 0
    for k0 in range(0, S - batch + 1, batch):
        X = torch.tensor(data.x[k0:k0 + batch].reshape(-1, 5), dtype=torch.bfloat16, device="cuda")
        Y = torch.tensor(data.y[k0:k0 + batch].reshape(-1, 4), dtype=torch.float32, device="cuda")
        Mk = torch.tensor(data.m[k0:k0 + batch].reshape(-1), dtype=torch.float32, device="cuda")
        net.forward(X)
        tot += float(net.loss(Y, Mk))
        cnt += 1
    return tot / max(cnt, 1)


# ---------------------------------------------------------------------------
# Residual analytics and the bound on what a macroscopic seed can gain
# ---------------------------------------------------------------------------
def decay_rates(history, check, lo=TOL, hi=100 * TOL):
    """Late-time decay rate lambda (per step) of every sample's residual,
    r(t) ~ C exp(-lambda t), fitted to the checks where lo <= r <= hi (NaN
    when fewer than three)."""
    h = np.array(history)                     # [checks, samples]
    t = check * (np.arange(h.shape[0]) + 1)
    out = np.full(h.shape[1], np.nan)
    for i in range(h.shape[1]):
        sel = (h[:, i] >= lo) & (h[:, i] <= hi)
        if sel.sum() >= 3:
            out[i] = -np.polyfit(t[sel], np.log(h[sel, i]), 1)[0]
    return out


def acoustic_rate(s):
    """Damping rate of the longest sound mode along the sample, nu k^2 / 2 with
    k = pi / L (a standing wave between the short walls; lattice units)."""
    return 0.5 * nu_lattice(s.tau) * (math.pi / s.nx) ** 2


def bound_seeds(samples, prec="f64", check=25, max_steps=40000):
    """Steps to residual <= TOL from the rest state and from seeds built out
    of the exact steady fields (as f^eq, partly, and with the first-order
    Chapman-Enskog part), plus the late decay rate of the residual against
    the damping of the longest sound mode.  Yields one dict per seed."""
    steps0, _, steady, _ = converge(samples, prec, check=check, max_steps=max_steps)
    one = lambda f: np.ones_like(f[0])
    seeds = {
        "rest (n = T = 1, u = 0)": dict(init=None),
        "exact steady n, u, T as f^eq": dict(init=steady),
        "exact steady n, u (T = 1)": dict(init=[(f[0], f[1], f[2], one(f)) for f in steady]),
        "exact steady u (n = T = 1)": dict(init=[(one(f), f[1], f[2], one(f)) for f in steady]),
        "exact fields + first-order Chapman-Enskog part": dict(init=steady, ce=True),
    }
    ac = np.array([acoustic_rate(s) for s in samples])
    for name, kw in seeds.items():
        hist = []
        st, _, _, _ = converge(samples, prec, check=check, max_steps=max_steps, history=hist, **kw)
        lam = decay_rates(hist, check)
        ok = np.isfinite(lam)
        yield {"seed": name, "samples": len(samples), "precision": prec,
               "steps_mean": float(st.mean()), "steps_median": float(np.median(st)),
               "late_decay_rate_median": float(np.median(lam[ok])) if ok.any() else None,
               "decay_rate_over_sound_damping_median": float(np.median(lam[ok] / ac[ok])) if ok.any() else None}


# ---------------------------------------------------------------------------
# Config-5 protocol: config-4-style samples, grouped runs, seeds and routes
# ---------------------------------------------------------------------------

def config4_samples(count, seed0, w_lo=128, w_hi=256):
    """Config-4-style samples (short side W ~ U[w_lo, w_hi], aspect U[1, 4],
    tau U[0.6, 2.0], contact width U{8..64}, |F| logU[1e-7, 1e-5], seed0 + i)."""
    return W.ensemble(count, seed0, w_lo=w_lo, w_hi=w_hi)


def groups_of(samples, size):
    """Index groups of `size` samples with similar expected convergence time
    (ordered by L^2 / nu: the slow mode along the long side sets it)."""
    order = sorted(range(len(samples)), key=lambda i: samples[i].nx ** 2 / nu_lattice(samples[i].tau))
    return [order[k:k + size] for k in range(0, len(order), size)]


def run_group(samples, init=None, ce=False, route="f64", tol=TOL, switch=1e-5, check=100,
              max32=20000, max64=60000, graph_steps=20):
    """Runs one group of samples to residual <= tol.
    route "f64": FP64 from the seed.  route "f32>f64": FP32 from the seed
    until every sample's residual is <= switch (FP32 storage has a rounding
    floor near that level) or max32 steps, then the states move to an FP64
    context (rlbm_get_state / rlbm_set_state on device buffers) that runs to
    tol.  Returns per-sample steps in each precision (the first check at which
    the sample met its criterion; max when never), the group's wall seconds
    (initialisation, steps, residual checks and the state transfer; the
    launch-shape tuning excluded) and the final fields."""
    import torch
    stream = torch.cuda.Stream()
    n = len(samples)
    s32 = np.zeros(n, dtype=np.int64)
    s64 = np.zeros(n, dtype=np.int64)
    tuned = {}

    def tune(sv, prec):
        # launch shape of the step kernel for this group (timed on the seeded
        # state without advancing it; outside the timed region)
        torch.cuda.synchronize()
        a = time.perf_counter()
        sv.autotune()
        torch.cuda.synchronize()
        tuned[prec] = time.perf_counter() - a

    def seed(sv):
        for i in range(n):
            if init is None:
                sv.init(i)
            else:
                f = [np.ascontiguousarray(a, dtype=np.float64) for a in init[i]]
                (sv.init_ce if ce else sv.init)(i, *f)

    def run(sv, limit, target, out):
        done = np.zeros(n, dtype=bool)
        steps = 0
        while steps < limit and not done.all():
            sv.step(check, residual=True)
            steps += check
            r = sv.sample_residuals()
            newly = ~done & (r <= target)
            out[newly] = steps
            done |= newly
        out[~done] = limit
        return steps

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        if route == "f32>f64":
            sv32 = rlbm.Solver(samples, prec="f32", stream=stream, graph_steps=graph_steps)
            seed(sv32)
            tune(sv32, "f32")
            run(sv32, max32, switch, s32)
            states = [sv32.get_state(i, out=torch.empty((rlbm.RLBM_Q, x.ny, x.nx),
                                                           dtype=torch.float64, device="cuda"))
                      for i, x in enumerate(samples)]
            sv32.close()
            sv = rlbm.Solver(samples, prec="f64", stream=stream, graph_steps=graph_steps)
            for i, st in enumerate(states):
                sv.set_state(st, i)
            del states
            tune(sv, "f64")
        else:
            sv = rlbm.Solver(samples, prec="f64", stream=stream, graph_steps=graph_steps)
            seed(sv)
            tune(sv, "f64")
        run(sv, max64, tol, s64)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0 - sum(tuned.values())
        fields = [sv.moments(i) for i in range(n)]
        sv.check()
        sv.close()
    return s32, s64, wall, fields


def converge_grouped(samples, prec, tol, group=48, check=200, max_steps=20000):
    """Steady fields of every sample for the dataset, in groups of similar
    convergence time (one batched context per group).  Returns (steps, wall
    seconds, fields)."""
    steps = np.zeros(len(samples), dtype=np.int64)
    fields = [None] * len(samples)
    wall = 0.0
    global TOL
    saved, TOL = TOL, tol
    try:
        for idx in groups_of(samples, group):
            st, w, f, _ = converge([samples[i] for i in idx], prec, check=check, max_steps=max_steps)
            wall += w
            for k, i in enumerate(idx):
                steps[i], fields[i] = st[k], f[k]
    finally:
        TOL = saved
    return steps, wall, fields


def evaluate_config5(net, held, cfg_N, chan, log, n_eval, max32=20000, max64=40000):
    """Steps and wall time to residual <= 1e-6 of the first `n_eval` held-out
    samples, each run alone (its own context, so that a slow sample holds up
    no other), from rest and from the operator's seed (its n, u as f^eq, and
    the same fields as the Chapman-Enskog seed), in plain FP64 and through the
    FP32-then-FP64 route.  Per arm the JSON line lists every sample's steps
    and seconds; the wall time of a seeded arm includes the operator's
    inference for that sample."""
    import torch
    arms = [("rest", None, False), ("operator n, u as f^eq", "eq", False),
            ("operator n, u + Chapman-Enskog part", "eq", True)]
    pred = predict_fields(net, held[:1], cfg_N, use=("n", "u"), chan=chan)     # warm-up
    per = {}
    for route, subset in (("f64", held[:n_eval]), ("f32>f64", held[:n_eval])):
        for name, kind, ce in arms:
            rec = []
            for s in subset:
                init, seed_s = None, 0.0
                if kind is not None:
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    init = predict_fields(net, [s], cfg_N, use=("n", "u"), chan=chan)
                    torch.cuda.synchronize()
                    seed_s = time.perf_counter() - t0
                s32, s64, w, _ = run_group([s], init=init, ce=ce, route=route,
                                           max32=max32, max64=max64)
                rec.append((int(s32[0]), int(s64[0]), w + seed_s, seed_s, s.sites))
            r = np.array(rec, dtype=np.float64)
            line = {"phase": "evaluation", "route": route, "seed": name, "samples": len(subset),
                    "sites": int(r[:, 4].sum()),
                    "steps_f64_mean": float(r[:, 1].mean()), "steps_f64_median": float(np.median(r[:, 1])),
                    "f64_cap_hits": int((r[:, 1] >= max64).sum()),
                    "seconds_total": float(r[:, 2].sum()), "seconds_mean": float(r[:, 2].mean()),
                    "seconds_median": float(np.median(r[:, 2])),
                    "seconds_seeding_total": float(r[:, 3].sum())}
            if route == "f32>f64":
                line.update(steps_f32_mean=float(r[:, 0].mean()),
                            steps_f32_median=float(np.median(r[:, 0])),
                            f32_cap_hits=int((r[:, 0] >= max32).sum()))
            line["per_sample_steps_f32_f64_seconds"] = [[int(a), int(b), round(float(c), 4)]
                                                        for a, b, c, _, _ in rec]
            per[(route, name)] = r
            log(json.dumps(line))
    # per-sample comparisons against plain FP64 from rest on the FP64 subset
    base = per[("f64", "rest")]
    for key, r in per.items():
        if key == ("f64", "rest"):
            continue
        m = min(len(base), len(r))
        ratio = r[:m, 2] / base[:m, 2]
        log(json.dumps({"phase": "comparison", "route": key[0], "seed": key[1],
                        "against": "plain FP64 from rest", "samples": int(m),
                        "wall_ratio_median": float(np.median(ratio)),
                        "wall_ratio_of_totals": float(r[:m, 2].sum() / base[:m, 2].sum()),
                        "faster_fraction": float((ratio < 1).mean())}))
    return per


def main_config5(args, log):
    cfg = fno.FNOConfig(N=args.canvas, C=args.width, Cq=4 * args.width, L=args.layers,
                        m1=args.modes, m2=args.modes)
    samples = config4_samples(args.samples + args.test, args.seed)
    steps, wall, fields = converge_grouped(samples, "f32", tol=1e-5, group=args.group)
    log(json.dumps({"phase": "dataset", "samples": len(samples),
                    "sites": int(sum(s.sites for s in samples)),
                    "short_side": [min(s.ny for s in samples), max(s.ny for s in samples)],
                    "long_side": [min(s.nx for s in samples), max(s.nx for s in samples)],
                    "criterion": "FP32 per-sample residual <= 1e-5 (cap 20,000 steps)",
                    "steps_mean": float(steps.mean()), "steps_median": float(np.median(steps)),
                    "cap_hits": int((steps >= 20000).sum()), "seconds": wall}))
    data = build_dataset(samples, fields, cfg.N)
    m_tr = data.m[:args.samples, ..., None]
    chan = np.sqrt((data.y[:args.samples] ** 2 * m_tr).sum((0, 1, 2)) / max(m_tr.sum(), 1.0))
    chan = np.where(chan > 0, chan, 1.0).astype(np.float32)
    data.y /= chan
    tr = Data(data.x[:args.samples], data.y[:args.samples], data.m[:args.samples])
    te = Data(data.x[args.samples:], data.y[args.samples:], data.m[args.samples:])
    net, hist, secs = train(tr, cfg, args.epochs, args.batch, log=log)
    log(json.dumps({"phase": "train", "epochs": args.epochs, "seconds": secs,
                    "train_mse": hist[-1], "test_mse": evaluate(net, te, args.batch),
                    "target_var": float((te.y ** 2 * te.m[..., None]).sum() / (4 * te.m.sum()))}))
    held = samples[args.samples:]
    ref = fields[args.samples:]
    pred = predict_fields(net, held, cfg.N, use=("n", "u"), chan=chan)
    err = [float(np.sqrt(((p[1] - r[1]) ** 2 + (p[2] - r[2]) ** 2).sum()
                         / max((r[1] ** 2 + r[2] ** 2).sum(), 1e-300))) for p, r in zip(pred, ref)]
    log(json.dumps({"phase": "prediction", "samples": len(held),
                    "u_rel_l2_error_median": float(np.median(err)),
                    "u_rel_l2_error_p90": float(np.percentile(err, 90))}))
    del data, tr, te
    evaluate_config5(net, held, cfg.N, chan, log, args.eval_samples)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--samples", type=int, default=2000)
    ap.add_argument("--test", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--canvas", type=int, default=256)
    ap.add_argument("--width", type=int, default=32)
    ap.add_argument("--modes", type=int, default=16)
    ap.add_argument("--layers", type=int, default=4)
    ap.add_argument("--seed", type=int, default=20180406)
    ap.add_argument("--eval-samples", type=int, default=64)
    ap.add_argument("--bound", type=int, default=0,
                    help="instead of training: the seed bound on this many held-out samples")
    ap.add_argument("--config5", action="store_true",
                    help="config-4-style samples (short side 128-256), grouped runs, evaluation "
                         "of plain FP64 and of the FP32-then-FP64 route from rest and from the seeds")
    ap.add_argument("--group", type=int, default=48)
    args = ap.parse_args()
    log = lambda m: print(m, flush=True)
    if args.config5:
        return main_config5(args, log)
    if args.bound:
        held = dataset_samples(args.samples + args.bound, args.seed)[args.samples:]
        for line in bound_seeds(held):
            log(json.dumps(line))
        return
    cfg = fno.FNOConfig(N=args.canvas, C=args.width, Cq=4 * args.width, L=args.layers,
                        m1=args.modes, m2=args.modes)
    samples = dataset_samples(args.samples + args.test, args.seed)
    t0 = time.perf_counter()
    steps, wall, fields, _ = converge(samples, "f32")
    log(json.dumps({"phase": "dataset", "samples": len(samples), "sites": int(sum(s.sites for s in samples)),
                    "steps_max": int(steps.max()), "steps_mean": float(steps.mean()),
                    "seconds": time.perf_counter() - t0}))
    data = build_dataset(samples, fields, cfg.N)
    # standardise every target channel over the training set (the physical
    # scales above fix the per-sample dependence on F, tau and size; the
    # channels still differ by orders of magnitude)
    m_tr = data.m[:args.samples, ..., None]
    chan = np.sqrt((data.y[:args.samples] ** 2 * m_tr).sum((0, 1, 2)) / max(m_tr.sum(), 1.0))
    chan = np.where(chan > 0, chan, 1.0).astype(np.float32)
    data.y /= chan
    log(json.dumps({"phase": "normalisation", "channel_scales": chan.tolist()}))
    tr = Data(data.x[:args.samples], data.y[:args.samples], data.m[:args.samples])
    te = Data(data.x[args.samples:], data.y[args.samples:], data.m[args.samples:])
    net, hist, secs = train(tr, cfg, args.epochs, args.batch, log=log)
    log(json.dumps({"phase": "train", "epochs": args.epochs, "seconds": secs,
                    "train_mse": hist[-1], "test_mse": evaluate(net, te, args.batch),
                    "target_var": float((te.y ** 2 * te.m[..., None]).sum() / (4 * te.m.sum()))}))
    held = samples[args.samples:args.samples + args.eval_samples]
    ref = fields[args.samples:args.samples + args.eval_samples]
    cold = {}
    for prec in ("f64", "f32"):
        c_steps, c_wall, _, c_dist = converge(held, prec, ref=ref, max_steps=20000)
        cold[prec] = (c_steps, c_wall, c_dist)
        log(json.dumps({"phase": "cold", "precision": prec, "samples": len(held),
                        "steps_mean": float(c_steps.mean()), "seconds": c_wall}))
    for use in (("u",), ("n", "u"), ("n_anchor", "u")):
        pred = predict_fields(net, held, cfg.N, use=use, chan=chan)
        err = [float(np.sqrt(((p[1] - r[1]) ** 2 + (p[2] - r[2]) ** 2).sum() / max((r[1] ** 2 + r[2] ** 2).sum(), 1e-300)))
               for p, r in zip(pred, ref)]
        for prec in ("f64", "f32"):
            w_steps, w_wall, _, w_dist = converge(held, prec, init=pred, ref=ref, max_steps=20000)
            c_steps, c_wall, c_dist = cold[prec]
            line = {"phase": "warm_start", "fields": "+".join(use), "precision": prec,
                    "samples": len(held), "u_rel_error_initial_median": float(np.median(err)),
                    "cold_steps_mean": float(c_steps.mean()), "warm_steps_mean": float(w_steps.mean()),
                    "step_ratio": float(w_steps.mean() / c_steps.mean()),
                    "cold_seconds": c_wall, "warm_seconds": w_wall,
                    "warm_fewer_steps_fraction": float((w_steps < c_steps).mean())}
            for lvl in (0.3, 0.1, 0.03, 0.01):
                cs, ws_ = steps_to(c_dist, lvl), steps_to(w_dist, lvl)
                line[f"steps_to_u_within_{lvl}"] = {"cold": float(np.median(cs)), "warm": float(np.median(ws_))}
            log(json.dumps(line))


if __name__ == "__main__":
    main()
