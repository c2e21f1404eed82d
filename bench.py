"""Benchmark of the fused relativistic LBM step (GLUPS and fraction of HBM peak).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec f32|f64|f16dev|bf16dev]
                    [--impl ours|reference] [--no-cpu-baseline]
                    [--workload graphene|ensemble|massive]

Workload: the graphene-like sample, 1024 x 512 sites, no-slip walls, injector
and collector contacts 32 sites wide on the y = 0 edge with centres 256 apart,
uniform body force 1e-6 along the edge, tau = 1, started from n = T = 1,
u = 0 (synthetic; the paper has no dataset).  One bench step is one time step
of the whole domain: pull-streaming with walls and contacts, moments, Landau
solve, equilibrium, forcing and relaxation, all in one kernel launch.

L2: the working set of one step (read 48 planes, write 48 planes) is larger
than L2 only in FP64, so a buffer larger than L2 is written before every
timed step and each step is timed alone with CUDA events on the library's
stream; `value` sums those device times.

e2e: the same metric through the C ABI with pinned host buffers: upload of
the initial fields, the K steps and the read-back of (n, u_x, u_y, T), all
inside the timed region.

N > 1 (torchrun): the sample is one coupled domain, so every rank runs an
independent replica ("replicas only"); value = total site updates / max time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
WORKLOAD = ("graphene sample 1024x512, walls, 2 contacts 32 wide 256 apart on y=0, "
            "F=1e-6 along x, tau=1, from rest")
METRIC = "GLUPS and % HBM peak"
L2_BYTES = 135_528_448
FALLBACK_HBM = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--prec", default="f32", choices=sorted(BYTES))
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=12)
    ap.add_argument("--tune-cache", default=None,
                    help="file where the launch-shape autotuner keeps its choice (a later run "
                         "with the same file reuses it instead of timing the candidates)")
    ap.add_argument("--workload", default="graphene", choices=["graphene", "ensemble", "massive"],
                    help="graphene: the 1024x512 sample (default line); ensemble: the "
                         "256-sample uneven ensemble, sharded by sample over the ranks; "
                         "massive: the m = 5 T0 variant on its 45-vector stencil, 1024x512 channel")
    ap.add_argument("--ensemble-size", type=int, default=256)
    ap.add_argument("--force", type=float, default=1e-6,
                    help="massive workload: the uniform force along x (0: none)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", FALLBACK_HBM)), "measured"
    return FALLBACK_HBM, "fallback"


# the sources each profiled step kernel is compiled from
KERNEL_SOURCES = {
    "f64": ["kernels.cuh", "site.cuh", "prec_impl.cuh", "ops.h", "kernels_f64.cu"],
    "f32": ["kernels.cuh", "site.cuh", "prec_impl.cuh", "ops.h", "kernels_f32.cu"],
    "f16dev": ["kernels.cuh", "site.cuh", "prec_impl.cuh", "ops.h", "kernels_f16.cu"],
    "bf16dev": ["kernels.cuh", "site.cuh", "prec_impl.cuh", "ops.h", "kernels_bf16.cu"],
    "massive_f32": ["massive.cu", "massive_tables.h", "massive_quadrature.cpp", "dd.h"],
    "massive_f64": ["massive.cu", "massive_tables.h", "massive_quadrature.cpp", "dd.h"],
}


def source_hash(key="f32"):
    """Hash of the sources the step kernel of `key` is built from."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1804_02418_gb300", "csrc")
    for fn in sorted(KERNEL_SOURCES[key]):
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_traffic(prec):
    """DRAM bytes per launch of the step kernel from the committed ncu summary
    (key: the precision, or "massive_<precision>"), or None when the kernel
    sources changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    e = d.get(prec)
    if not e or prec not in KERNEL_SOURCES or e.get("source_hash") != source_hash(prec):
        return None
    return e.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# CPU oracle legs (the reference arm and the cpu_baseline of our line)
# ---------------------------------------------------------------------------

ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
from oracle import lbm
from paper_1804_02418_gb300 import workloads as W
nx, ny, steps, warm = {nx}, {ny}, {steps}, {warm}
s = W.graphene_sample() if (nx, ny) == (1024, 512) else W.graphene_sample(
    nx=nx, ny=ny, contact_width=max(2, 32 * nx // 1024), contact_spacing=max(4, 256 * nx // 1024))
lat = lbm.Lattice(s)
post = lbm.init(lat, *W.rest_fields(s))
for _ in range(warm):
    post = lbm.step(lat, post)
times = []
for _ in range(steps):
    t0 = time.perf_counter()
    post = lbm.step(lat, post)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(sites=nx * ny, times=times)))
"""


def run_oracle(nx, ny, steps, warm):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, nx=nx, ny=ny, steps=steps, warm=warm)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_oracle_copies(nx, ny, steps, copies):
    """`copies` single-threaded oracle processes on the same workload at the
    same time (one per host core): the oracle's throughput on the whole host."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = ORACLE_SNIPPET.format(root=ROOT, nx=nx, ny=ny, steps=steps, warm=0)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for _ in range(copies)]
    out = []
    for p in procs:
        o, e = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(e[-2000:])
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out


def host_copies():
    """Oracle copies the host can run at once: one per core, at most one per
    ~7 GB of physical memory (a copy of the 1024x512 workload peaks at 3.5 GB)."""
    cores = os.cpu_count() or 1
    try:
        mem = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        mem = 8 << 30
    return max(1, min(cores, int(mem // (7 << 30))))


def cpu_baseline(steps):
    d = run_oracle(1024, 512, steps, 0)
    t1 = sum(d["times"])
    one = d["sites"] * len(d["times"]) / t1 / 1e9
    copies = host_copies()
    msteps = max(2, steps // 2)
    runs = run_oracle_copies(1024, 512, msteps, copies)
    tm = max(sum(r["times"]) for r in runs)
    many = copies * d["sites"] * msteps / tm / 1e9
    return {"value": many, "unit": "GLUPS", "cores": copies, "kind": "oracle",
            "value_1core": one,
            "sample": f"{copies} concurrent single-threaded copies x {msteps} full steps of the "
                      f"1024x512 workload (FP64 numpy; slowest copy {tm:.1f} s); 1 core alone: "
                      f"{len(d['times'])} steps in {t1:.1f} s"}


MASSIVE_WORKLOAD = ("massive-particle fluid m = 5 T0 (45-vector stencil), channel 1024x512, "
                    "periodic along x, walls at y = 0 and y = ny - 1, F = 1e-6 along x, tau = 1, "
                    "from rest")

MASSIVE_ORACLE_SNIPPET = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, {root!r})
from oracle import massive as M
nx, ny, steps, warm = {nx}, {ny}, {steps}, {warm}
M.quadrature(); M.polynomials(); M._rest_projection_and_nodes()
lat = M.Lattice(nx, ny, True, False, 1.0, 1e-6, 0.0)
o = np.ones((ny, nx))
post = M.init(lat, o, 0 * o, 0 * o, o)
for _ in range(warm):
    post = M.step(lat, post)
times = []
for _ in range(steps):
    t0 = time.perf_counter()
    post = M.step(lat, post)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(sites=nx * ny, times=times)))
"""


def run_massive_oracle(nx, ny, steps, warm, copies=1):
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    code = MASSIVE_ORACLE_SNIPPET.format(root=ROOT, nx=nx, ny=ny, steps=steps, warm=warm)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True, env=env) for _ in range(copies)]
    out = []
    for p in procs:
        o, e = p.communicate()
        if p.returncode != 0:
            raise RuntimeError(e[-2000:])
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out


def massive_cpu_baseline(steps, nx=256, ny=128):
    """The massive-particle oracle on a bounded sample of the same geometry
    (256x128; one copy per host core, memory permitting, and one copy alone)."""
    one = run_massive_oracle(nx, ny, steps, 1)[0]
    t1 = sum(one["times"])
    copies = host_copies()
    runs = run_massive_oracle(nx, ny, max(2, steps // 2), 1, copies)
    tm = max(sum(r["times"]) for r in runs)
    many = copies * one["sites"] * len(runs[0]["times"]) / tm / 1e9
    return {"value": many, "unit": "GLUPS", "cores": copies, "kind": "oracle",
            "value_1core": one["sites"] * len(one["times"]) / t1 / 1e9,
            "sample": f"{copies} concurrent single-threaded copies x {len(runs[0]['times'])} steps "
                      f"of the same channel scaled to {nx}x{ny} (FP64 numpy, extended-precision "
                      f"moments; slowest copy {tm:.1f} s); 1 core alone: {len(one['times'])} steps "
                      f"in {t1:.1f} s"}


def massive_reference_arm(args):
    copies = host_copies()
    nx, ny = 128, 64
    runs = run_massive_oracle(nx, ny, args.steps, args.warmup, copies)
    t = max(sum(r["times"]) for r in runs)
    value = copies * runs[0]["sites"] * args.steps / t / 1e9
    sample = (f"{copies} concurrent single-threaded copies x {args.steps} oracle steps of the "
              f"same channel scaled to {nx}x{ny} (bounded so the run ends within minutes), FP64 numpy")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": MASSIVE_WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": copies, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def reference_arm(args):
    if args.workload == "massive":
        return massive_reference_arm(args)
    ladder = [(1024, 512), (512, 256), (256, 128), (128, 64), (64, 32), (32, 16)]
    budget = 150.0
    chosen = ladder[-1]
    for nx, ny in ladder:
        probe = run_oracle(nx, ny, 1, 0)
        if probe["times"][0] * (args.steps + args.warmup) <= budget:
            chosen = (nx, ny)
            break
    # one single-threaded copy per host core (memory permitting), run at once:
    # the oracle's throughput on the whole host; warm-up steps are not timed
    copies = host_copies()
    runs = run_oracle_copies(chosen[0], chosen[1], args.steps + args.warmup, copies)
    t = max(sum(r["times"][args.warmup:]) for r in runs)
    value = copies * runs[0]["sites"] * args.steps / t / 1e9
    sample = (f"{copies} concurrent single-threaded copies x {args.steps} oracle steps of the "
              f"same geometry scaled to {chosen[0]}x{chosen[1]} (bounded so the run ends within "
              f"minutes), FP64 numpy")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "sample": sample},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": copies, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------

class Clocks:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def gpu_arm(args, rank, world, cpu_line):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1804_02418_gb300 import build, parallel, rlbm, workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    s = W.graphene_sample()
    sites = s.sites
    stream = torch.cuda.Stream()
    sv = rlbm.Solver(s, prec=args.prec, stream=stream, tune_cache=args.tune_cache)
    # L2 flush before every timed step: write one buffer larger than L2, then
    # read another one, so that the dirty lines the write leaves are written
    # back before the step starts (the step neither finds its inputs in L2 nor
    # pays for the flush buffer's write-backs)
    flush = torch.empty(max(2 * L2_BYTES, 256 << 20), dtype=torch.uint8, device="cuda")
    evict = torch.ones(max(2 * L2_BYTES, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    sink = torch.empty((), dtype=torch.float32, device="cuda")

    def flush_l2():
        flush.zero_()
        torch.sum(evict, dim=0, out=sink)
    with torch.cuda.stream(stream):
        sv.init(0)
    shape = sv.autotune()

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    # -- device-timed region: K single steps, L2 flushed before each ----------
    with torch.cuda.stream(stream):
        sv.init(0)
        for _ in range(args.warmup):
            flush_l2()
            sv.step(1)
    sync_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    l0 = sv.launches
    sync_all()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush_l2()
            ev[k][0].record(stream)
            sv.step(1)
            ev[k][1].record(stream)
    sync_all()
    launches = sv.launches - l0
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    sv.check()
    t_ms = parallel.max_over_ranks(t_ms, device="cuda")

    # -- end to end through the C ABI with pinned host buffers ----------------
    host_in = [torch.ones((s.ny, s.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    host_in[1].zero_()
    host_in[2].zero_()
    host_out = [torch.empty((s.ny, s.nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    sync_all()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sv.init(0, *host_in)
    sv.step(args.steps)
    sv.moments(0, out=host_out)
    e1.record(stream)
    sync_all()
    e2e_ms = parallel.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    finite = bool(np.isfinite(host_out[1].numpy()).all())
    sv.close()

    if rank != 0:
        return
    hbm, hbm_kind = peaks()
    alg_bytes = 2 * 48 * BYTES[args.prec] * sites
    avg_launch_s = t_ms / 1e3 / args.steps
    achieved = alg_bytes / avg_launch_s / 1e9
    value = world * sites * args.steps / (t_ms / 1e3) / 1e9
    field_bytes = 4 * 8 * sites
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16dev": "f16 storage / f32 compute",
                  "bf16dev": "bf16 storage / f32 compute"}[args.prec],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.prec, "sites": sites,
                   "launch_shape": {"sites_per_block": shape[0] or 128,
                                    "blocks": shape[1] or "one per tile",
                                    "kernel": "single-sample" if shape[0] == 0 else
                                              ("batched, staged pulls" if shape[2] else "batched")},
                   "l2": "before every timed step a 2x L2 buffer is written, then another 2x L2 buffer read (cold L2, no pending write-backs); steps timed alone",
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": ncu_traffic(args.prec),
                     "peak_kind": hbm_kind,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "e2e": {"value": world * sites * args.steps / (e2e_ms / 1e3) / 1e9, "unit": "GLUPS",
                "h2d_bytes_per_step": field_bytes / args.steps,
                "d2h_bytes_per_step": field_bytes / args.steps},
        "gpu_launches": launches,
        "clocks": clk,
        "fields_finite": finite,
    }
    if cpu_line is not None:
        line["cpu_baseline"] = cpu_line
    print(json.dumps(line), flush=True)


def massive_arm(args, rank, world, cpu_line):
    """The massive-particle variant (m = 5 T0) on the 1024x512 channel: same
    timing rules as the default line (L2 flushed before every timed step,
    steps timed alone; e2e through the C ABI with pinned host fields)."""
    import numpy as np
    import torch

    from paper_1804_02418_gb300 import build, massive, parallel

    if args.prec not in ("f32", "f64"):
        raise SystemExit("the massive variant stores f32 or f64")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    nx, ny = 1024, 512
    sites = nx * ny
    stream = torch.cuda.Stream()
    sv = massive.MassiveSolver(nx, ny, True, False, 1.0, args.force, 0.0, prec=args.prec, stream=stream)
    flush = torch.empty(max(2 * L2_BYTES, 256 << 20), dtype=torch.uint8, device="cuda")
    evict = torch.ones(max(2 * L2_BYTES, 256 << 20) // 4, dtype=torch.float32, device="cuda")
    sink = torch.empty((), dtype=torch.float32, device="cuda")

    def flush_l2():
        flush.zero_()
        torch.sum(evict, dim=0, out=sink)

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    with torch.cuda.stream(stream):
        sv.init()
        for _ in range(args.warmup):
            flush_l2()
            sv.step(1)
    sync_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    l0 = sv.launches
    sync_all()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush_l2()
            ev[k][0].record(stream)
            sv.step(1)
            ev[k][1].record(stream)
    sync_all()
    launches = sv.launches - l0
    clk = clocks.stop()
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    sv.check()
    t_ms = parallel.max_over_ranks(t_ms, device="cuda")

    host_in = [torch.ones((ny, nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    host_in[1].zero_()
    host_in[2].zero_()
    host_out = [torch.empty((ny, nx), dtype=torch.float64).pin_memory() for _ in range(4)]
    sync_all()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sv.init(*[h.numpy() for h in host_in])
    sv.step(args.steps)
    sv.moments(out=[h.numpy() for h in host_out])
    e1.record(stream)
    sync_all()
    e2e_ms = parallel.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    finite = bool(np.isfinite(host_out[1].numpy()).all())
    sv.check()
    sv.close()
    if rank != 0:
        return
    hbm, hbm_kind = peaks()
    alg_bytes = 2 * 45 * BYTES[args.prec] * sites
    achieved = alg_bytes / (t_ms / 1e3 / args.steps) / 1e9
    field_bytes = 4 * 8 * sites
    line = {
        "metric": METRIC, "value": world * sites * args.steps / (t_ms / 1e3) / 1e9, "unit": "GLUPS",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
        "config": {"workload": MASSIVE_WORKLOAD if args.force == 1e-6 else
                   MASSIVE_WORKLOAD.replace("F = 1e-6", f"F = {args.force:g}"),
                   "precision": args.prec, "sites": sites,
                   "l2": "before every timed step a 2x L2 buffer is written, then another 2x L2 "
                         "buffer read (cold L2, no pending write-backs); steps timed alone",
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": ncu_traffic("massive_" + args.prec),
                     "peak_kind": hbm_kind, "algorithmic_bytes_per_launch": alg_bytes},
        "e2e": {"value": world * sites * args.steps / (e2e_ms / 1e3) / 1e9, "unit": "GLUPS",
                "h2d_bytes_per_step": field_bytes / args.steps,
                "d2h_bytes_per_step": field_bytes / args.steps},
        "gpu_launches": launches, "clocks": clk, "fields_finite": finite,
    }
    if cpu_line is not None:
        line["cpu_baseline"] = cpu_line
    print(json.dumps(line), flush=True)


def ensemble_arm(args, rank, world):
    """The uneven ensemble, sharded by sample over the ranks (no data-path
    collective).  Its working set is far larger than L2, so steps run back to
    back inside CUDA-graph replays; e2e adds the per-sample residual read-back."""
    import torch
    import torch.distributed as dist

    from paper_1804_02418_gb300 import build, parallel, rlbm, workloads as W

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    samples = W.ensemble(args.ensemble_size)
    mine = parallel.shard_samples([x.sites for x in samples], rank, world)
    shard = [samples[i] for i in mine]
    sites = sum(x.sites for x in shard)
    stream = torch.cuda.Stream()
    sv = rlbm.Solver(shard, prec=args.prec, stream=stream, graph_steps=10,
                     tune_cache=args.tune_cache)
    with torch.cuda.stream(stream):
        for i in range(len(shard)):
            sv.init(i)
    shape = sv.autotune()

    def sync_all():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()

    with torch.cuda.stream(stream):
        sv.step(args.warmup)
    sync_all()
    clocks = Clocks(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sv.launches
    sync_all()
    e0.record(stream)
    sv.step(args.steps)
    e1.record(stream)
    sync_all()
    launches = sv.launches - l0
    clk = clocks.stop()
    t_s = e0.elapsed_time(e1) / 1e3
    sv.check()
    value = parallel.job_throughput(sites * args.steps, t_s, device="cuda") / 1e9
    t_max = parallel.max_over_ranks(t_s, device="cuda")
    # e2e: the same steps plus the per-sample residual read back to the host
    sync_all()
    w0 = time.perf_counter()
    sv.step(args.steps, residual=True)
    res = sv.sample_residuals()
    w1 = time.perf_counter()
    e2e = parallel.job_throughput(sites * args.steps, w1 - w0, device="cuda") / 1e9
    sv.close()
    if rank != 0:
        return
    hbm, hbm_kind = peaks()
    total_sites = sum(x.sites for x in samples)
    alg_bytes = 2 * 48 * BYTES[args.prec] * sites
    achieved = alg_bytes / t_s * args.steps / 1e9
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16dev": "f16 storage / f32 compute",
                  "bf16dev": "bf16 storage / f32 compute"}[args.prec],
        "data": "synthetic",
        "config": {"workload": f"ensemble of {args.ensemble_size} uneven samples (seed 1234 + i), "
                               f"{total_sites} sites, sharded by sample",
                   "precision": args.prec, "sites_rank0": sites,
                   "launch_shape": {"sites_per_block": shape[0] or 128, "blocks": shape[1] or "one per tile",
                                    "staged_pulls": bool(shape[2])},
                   "l2": "working set far larger than L2; steps back to back (CUDA graphs of 10)",
                   "parallelism": f"sample sharding over {world} rank(s)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": None, "peak_kind": hbm_kind,
                     "algorithmic_bytes_per_launch": alg_bytes},
        "e2e": {"value": e2e, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": (16 * len(shard) + 4) / args.steps},
        "gpu_launches": launches, "clocks": clk,
        "residual_max": float(max(res)),
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank == 0:
            reference_arm(args)
        return
    # the CPU oracle runs before any CUDA call of this process
    cpu_line = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "graphene":
        cpu_line = cpu_baseline(args.cpu_sample_steps)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.workload == "massive":
        cpu_line = massive_cpu_baseline(args.cpu_sample_steps)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        dist.init_process_group("nccl")
    try:
        if args.workload == "ensemble":
            ensemble_arm(args, rank, world)
        elif args.workload == "massive":
            massive_arm(args, rank, world, cpu_line)
        else:
            gpu_arm(args, rank, world, cpu_line)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
