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
stream; `value` sums those device times.  `back_to_back` times the same K steps
in one event pair without flushes (each step's write-backs inside the timed
region).

Clocks: NVML is read every ~2 ms by a background thread from before the
warm-up to after the e2e leg; the line reports the median SM clock inside the
timed region and refuses to print without any sample.

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
    "massive_f32_force0": ["massive.cu", "massive_tables.h", "massive_quadrature.cpp", "dd.h"],
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
    (key: the precision, "massive_<precision>", or "massive_f32_force0" for the
    massive kernel without the force), or None when the kernel
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


def ncu_fp64_per_site():
    """FP64-pipe thread instructions per site update of the FP64 step kernel
    from the committed ncu capture, or None when its sources changed since."""
    p = os.path.join(ROOT, "profiles", "step_kernel_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        e = json.load(f).get("f64")
    if not e or e.get("source_hash") != source_hash("f64"):
        return None
    return e.get("fp64_instructions_per_site")


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
    """SM clock and throttle reasons sampled DURING the run by a background
    thread: NVML through ctypes every ~2 ms (nvidia-smi every 50 ms if NVML
    cannot be loaded), from before the warm-up to after the e2e leg.
    `mark(name)` stamps the host time; `stop()` reports the median SM clock of
    the samples taken inside the device-timed window (marks "timed0" ..
    "timed1", host stamps around the enqueue and the closing synchronize),
    and of all samples.  Reading clocks changes no GPU setting."""
    # NVML clocks-event-reason bits (nvml.h)
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown",
               0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown"}

    def __init__(self, index):
        import threading
        self.index = index
        self.samples = []          # (t, sm_mhz, max_mhz, reasons bitmask)
        self.marks = {}
        self._stop = threading.Event()
        self._thread = None
        self.source = None

    def _nvml(self):
        import ctypes
        for name in ("libnvidia-ml.so.1", "libnvidia-ml.so"):
            try:
                lib = ctypes.CDLL(name)
                break
            except OSError:
                lib = None
        if lib is None or lib.nvmlInit_v2() != 0:
            return None
        h = ctypes.c_void_p()
        idx = self.index
        try:
            import torch
            idx = torch.cuda._get_nvml_device_index(self.index)
        except Exception:
            pass
        if lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(idx), ctypes.byref(h)) != 0:
            return None
        reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")

        def read():
            mhz, mx, rs = ctypes.c_uint(), ctypes.c_uint(), ctypes.c_ulonglong()
            if lib.nvmlDeviceGetClockInfo(h, 1, ctypes.byref(mhz)) != 0:   # NVML_CLOCK_SM
                return None
            lib.nvmlDeviceGetMaxClockInfo(h, 1, ctypes.byref(mx))
            reasons_fn(h, ctypes.byref(rs))
            return float(mhz.value), float(mx.value), int(rs.value)
        return read

    def _run_nvml(self, read):
        while not self._stop.is_set():
            r = read()
            if r is not None:
                self.samples.append((time.perf_counter(),) + r)
            self._stop.wait(0.002)

    def _run_smi(self):
        q = ("clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        bits = [0x8, 0x40, 0x20, 0x4]
        try:
            p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                  "--format=csv,noheader,nounits", "-lms", "50"],
                                 stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            return
        self._smi = p
        for line in p.stdout:
            parts = [x.strip() for x in line.split(",")]
            try:
                mask = sum(b for b, v in zip(bits, parts[2:6]) if v.lower() == "active")
                self.samples.append((time.perf_counter(), float(parts[0]), float(parts[1]), mask))
            except (ValueError, IndexError):
                continue
            if self._stop.is_set():
                break

    def start(self):
        import threading
        read = None
        try:
            read = self._nvml()
        except Exception:
            read = None
        if read is not None:
            self.source = "nvml, ~2 ms"
            self._thread = threading.Thread(target=self._run_nvml, args=(read,), daemon=True)
        else:
            self.source = "nvidia-smi, 50 ms"
            self._thread = threading.Thread(target=self._run_smi, daemon=True)
        self._thread.start()
        time.sleep(0.05)

    def mark(self, name):
        self.marks[name] = time.perf_counter()

    def stop(self):
        time.sleep(0.02)
        self._stop.set()
        p = getattr(self, "_smi", None)
        if p is not None:
            p.terminate()
        if self._thread is not None:
            self._thread.join(timeout=5)
        t0, t1 = self.marks.get("timed0"), self.marks.get("timed1")
        timed = [x for x in self.samples if t0 is not None and t1 is not None and t0 <= x[0] <= t1]
        use = timed if timed else self.samples
        if not use:
            raise SystemExit("bench: no clock sample was taken (NVML and nvidia-smi unavailable); "
                             "refusing to print a line without a clock record")
        sm = sorted(x[1] for x in use)
        every = sorted(x[1] for x in self.samples)
        reasons = sorted({nm for x in use for b, nm in self.REASONS.items() if x[3] & b})
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(x[2] for x in use),
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(timed),
                "samples_whole_run": len(self.samples),
                "sm_mhz_whole_run_median": every[len(every) // 2],
                "sm_mhz_whole_run_min": every[0], "source": self.source,
                "window": "device-timed region" if timed else
                          "whole GPU phase (warm-up .. e2e): no sample fell inside the timed region"}


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

    # clocks are sampled from before the warm-up to the end of the e2e leg
    clocks = Clocks(local)
    clocks.start()
    # -- device-timed region: K single steps, L2 flushed before each ----------
    with torch.cuda.stream(stream):
        sv.init(0)
        for _ in range(args.warmup):
            flush_l2()
            sv.step(1)
    sync_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = sv.launches
    sync_all()
    clocks.mark("timed0")
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush_l2()
            ev[k][0].record(stream)
            sv.step(1)
            ev[k][1].record(stream)
    sync_all()
    clocks.mark("timed1")
    launches = sv.launches - l0
    t_ms = sum(a.elapsed_time(b) for a, b in ev)
    sv.check()
    t_ms = parallel.max_over_ranks(t_ms, device="cuda")

    # -- the same K steps back to back in one event pair, no flush: every
    # step's write-backs fall inside the timed region -------------------------
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sync_all()
    b0.record(stream)
    sv.step(args.steps)
    b1.record(stream)
    sync_all()
    b2b_ms = parallel.max_over_ranks(b0.elapsed_time(b1), device="cuda")
    sv.check()

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
    clk = clocks.stop()
    fma_peak = rlbm.fma_peak(True) if args.prec == "f64" else None
    sv.close()

    if rank != 0:
        return
    hbm, hbm_kind = peaks()
    alg_bytes = 2 * 48 * BYTES[args.prec] * sites
    avg_launch_s = t_ms / 1e3 / args.steps
    achieved = alg_bytes / avg_launch_s / 1e9
    value = world * sites * args.steps / (t_ms / 1e3) / 1e9
    field_bytes = 4 * 8 * sites
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": ncu_traffic(args.prec), "peak_kind": hbm_kind,
            "algorithmic_bytes_per_launch": alg_bytes}
    if args.prec == "f64":
        # FP64 arithmetic, not HBM, bounds this path: FP64-pipe instructions per
        # site (committed ncu count) x sites / launch time against the FP64 FMA
        # rate the library's probe measures on this GPU now
        per_site = ncu_fp64_per_site()
        ach = per_site * sites / avg_launch_s / 1e9 if per_site else None
        roof = {"bound": "alu", "achieved": ach, "peak": fma_peak / 1e9,
                "unit": "G FP64 instructions/s", "frac": ach / (fma_peak / 1e9) if ach else None,
                "traffic": ncu_traffic(args.prec), "peak_kind": "measured (rlbm_fma_peak probe, "
                "FP64 FMA chains on every SM, this run)",
                "fp64_instructions_per_site": per_site,
                "hbm": {"achieved": achieved, "peak": hbm, "frac": achieved / hbm}}
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16dev": "f16 storage / f32 compute",
                  "bf16dev": "bf16 storage / f32 compute (unsuitable for these low-Mach flows: "
                             "u error 0.37 after 10k steps at 4096x2048)"}[args.prec],
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": args.prec, "sites": sites,
                   "launch_shape": {"sites_per_block": shape[0] or 128,
                                    "blocks": shape[1] or "one per tile",
                                    "kernel": "single-sample" if shape[0] == 0 else
                                              ("batched, staged pulls" if shape[2] else "batched")},
                   "l2": "before every timed step a 2x L2 buffer is written, then another 2x L2 buffer read (cold L2, no pending write-backs); steps timed alone",
                   "parallelism": "replicas only" if world > 1 else "single GPU"},
        "roofline": roof,
        "back_to_back": {"value": world * sites * args.steps / (b2b_ms / 1e3) / 1e9,
                         "unit": "GLUPS", "ms_per_step": b2b_ms / args.steps,
                         "frac_of_hbm_peak": alg_bytes * args.steps / (b2b_ms / 1e3) / 1e9 / hbm,
                         "note": "the same K steps in one event pair, no L2 flush: each step's "
                                 "write-backs land inside the timed region"},
        "e2e": {"value": world * sites * args.steps / (e2e_ms / 1e3) / 1e9, "unit": "GLUPS",
                "h2d_bytes_per_step": field_bytes / args.steps,
                "d2h_bytes_per_step": field_bytes / args.steps,
                "note": f"init from pinned host fields + {args.steps} steps + read-back of four "
                        "FP64 fields in one event pair"},
        "gpu_launches": launches,
        "clocks": clk,
        "ms_per_step_x_sm_mhz": t_ms / args.steps * clk["sm_mhz"],
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

    clocks = Clocks(local)
    clocks.start()
    with torch.cuda.stream(stream):
        sv.init()
        for _ in range(args.warmup):
            flush_l2()
            sv.step(1)
    sync_all()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    l0 = sv.launches
    sync_all()
    clocks.mark("timed0")
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush_l2()
            ev[k][0].record(stream)
            sv.step(1)
            ev[k][1].record(stream)
    sync_all()
    clocks.mark("timed1")
    launches = sv.launches - l0
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
    clk = clocks.stop()
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
                     "frac": achieved / hbm, "traffic": ncu_traffic("massive_" + args.prec + ("_force0" if args.force == 0 else "")),
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

    clocks = Clocks(local)
    clocks.start()
    with torch.cuda.stream(stream):
        sv.step(args.warmup)
    sync_all()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = sv.launches
    sync_all()
    clocks.mark("timed0")
    e0.record(stream)
    sv.step(args.steps)
    e1.record(stream)
    sync_all()
    clocks.mark("timed1")
    launches = sv.launches - l0
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
    clk = clocks.stop()
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
                  "bf16dev": "bf16 storage / f32 compute (unsuitable for these low-Mach flows: "
                             "u error 0.37 after 10k steps at 4096x2048)"}[args.prec],
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
