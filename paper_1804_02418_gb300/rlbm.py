"""Python binding of librlbm (C ABI in include/rlbm.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch provides the device memory (the workspace tensor the
context borrows) and the stream (torch.cuda.current_stream()).  If the
library cannot be loaded, constructing a Solver raises; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from . import workloads

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "librlbm.so")

RLBM_Q = 48
PRECISIONS = {"f64": 0, "f32": 1, "f16dev": 2, "bf16dev": 3}
ERRORS = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ENAN", -5: "ETIMEOUT", -6: "ESTATE"}


class RlbmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rlbm error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class _Contact(ctypes.Structure):
    _fields_ = [("edge", ctypes.c_int), ("x0", ctypes.c_int), ("length", ctypes.c_int),
                ("u_n", ctypes.c_double), ("n", ctypes.c_double), ("T", ctypes.c_double)]


class _Sample(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
                ("tau", ctypes.c_double), ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
                ("ncontacts", ctypes.c_int), ("contacts", _Contact * 4),
                ("inv_cg", ctypes.c_double)]


class _Config(ctypes.Structure):
    _fields_ = [("prec", ctypes.c_int), ("nsamples", ctypes.c_int),
                ("samples", ctypes.POINTER(_Sample)), ("stream", ctypes.c_void_p),
                ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("graph_steps", ctypes.c_int), ("tune_cache", ctypes.c_char_p)]


_LIB = None

EXPORTS = {
    "rlbm_version": (ctypes.c_int, []),
    "rlbm_quadrature": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)] * 3),
    "rlbm_workspace_size": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_size_t)]),
    "rlbm_create": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_void_p)]),
    "rlbm_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "rlbm_init_ce": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "rlbm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "rlbm_moments": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_int]),
    "rlbm_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "rlbm_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int]),
    "rlbm_check": (ctypes.c_int, [ctypes.c_void_p]),
    "rlbm_steps_done": (ctypes.c_longlong, [ctypes.c_void_p]),
    "rlbm_launch_count": (ctypes.c_longlong, [ctypes.c_void_p]),
    "rlbm_destroy": (None, [ctypes.c_void_p]),
    "rlbm_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "rlbm_sample_residuals": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "rlbm_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int),
                                     ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "rlbm_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "rlbm_rows_raw_bytes": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "rlbm_get_rows_raw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p]),
    "rlbm_set_rows_raw": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p]),
    "rlbm_set_launch_shape": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_int]),
    "rlbm_velocity_residual_static": (ctypes.c_int, [ctypes.c_void_p] * 4 + [
        ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]),
    "rlbm_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
}


def load_library(path: str = LIB_PATH):
    """Loads librlbm.so (raises if it is missing: build it first)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run `python -m paper_1804_02418_gb300.build`")
    lib = ctypes.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def quadrature():
    """The library's refined (w1, w2, p0) as numpy arrays (host only)."""
    lib = load_library()
    w1, w2, p0 = (ctypes.c_double * 4)(), (ctypes.c_double * 4)(), (ctypes.c_double * 4)()
    rc = lib.rlbm_quadrature(w1, w2, p0)
    if rc:
        raise RlbmError(rc, lib.rlbm_last_error(None).decode())
    return np.array(w1[:]), np.array(w2[:]), np.array(p0[:])


def fma_peak(fp64: bool) -> float:
    """FMA instructions per second the current device retires (FP64 or FP32),
    measured by the library's probe kernel."""
    lib = load_library()
    r = ctypes.c_double()
    rc = lib.rlbm_fma_peak(int(bool(fp64)), ctypes.byref(r))
    if rc:
        raise RlbmError(rc, lib.rlbm_last_error(None).decode())
    return r.value


def _to_c_sample(s: workloads.Sample) -> _Sample:
    c = _Sample()
    c.nx, c.ny = int(s.nx), int(s.ny)
    c.periodic_x, c.periodic_y = int(bool(s.periodic_x)), int(bool(s.periodic_y))
    c.tau, c.Fx, c.Fy = float(s.tau), float(s.Fx), float(s.Fy)
    c.inv_cg = float(getattr(s, "inv_cg", 0.0))
    c.ncontacts = len(s.contacts)
    if c.ncontacts > 4:
        raise ValueError("at most 4 contacts per sample")
    for k, ct in enumerate(s.contacts):
        c.contacts[k].edge, c.contacts[k].x0, c.contacts[k].length = int(ct.edge), int(ct.x0), int(ct.length)
        c.contacts[k].u_n, c.contacts[k].n, c.contacts[k].T = float(ct.u_n), float(ct.n), float(ct.T)
    return c


def _ptr(a):
    """(pointer, is_device) for a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise ValueError("host arrays must be C-contiguous float64")
        return a.ctypes.data, False
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors must be contiguous float64")
        if a.is_cuda:
            return a.data_ptr(), True
        return a.data_ptr(), False
    raise TypeError(f"unsupported array type {type(a)}")


class Solver:
    """A context advancing one or more samples together on the current CUDA device."""

    def __init__(self, samples, prec: str = "f32", stream=None, workspace: Optional[str] = "torch",
                 graph_steps: int = 0, tune_cache: Optional[str] = None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = load_library()
        if isinstance(samples, workloads.Sample):
            samples = [samples]
        self.samples = list(samples)
        self._csamples = (_Sample * len(self.samples))(*[_to_c_sample(s) for s in self.samples])
        self.prec = prec
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = _Config()
        cfg.prec = PRECISIONS[prec]
        cfg.nsamples = len(self.samples)
        cfg.samples = self._csamples
        cfg.stream = ctypes.c_void_p(self._stream.cuda_stream)
        cfg.graph_steps = int(graph_steps)
        self._tune_cache = tune_cache.encode() if tune_cache else None
        cfg.tune_cache = self._tune_cache
        need = ctypes.c_size_t()
        self._check(self.lib.rlbm_workspace_size(ctypes.byref(cfg), ctypes.byref(need)), None)
        self.workspace_bytes = need.value
        self._ws = None
        if workspace == "torch":
            self._ws = torch.empty(need.value + 256, dtype=torch.uint8, device="cuda")
            base = self._ws.data_ptr()
            aligned = (base + 255) // 256 * 256
            cfg.workspace = ctypes.c_void_p(aligned)
            cfg.workspace_bytes = need.value
        self._cfg = cfg
        ctx = ctypes.c_void_p()
        self._check(self.lib.rlbm_create(ctypes.byref(cfg), ctypes.byref(ctx)), None)
        self.ctx = ctx

    # -- helpers -----------------------------------------------------------
    def _check(self, rc, ctx="self"):
        if rc != 0:
            c = self.ctx if ctx == "self" else None
            msg = self.lib.rlbm_last_error(c)
            raise RlbmError(rc, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.rlbm_destroy(self.ctx)
            self.ctx = None
        self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API ---------------------------------------------------------------
    def init(self, sample: int = 0, n=None, ux=None, uy=None, T=None):
        ptrs = [_ptr(a) for a in (n, ux, uy, T)]
        dev = any(p[1] for p in ptrs if p[0] is not None)
        args = [ctypes.c_void_p(p[0]) if p[0] is not None else None for p in ptrs]
        self._check(self.lib.rlbm_init(self.ctx, sample, *args, int(bool(dev))))

    def init_ce(self, sample: int = 0, n=None, ux=None, uy=None, T=None):
        """The Chapman-Enskog seed of the fields (rlbm_init_ce): f^eq plus its
        first-order non-equilibrium part after the first streaming."""
        ptrs = [_ptr(a) for a in (n, ux, uy, T)]
        dev = any(p[1] for p in ptrs if p[0] is not None)
        args = [ctypes.c_void_p(p[0]) if p[0] is not None else None for p in ptrs]
        self._check(self.lib.rlbm_init_ce(self.ctx, sample, *args, int(bool(dev))))

    def step(self, nsteps: int, residual: bool = False):
        if residual:
            r = ctypes.c_double()
            self._check(self.lib.rlbm_step(self.ctx, int(nsteps), ctypes.byref(r)))
            return r.value
        self._check(self.lib.rlbm_step(self.ctx, int(nsteps), None))
        return None

    def moments(self, sample: int = 0, out=None):
        """(n, ux, uy, T).  With out=None returns host numpy arrays [ny][nx];
        out may be four preallocated arrays (host numpy or CUDA tensors)."""
        s = self.samples[sample]
        if out is None:
            out = [np.empty((s.ny, s.nx)) for _ in range(4)]
        ptrs = [_ptr(a) for a in out]
        dev = any(p[1] for p in ptrs if p[0] is not None)
        args = [ctypes.c_void_p(p[0]) if p[0] is not None else None for p in ptrs]
        self._check(self.lib.rlbm_moments(self.ctx, sample, *args, int(bool(dev))))
        return tuple(out)

    def get_state(self, sample: int = 0, out=None):
        s = self.samples[sample]
        if out is None:
            out = np.empty((RLBM_Q, s.ny, s.nx))
        p, dev = _ptr(out)
        self._check(self.lib.rlbm_get_state(self.ctx, sample, ctypes.c_void_p(p), int(bool(dev))))
        return out

    def set_state(self, delta, sample: int = 0):
        p, dev = _ptr(delta)
        self._check(self.lib.rlbm_set_state(self.ctx, sample, ctypes.c_void_p(p), int(bool(dev))))

    def check(self):
        self._check(self.lib.rlbm_check(self.ctx))

    def sample_residuals(self):
        out = (ctypes.c_double * len(self.samples))()
        self._check(self.lib.rlbm_sample_residuals(self.ctx, out))
        return np.array(out[:])

    def autotune(self):
        """Times the launch shapes on the current state; returns (bx, grid, staged)."""
        bx, grid, staged = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self._check(self.lib.rlbm_autotune(self.ctx, ctypes.byref(bx), ctypes.byref(grid),
                                           ctypes.byref(staged)))
        return bx.value, grid.value, staged.value

    def set_launch_shape(self, bx, grid=0, staged=0):
        """Pins the launch shape (bx 0: single-sample kernel; 64 / 128 / 256:
        batched, grid blocks (0: one per tile), staged pulls if staged)."""
        self._check(self.lib.rlbm_set_launch_shape(self.ctx, int(bx), int(grid), int(staged)))

    def rows_raw_bytes(self, nrows: int, sample: int = 0) -> int:
        n = ctypes.c_size_t()
        self._check(self.lib.rlbm_rows_raw_bytes(self.ctx, sample, int(nrows), ctypes.byref(n)))
        return n.value

    def get_rows_raw(self, y0: int, nrows: int, out, sample: int = 0):
        """Raw stored values of rows y0 .. y0 + nrows - 1 into the device
        tensor `out` (rows_raw_bytes(nrows) bytes)."""
        if not out.is_cuda or out.numel() * out.element_size() < self.rows_raw_bytes(nrows, sample):
            raise ValueError("out: a device tensor of rows_raw_bytes(nrows) bytes")
        self._check(self.lib.rlbm_get_rows_raw(self.ctx, sample, int(y0), int(nrows),
                                               ctypes.c_void_p(out.data_ptr())))
        return out

    def set_rows_raw(self, y0: int, nrows: int, src, sample: int = 0):
        if not src.is_cuda or src.numel() * src.element_size() < self.rows_raw_bytes(nrows, sample):
            raise ValueError("src: a device tensor of rows_raw_bytes(nrows) bytes")
        self._check(self.lib.rlbm_set_rows_raw(self.ctx, sample, int(y0), int(nrows),
                                               ctypes.c_void_p(src.data_ptr())))

    def set_wait_limit(self, cycles: int):
        """Longest bounded device wait in clock cycles (0: the default, ~1 s)."""
        self._check(self.lib.rlbm_set_wait_limit(self.ctx, int(cycles)))

    @property
    def steps_done(self) -> int:
        return int(self.lib.rlbm_steps_done(self.ctx))

    @property
    def launches(self) -> int:
        return int(self.lib.rlbm_launch_count(self.ctx))
