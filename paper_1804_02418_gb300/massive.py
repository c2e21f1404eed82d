"""Python binding of the massive-particle variant (C ABI in include/rlbm_massive.h).

Argument marshalling only: the quadrature solve runs in the library's host
code and every step in its CUDA kernels.  Rest mass m = 5 T0 on the 45-vector
stencil of Fig. m5-stencil (Sec. 2.3); see the header for the population
order, units and readings.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import rlbm

Q = 45
PRECISIONS = {"f64": 0, "f32": 1}


class _Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("periodic_x", ctypes.c_int), ("periodic_y", ctypes.c_int),
                ("tau", ctypes.c_double), ("Fx", ctypes.c_double), ("Fy", ctypes.c_double),
                ("prec", ctypes.c_int), ("stream", ctypes.c_void_p)]


_P = ctypes.c_void_p
_EXPORTS = {
    "rlbm_massive_quadrature": (ctypes.c_int, [ctypes.POINTER(ctypes.c_double)] * 4),
    "rlbm_massive_stencil": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)] * 2),
    "rlbm_massive_create": (ctypes.c_int, [ctypes.POINTER(_Config), ctypes.POINTER(_P)]),
    "rlbm_massive_init": (ctypes.c_int, [_P] * 5 + [ctypes.c_int]),
    "rlbm_massive_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "rlbm_massive_moments": (ctypes.c_int, [_P] * 5 + [ctypes.c_int]),
    "rlbm_massive_get_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "rlbm_massive_set_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "rlbm_massive_check": (ctypes.c_int, [_P]),
    "rlbm_massive_steps_done": (ctypes.c_longlong, [_P]),
    "rlbm_massive_launch_count": (ctypes.c_longlong, [_P]),
    "rlbm_massive_destroy": (None, [_P]),
    "rlbm_massive_last_error": (ctypes.c_char_p, [_P]),
}
rlbm.EXPORTS.update(_EXPORTS)


def _lib():
    lib = rlbm.load_library()
    for name, (res, args) in _EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _raise(lib, rc, ctx=None):
    if rc != 0:
        msg = lib.rlbm_massive_last_error(ctx)
        raise rlbm.RlbmError(rc, msg.decode() if msg else "")


def quadrature():
    """dict: v0, window (lo, hi), class weights w[10] and energies p0[10]
    (classes (1,0) (1,1) (2,0) (2,1) (2,2) (3,0) (3,2) (3,3) (4,0) (0,0)); host only."""
    lib = _lib()
    v0 = ctypes.c_double()
    win = (ctypes.c_double * 2)()
    w = (ctypes.c_double * 10)()
    p0 = (ctypes.c_double * 10)()
    _raise(lib, lib.rlbm_massive_quadrature(ctypes.byref(v0), win, w, p0))
    return {"v0": v0.value, "window": (win[0], win[1]), "w": np.array(w[:]), "p0": np.array(p0[:])}


def stencil():
    """(45, 2) integer stencil vectors in population order (host only)."""
    lib = _lib()
    vx, vy = (ctypes.c_int * Q)(), (ctypes.c_int * Q)()
    _raise(lib, lib.rlbm_massive_stencil(vx, vy))
    return np.stack([np.array(vx[:]), np.array(vy[:])], axis=1)


class MassiveSolver:
    """One nx x ny sample of the massive-particle fluid on the current CUDA device."""

    def __init__(self, nx, ny, periodic_x=False, periodic_y=False, tau=1.0, Fx=0.0, Fy=0.0,
                 prec="f64", stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        self.lib = _lib()
        self.nx, self.ny = int(nx), int(ny)
        self._stream = stream if stream is not None else torch.cuda.current_stream()
        cfg = _Config()
        cfg.nx, cfg.ny = self.nx, self.ny
        cfg.periodic_x, cfg.periodic_y = int(bool(periodic_x)), int(bool(periodic_y))
        cfg.tau, cfg.Fx, cfg.Fy = float(tau), float(Fx), float(Fy)
        cfg.prec = PRECISIONS[prec]
        cfg.stream = ctypes.c_void_p(self._stream.cuda_stream)
        self.prec = prec
        ctx = ctypes.c_void_p()
        _raise(self.lib, self.lib.rlbm_massive_create(ctypes.byref(cfg), ctypes.byref(ctx)))
        self.ctx = ctx

    def _check(self, rc):
        _raise(self.lib, rc, self.ctx)

    def close(self):
        if getattr(self, "ctx", None) is not None and self.ctx.value:
            self.lib.rlbm_massive_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def init(self, n=None, ux=None, uy=None, T=None):
        ptrs = [rlbm._ptr(a) for a in (n, ux, uy, T)]
        dev = any(p[1] for p in ptrs if p[0] is not None)
        args = [ctypes.c_void_p(p[0]) if p[0] is not None else None for p in ptrs]
        self._check(self.lib.rlbm_massive_init(self.ctx, *args, int(bool(dev))))

    def step(self, nsteps: int, residual: bool = False):
        """Advances nsteps; with residual=True returns ||u(t) - u(t-1)|| / ||u(t)||
        over the last step (synchronises)."""
        if residual:
            r = ctypes.c_double()
            self._check(self.lib.rlbm_massive_step(self.ctx, int(nsteps), ctypes.byref(r)))
            return r.value
        self._check(self.lib.rlbm_massive_step(self.ctx, int(nsteps), None))
        return None

    def moments(self, out=None):
        """(n, ux, uy, T): host numpy arrays [ny][nx], or into `out` (four
        host arrays or CUDA float64 tensors)."""
        if out is None:
            out = [np.empty((self.ny, self.nx)) for _ in range(4)]
        ptrs = [rlbm._ptr(a) for a in out]
        dev = any(p[1] for p in ptrs if p[0] is not None)
        args = [ctypes.c_void_p(p[0]) if p[0] is not None else None for p in ptrs]
        self._check(self.lib.rlbm_massive_moments(self.ctx, *args, int(bool(dev))))
        return tuple(out)

    def get_state(self, out=None):
        """Deviations f_i - f0_i, [45][ny][nx] FP64."""
        if out is None:
            out = np.empty((Q, self.ny, self.nx))
        p, dev = rlbm._ptr(out)
        self._check(self.lib.rlbm_massive_get_state(self.ctx, ctypes.c_void_p(p), int(bool(dev))))
        return out

    def set_state(self, delta):
        p, dev = rlbm._ptr(delta)
        self._check(self.lib.rlbm_massive_set_state(self.ctx, ctypes.c_void_p(p), int(bool(dev))))

    def check(self):
        self._check(self.lib.rlbm_massive_check(self.ctx))

    @property
    def steps_done(self) -> int:
        return int(self.lib.rlbm_massive_steps_done(self.ctx))

    @property
    def launches(self) -> int:
        return int(self.lib.rlbm_massive_launch_count(self.ctx))
