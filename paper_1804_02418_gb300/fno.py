"""Spectral neural operator (Fourier neural operator) on the GPU: forward,
backward and Adam, every step in the library's kernels (include/rlbm_fno.h).

Used as a learned warm start of the relativistic LBM: it maps per-site
inputs on an N x N canvas (geometry mask, drive, relaxation time, x, y) to
normalised steady fields (n, u_x, u_y, T).  PyTorch only allocates the
buffers; this module marshals pointers and sizes.

Network (channels-last [B, N, N, C]):
    h0  = x P + bp
    z_l = S_l(h_l) + h_l W_l + b_l,   h_{l+1} = gelu(z_l)  (identity after the last layer)
    y   = gelu(h_L Q1 + bq1) Q2 + bq2
with the spectral convolution S_l = truncated real DFT (modes kx in
{0..m1-1} U {N-m1..N-1}, ky < m2) -> per-mode complex C x C mixing R_l ->
inverse real DFT, evaluated as BF16 tensor-core GEMMs with DFT matrices:
    step 1  (y):  S1[b, x]  = F1   h[b, x]        [2 m2, C]
    step 2  (x):  S2[b]     = D    S1[b]          [2 KX, m2 C]
    mixing:       U         = R (x) S2            (FP32, per mode)
    step 2' (x):  Wm[b]     = Dinv U[b]           [2 N, m2 C]
    step 1' (y):  out[b, x] = G    Wm[b, x]       [N, C]
"""
from __future__ import annotations

import ctypes
import math
from dataclasses import dataclass

import numpy as np

from . import rlbm

EPI_NONE, EPI_GELU, EPI_ATOMIC = 0, 1, 2
# GEMM back ends: "tc" (default) = tcgen05 with the accumulator in tensor
# memory, "mma" = warp-level mma.sync m16n8k16 (kept as a cross-check)
GEMM_IMPLS = {"mma": "rlbm_gemm_bf16", "tc": "rlbm_gemm_bf16_tc"}

_FNO_EXPORTS = {
    "rlbm_gemm_bf16": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                      ctypes.c_int, ctypes.c_float,
                                      ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong,
                                      ctypes.c_void_p, ctypes.c_longlong, ctypes.c_longlong,
                                      ctypes.c_float, ctypes.c_void_p, ctypes.c_longlong,
                                      ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
    "rlbm_gemm_tc_error": (ctypes.c_int, [ctypes.POINTER(ctypes.c_int)]),
    "rlbm_fno_mix_forward": (ctypes.c_int, [ctypes.c_void_p] * 3 + [ctypes.c_int] * 4 + [ctypes.c_void_p]),
    "rlbm_fno_mix_backward": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_int] * 4 + [ctypes.c_void_p]),
    "rlbm_fno_gelu_backward": (ctypes.c_int, [ctypes.c_void_p] * 4 + [ctypes.c_longlong, ctypes.c_void_p]),
    "rlbm_fno_to_bf16": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p]),
    "rlbm_fno_mse": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p]),
    "rlbm_fno_colsum": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p]),
    "rlbm_fno_adam": (ctypes.c_int, [ctypes.c_void_p] * 5 + [ctypes.c_longlong] + [ctypes.c_float] * 4 + [ctypes.c_int, ctypes.c_void_p]),
    "rlbm_resample_bilinear": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p]),
}
_FNO_EXPORTS["rlbm_gemm_bf16_tc"] = _FNO_EXPORTS["rlbm_gemm_bf16"]
_FNO_EXPORTS["rlbm_gemm_f32"] = _FNO_EXPORTS["rlbm_gemm_bf16"]
rlbm.EXPORTS.update(_FNO_EXPORTS)


def _lib():
    lib = rlbm.load_library()
    for name, (res, args) in _FNO_EXPORTS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def _p(t):
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("FNO kernels take dense row-major buffers")
    return ctypes.c_void_p(t.data_ptr())


def _ok(rc, what):
    if rc != 0:
        raise rlbm.RlbmError(rc, what)


def dft_mats(N, m1, m2):
    """Real truncated-DFT matrices (see module docstring for the orders)."""
    y = np.arange(N)
    ky = np.arange(m2)
    th = 2 * np.pi * np.outer(ky, y) / N
    F1 = np.concatenate([np.cos(th), -np.sin(th)], axis=0)                  # [2 m2, N]
    kx = np.concatenate([np.arange(m1), np.arange(N - m1, N)])
    ph = 2 * np.pi * np.outer(kx, y) / N                                     # [KX, N]
    KX = 2 * m1
    D = np.zeros((2 * KX, 2 * N))
    D[0::2, 0::2], D[0::2, 1::2] = np.cos(ph), np.sin(ph)
    D[1::2, 0::2], D[1::2, 1::2] = -np.sin(ph), np.cos(ph)
    Dinv = np.zeros((2 * N, 2 * KX))
    Dinv[0::2, 0::2], Dinv[0::2, 1::2] = np.cos(ph).T, -np.sin(ph).T
    Dinv[1::2, 0::2], Dinv[1::2, 1::2] = np.sin(ph).T, np.cos(ph).T
    c = np.where(ky == 0, 1.0, 2.0)
    G = np.concatenate([(c[:, None] * np.cos(th)).T, (-c[:, None] * np.sin(th)).T], axis=1) / (N * N)
    return F1, D, Dinv, G


@dataclass
class FNOConfig:
    N: int = 256          # canvas
    C: int = 32           # width
    Cq: int = 128         # projection width
    L: int = 4            # Fourier layers
    m1: int = 16          # kept modes along x (each sign)
    m2: int = 16          # kept modes along y
    cin: int = 5
    cout: int = 4


class FNO:
    """Parameters live in one flat FP32 vector (Adam state alongside) with a
    BF16 shadow used by the GEMMs.

    act = "bf16" (default): weights, activations and DFT matrices in BF16 on
    the tensor cores (gemm_impl "tc" or "mma"), FP32 accumulation and FP32
    spectral mixing.  act = "f32": everything in FP32 on the FP32 units
    (rlbm_gemm_f32), the same sequence of kernels; the "16" buffers are then
    the FP32 buffers themselves.  Inputs to forward() are of the act type."""

    def __init__(self, cfg: FNOConfig, batch: int, seed: int = 0, device="cuda",
                 gemm_impl: str = "tc", act: str = "bf16"):
        import torch
        self.torch = torch
        self.cfg, self.B = cfg, batch
        self.lib = _lib()
        if act not in ("bf16", "f32"):
            raise ValueError("act must be 'bf16' or 'f32'")
        self.act = act
        if act == "f32":
            gemm_impl = "f32"
        elif gemm_impl not in GEMM_IMPLS:
            raise ValueError(f"gemm_impl must be one of {sorted(GEMM_IMPLS)}")
        self._gemm_fn = getattr(self.lib, "rlbm_gemm_f32" if act == "f32" else GEMM_IMPLS[gemm_impl])
        N, C, Cq, L, m1, m2, cin = cfg.N, cfg.C, cfg.Cq, cfg.L, cfg.m1, cfg.m2, cfg.cin
        KX = 2 * m1
        self.KX = KX
        shapes = [("P", (cin, C)), ("bp", (C,)), ("W", (L, C, C)), ("b", (L, C)),
                  ("R", (L, KX, m2, C, C, 2)), ("Q1", (C, Cq)), ("bq1", (Cq,)),
                  ("Q2", (Cq, cfg.cout)), ("bq2", (cfg.cout,))]
        self.offsets, off = {}, 0
        for name, shp in shapes:
            n = int(np.prod(shp))
            self.offsets[name] = (off, shp)
            off += (n + 63) // 64 * 64
        self.nparam = off
        f32 = dict(dtype=torch.float32, device=device)
        self.theta = torch.zeros(off, **f32)
        self.grad = torch.zeros(off, **f32)
        self.m = torch.zeros(off, **f32)
        self.v = torch.zeros(off, **f32)
        f32mode = act == "f32"
        self.theta16 = self.theta if f32mode else torch.zeros(off, dtype=torch.bfloat16, device=device)
        self.t = 0
        self.set_params(self.init_params(np.random.default_rng(seed)))
        F1, D, Dinv, G = dft_mats(N, m1, m2)
        b16 = dict(dtype=torch.float32 if f32mode else torch.bfloat16, device=device)
        # row-major copies (G is built column by column and is not C-ordered)
        self.F1 = torch.tensor(np.ascontiguousarray(F1), **b16).contiguous()
        self.D = torch.tensor(np.ascontiguousarray(D), **b16).contiguous()
        self.Dinv = torch.tensor(np.ascontiguousarray(Dinv), **b16).contiguous()
        self.G = torch.tensor(np.ascontiguousarray(G), **b16).contiguous()
        rows = batch * N * N
        self.rows = rows
        e16 = lambda *s: torch.empty(*s, **b16)
        e32 = lambda *s: torch.empty(*s, **f32)
        self.x16 = e16(rows, cin)
        self.h16 = [e16(rows, C) for _ in range(L + 1)]
        self.z = [e32(rows, C) for _ in range(L)]
        self.S1 = [e16(batch * N, 2 * m2, C) for _ in range(L)]
        self.S2 = [e32(batch, 2 * KX, m2 * C) for _ in range(L)]
        self.U = e32(batch, 2 * KX, m2 * C)
        self.U16 = self.U if f32mode else e16(batch, 2 * KX, m2 * C)
        self.Wm16 = e16(batch * N, 2 * m2, C)
        self.z1 = e32(rows, Cq)
        self.y116 = e16(rows, Cq)
        self.y = e32(rows, cfg.cout)
        # backward buffers
        self.dy = e32(rows, cfg.cout)
        self.dy16 = self.dy if f32mode else e16(rows, cfg.cout)
        self.dy1 = e32(rows, Cq)
        self.dz1 = e32(rows, Cq)
        self.dz116 = self.dz1 if f32mode else e16(rows, Cq)
        self.dh = e32(rows, C)
        self.dz = e32(rows, C)
        self.dz16 = self.dz if f32mode else e16(rows, C)
        self.dWm16 = e16(batch * N, 2 * m2, C)
        self.dU = e32(batch, 2 * KX, m2 * C)
        self.dS2 = e32(batch, 2 * KX, m2 * C)
        self.dS216 = self.dS2 if f32mode else e16(batch, 2 * KX, m2 * C)
        self.dS116 = e16(batch * N, 2 * m2, C)
        self.dh16 = self.dh if f32mode else e16(rows, C)
        self.loss_buf = torch.zeros(4, **f32)

    # -- parameters ---------------------------------------------------------
    def init_params(self, rng):
        c = self.cfg
        def u(shape, fan):
            a = 1.0 / math.sqrt(fan)
            return rng.uniform(-a, a, shape)
        s = 1.0 / (c.C * c.C)
        R = s * rng.uniform(0, 1, (c.L, self.KX, c.m2, c.C, c.C, 2))
        return {"P": u((c.cin, c.C), c.cin), "bp": u((c.C,), c.cin),
                "W": u((c.L, c.C, c.C), c.C), "b": u((c.L, c.C), c.C), "R": R,
                "Q1": u((c.C, c.Cq), c.C), "bq1": u((c.Cq,), c.C),
                "Q2": u((c.Cq, c.cout), c.Cq), "bq2": u((c.cout,), c.Cq)}

    def set_params(self, params):
        th = np.zeros(self.nparam, dtype=np.float32)
        for name, (off, shp) in self.offsets.items():
            th[off:off + int(np.prod(shp))] = np.asarray(params[name], dtype=np.float64).reshape(-1)
        self.theta.copy_(self.torch.from_numpy(th))
        if self.act == "bf16":
            _ok(self.lib.rlbm_fno_to_bf16(_p(self.theta), _p(self.theta16), self.nparam, None),
                "to_bf16")

    def get(self, name, which="theta"):
        off, shp = self.offsets[name]
        buf = getattr(self, which)
        return buf[off:off + int(np.prod(shp))].view(*shp)

    def params_numpy(self):
        return {n: self.get(n).cpu().numpy().astype(np.float64) for n in self.offsets}

    # -- kernels --------------------------------------------------------------
    def _stream(self):
        return ctypes.c_void_p(self.torch.cuda.current_stream().cuda_stream)

    def gemm(self, A, B, M, N, K, *, lda, ldb, transA=0, transB=0, C=None, ldc=None, D=None,
             bias=None, beta=0.0, epi=EPI_NONE, batch=1, sA=0, sB=0, sC=0, alpha=1.0):
        rc = self._gemm_fn(transA, transB, M, N, K, alpha, _p(A), lda, sA, _p(B), ldb, sB,
                                     beta, _p(C), ldc if ldc is not None else N, sC, _p(bias),
                                     _p(D), epi, batch, self._stream())
        _ok(rc, "gemm")

    def gemm_tn_sum(self, A16, B16, M, N, K, out):
        """out (f32 [M, N]) += A^T B with A [K, M], B [K, N] bf16: split-K over
        chunks of 512 rows (one block each, atomic accumulation into out); a
        ragged remainder is a second call."""
        chunk = 512
        nb = K // chunk
        if nb:
            self.gemm(A16, B16, M, N, chunk, lda=M, ldb=N, transA=1, C=out, ldc=N,
                      epi=EPI_ATOMIC, batch=nb, sA=chunk * M, sB=chunk * N, sC=0)
        rem = K - nb * chunk
        if rem:
            A = A16.reshape(K, M)[nb * chunk:]
            B = B16.reshape(K, N)[nb * chunk:]
            self.gemm(A, B, M, N, rem, lda=M, ldb=N, transA=1, C=out, ldc=N, epi=EPI_ATOMIC)

    def to16(self, x, y):
        """The GEMM-operand copy of an FP32 buffer (BF16 rounding; nothing in
        FP32 mode, where the two are the same buffer)."""
        if y.data_ptr() == x.data_ptr():
            return
        _ok(self.lib.rlbm_fno_to_bf16(_p(x), _p(y), x.numel(), self._stream()), "to_bf16")

    # -- forward ------------------------------------------------------------
    def forward(self, x16):
        """x16: [B N N, cin] of the act type (already on the device).  Returns
        y (f32 [B N N, 4])."""
        c = self.cfg
        N, C, Cq, L, m2, KX = c.N, c.C, c.Cq, c.L, c.m2, self.KX
        B, rows = self.B, self.rows
        t16 = self.theta16
        self.x16.copy_(x16)
        self.gemm(self.x16, self.get("P", "theta16"), rows, C, c.cin, lda=c.cin, ldb=C,
                  bias=self.get("bp"), D=self.h16[0])
        for l in range(L):
            h = self.h16[l]
            # step 1 over (b, x): S1 = F1 h[b, x]
            self.gemm(self.F1, h, 2 * m2, C, N, lda=N, ldb=C, D=self.S1[l], batch=B * N,
                      sA=0, sB=N * C, sC=2 * m2 * C)
            # step 2 over b: S2 = D S1[b]
            self.gemm(self.D, self.S1[l], 2 * KX, m2 * C, 2 * N, lda=2 * N, ldb=m2 * C,
                      C=self.S2[l], batch=B, sA=0, sB=2 * N * m2 * C, sC=2 * KX * m2 * C)
            _ok(self.lib.rlbm_fno_mix_forward(_p(self.S2[l]), _p(self.get("R")[l]), _p(self.U),
                                              B, KX, m2, C, self._stream()), "mix")
            self.to16(self.U, self.U16)
            # step 2': Wm = Dinv U[b]
            self.gemm(self.Dinv, self.U16, 2 * N, m2 * C, 2 * KX, lda=2 * KX, ldb=m2 * C,
                      D=self.Wm16, batch=B, sA=0, sB=2 * KX * m2 * C, sC=2 * N * m2 * C)
            # step 1' over (b, x): z = G Wm[b, x]
            self.gemm(self.G, self.Wm16, N, C, 2 * m2, lda=2 * m2, ldb=C, C=self.z[l],
                      batch=B * N, sA=0, sB=2 * m2 * C, sC=N * C)
            # z += h W + b, h_{l+1} = gelu(z) (identity after the last layer)
            self.gemm(h, self.get("W", "theta16")[l], rows, C, C, lda=C, ldb=C, C=self.z[l],
                      beta=1.0, bias=self.get("b")[l], D=self.h16[l + 1],
                      epi=EPI_GELU if l < L - 1 else EPI_NONE)
        self.gemm(self.h16[L], self.get("Q1", "theta16"), rows, Cq, C, lda=C, ldb=Cq, C=self.z1,
                  bias=self.get("bq1"), D=self.y116, epi=EPI_GELU)
        self.gemm(self.y116, self.get("Q2", "theta16"), rows, c.cout, Cq, lda=Cq, ldb=c.cout,
                  C=self.y, bias=self.get("bq2"))
        return self.y

    def loss(self, target, mask):
        """Masked MSE of the last forward against target (f32 [rows, 4]), mask
        (f32 [rows]); fills dy.  Returns the loss as a device scalar tensor."""
        _ok(self.lib.rlbm_fno_mse(_p(self.y), _p(target), _p(mask), _p(self.dy),
                                  _p(self.loss_buf), self.rows, self.cfg.cout, self._stream()), "mse")
        return self.loss_buf[0]

    # -- backward -----------------------------------------------------------
    def backward(self):
        """Gradients of the last loss() into self.grad (overwritten)."""
        c = self.cfg
        N, C, Cq, L, m2, KX = c.N, c.C, c.Cq, c.L, c.m2, self.KX
        B, rows = self.B, self.rows
        st = self._stream()
        self.grad.zero_()
        self.to16(self.dy, self.dy16)
        self.gemm_tn_sum(self.y116, self.dy16, Cq, c.cout, rows, self.get("Q2", "grad"))
        _ok(self.lib.rlbm_fno_colsum(_p(self.dy), _p(self.get("bq2", "grad")), rows, c.cout, st), "colsum")
        # dy1 = dy Q2^T ; dz1 = dy1 * gelu'(z1)
        self.gemm(self.dy16, self.get("Q2", "theta16"), rows, Cq, c.cout, lda=c.cout, ldb=c.cout,
                  transB=1, C=self.dy1)
        _ok(self.lib.rlbm_fno_gelu_backward(_p(self.z1), _p(self.dy1), _p(self.dz1),
                                            self._p16(self.dz116, self.dz1), rows * Cq, st),
            "gelu_bwd")
        self.gemm_tn_sum(self.h16[L], self.dz116, C, Cq, rows, self.get("Q1", "grad"))
        _ok(self.lib.rlbm_fno_colsum(_p(self.dz1), _p(self.get("bq1", "grad")), rows, Cq, st), "colsum")
        self.gemm(self.dz116, self.get("Q1", "theta16"), rows, C, Cq, lda=Cq, ldb=Cq, transB=1,
                  C=self.dh)
        for l in reversed(range(L)):
            if l < L - 1:
                _ok(self.lib.rlbm_fno_gelu_backward(_p(self.z[l]), _p(self.dh), _p(self.dz),
                                                    self._p16(self.dz16, self.dz), rows * C, st),
                    "gelu_bwd")
            else:
                self.dz.copy_(self.dh)
                self.to16(self.dz, self.dz16)
            self.gemm_tn_sum(self.h16[l], self.dz16, C, C, rows, self.get("W", "grad")[l])
            _ok(self.lib.rlbm_fno_colsum(_p(self.dz), _p(self.get("b", "grad")[l]), rows, C, st), "colsum")
            # spectral path backwards
            self.gemm(self.G, self.dz16, 2 * m2, C, N, lda=2 * m2, ldb=C, transA=1, D=self.dWm16,
                      batch=B * N, sA=0, sB=N * C, sC=2 * m2 * C)
            self.gemm(self.Dinv, self.dWm16, 2 * KX, m2 * C, 2 * N, lda=2 * KX, ldb=m2 * C,
                      transA=1, C=self.dU, batch=B, sA=0, sB=2 * N * m2 * C, sC=2 * KX * m2 * C)
            _ok(self.lib.rlbm_fno_mix_backward(_p(self.S2[l]), _p(self.get("R")[l]), _p(self.dU),
                                               _p(self.dS2), _p(self.get("R", "grad")[l]),
                                               B, KX, m2, C, st), "mix_bwd")
            self.to16(self.dS2, self.dS216)
            self.gemm(self.D, self.dS216, 2 * N, m2 * C, 2 * KX, lda=2 * N, ldb=m2 * C, transA=1,
                      D=self.dS116, batch=B, sA=0, sB=2 * KX * m2 * C, sC=2 * N * m2 * C)
            # dh = dz W^T + F1^T dS1[b, x]
            self.gemm(self.dz16, self.get("W", "theta16")[l], rows, C, C, lda=C, ldb=C, transB=1,
                      C=self.dh)
            self.gemm(self.F1, self.dS116, N, C, 2 * m2, lda=N, ldb=C, transA=1, C=self.dh,
                      beta=1.0, batch=B * N, sA=0, sB=2 * m2 * C, sC=N * C)
        self.to16(self.dh, self.dh16)
        self.gemm_tn_sum(self.x16, self.dh16, c.cin, C, rows, self.get("P", "grad"))
        _ok(self.lib.rlbm_fno_colsum(_p(self.dh), _p(self.get("bp", "grad")), rows, C, st), "colsum")
        return self.grad

    def _p16(self, y16, y32):
        """Pointer of a kernel's optional BF16 copy output (NULL in FP32 mode)."""
        return None if y16.data_ptr() == y32.data_ptr() else _p(y16)

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.t += 1
        _ok(self.lib.rlbm_fno_adam(_p(self.theta), _p(self.grad), _p(self.m), _p(self.v),
                                   self._p16(self.theta16, self.theta), self.nparam, lr, beta1,
                                   beta2, eps, self.t, self._stream()), "adam")
