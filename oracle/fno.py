"""Oracle: FP64 reference of the spectral neural operator used as a learned
warm start (no counterpart in the paper; it only initialises the method).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, FP64.

Network (channels-last fields [B, N, N, C]):
    h0   = x P + bp
    z_l  = S_l(h_l) + h_l W_l + b_l,  h_{l+1} = gelu(z_l) (no gelu after the last layer)
    y    = gelu(h_L Q1 + bq1) Q2 + bq2
    loss = sum_m |y - t|^2 / (4 sum_m)      (mask m over sites)
Spectral convolution S_l: 2-D real DFT of every channel, keep the modes
kx in {0..m1-1} U {N-m1..N-1}, ky in {0..m2-1}, multiply every kept mode by a
complex C x C matrix R_l(kx, ky), inverse real DFT (numpy.fft.irfft2
conventions: the ky = 0 column counts once and its imaginary part is
dropped, ky > 0 counts twice, normalisation 1/N^2).

Both the forward map and its adjoint are written here as products with the
real DFT matrices of that definition (`dft_mats`), so the backward pass is
the exact transpose; `spectral_conv_fft` restates the forward with
numpy.fft as the independent definition the matrices are checked against,
and the gradients are checked against finite differences (tests).
"""
from __future__ import annotations

import numpy as np
from scipy.special import erf


def gelu(x):
    return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))


def gelu_grad(x):
    return 0.5 * (1.0 + erf(x / np.sqrt(2.0))) + x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)


def kx_list(N, m1):
    return np.concatenate([np.arange(m1), np.arange(N - m1, N)])


def dft_mats(N, m1, m2):
    """Real matrices of the truncated forward / inverse DFT.

    F1 [2 m2, N]:      y -> (re, im) x ky        (exp(-i 2 pi ky y / N))
    D  [2 KX, 2 N]:    (x, re/im) -> (kx, re/im)  (exp(-i 2 pi kx x / N)), KX = 2 m1
    Dinv [2 N, 2 KX]:  (kx, re/im) -> (x, re/im)  (exp(+i 2 pi kx x / N))
    G  [N, 2 m2]:      (re/im, ky) -> y           (c_ky Re(. exp(+i 2 pi ky y / N)) / N^2)
    Row / column orders: F1 rows reim * m2 + ky; D rows kxi * 2 + reim,
    columns x * 2 + reim; G columns reim * m2 + ky.
    """
    y = np.arange(N)
    ky = np.arange(m2)
    th = 2 * np.pi * np.outer(ky, y) / N                         # [m2, N]
    F1 = np.concatenate([np.cos(th), -np.sin(th)], axis=0)
    kx = kx_list(N, m1)
    ph = 2 * np.pi * np.outer(kx, np.arange(N)) / N              # [KX, N]
    KX = len(kx)
    D = np.zeros((2 * KX, 2 * N))
    D[0::2, 0::2] = np.cos(ph)       # re <- re
    D[0::2, 1::2] = np.sin(ph)       # re <- im
    D[1::2, 0::2] = -np.sin(ph)      # im <- re
    D[1::2, 1::2] = np.cos(ph)       # im <- im
    Dinv = np.zeros((2 * N, 2 * KX))
    Dinv[0::2, 0::2] = np.cos(ph).T
    Dinv[0::2, 1::2] = -np.sin(ph).T
    Dinv[1::2, 0::2] = np.sin(ph).T
    Dinv[1::2, 1::2] = np.cos(ph).T
    c = np.where(ky == 0, 1.0, 2.0)
    G = np.concatenate([(c[:, None] * np.cos(th)).T, (-c[:, None] * np.sin(th)).T], axis=1) / (N * N)
    return F1, D, Dinv, G


def spectral_conv_fft(h, R, m1):
    """Definition of the spectral convolution with numpy.fft.  h [B, N, N, C],
    R complex [2 m1, m2, C, C] (kx order of kx_list)."""
    B, N, _, C = h.shape
    m2 = R.shape[1]
    H = np.fft.rfft2(h, axes=(1, 2))                            # [B, N, N/2+1, C]
    kx = kx_list(N, m1)
    Ht = H[:, kx][:, :, :m2]                                    # [B, 2 m1, m2, C]
    U = np.einsum("bxyi,xyio->bxyo", Ht, R)
    Up = np.zeros_like(H)
    Up[:, kx, :m2] = U
    return np.fft.irfft2(Up, s=(N, N), axes=(1, 2))


class Oracle:
    """Parameters: dict with P [cin, C], bp [C], W [L, C, C], b [L, C],
    R [L, 2 m1, m2, C, C] complex, Q1 [C, Cq], bq1 [Cq], Q2 [Cq, 4], bq2 [4]."""

    def __init__(self, N, m1, m2):
        self.N, self.m1, self.m2 = N, m1, m2
        self.F1, self.D, self.Dinv, self.G = dft_mats(N, m1, m2)

    # -- spectral convolution as matrix products ---------------------------
    def spec_fwd(self, h, R):
        B, N, _, C = h.shape
        m2, KX = self.m2, 2 * self.m1
        S1 = np.einsum("ky,bxyc->bxkc", self.F1, h)              # [B, x, (reim, ky), C]
        S1 = S1.reshape(B, N, 2, m2, C).reshape(B, 2 * N, m2 * C)  # rows (x, reim)
        S2 = np.einsum("rs,bsj->brj", self.D, S1)                # [B, (kx, reim), (ky, C)]
        S2c = S2.reshape(B, KX, 2, m2, C)
        Sc = S2c[:, :, 0] + 1j * S2c[:, :, 1]                    # [B, KX, m2, C]
        Uc = np.einsum("bxyi,xyio->bxyo", Sc, R)
        U = np.stack([Uc.real, Uc.imag], axis=2).reshape(B, 2 * KX, m2 * C)
        Wm = np.einsum("sr,brj->bsj", self.Dinv, U)              # [B, (x, reim), (ky, C)]
        Wm = Wm.reshape(B, N, 2 * m2, C)                         # [B, x, (reim, ky), C]
        out = np.einsum("yk,bxkc->bxyc", self.G, Wm)
        return out, (S1, Sc, Wm)

    def spec_bwd(self, dout, R, cache):
        S1, Sc, Wm = cache
        B, N, _, C = dout.shape
        m2, KX = self.m2, 2 * self.m1
        dWm = np.einsum("yk,bxyc->bxkc", self.G, dout)           # [B, x, (reim, ky), C]
        dWm = dWm.reshape(B, 2 * N, m2 * C)
        dU = np.einsum("sr,bsj->brj", self.Dinv, dWm)            # [B, (kx, reim), (ky, C)]
        dUc4 = dU.reshape(B, KX, 2, m2, C)
        dUc = dUc4[:, :, 0] + 1j * dUc4[:, :, 1]
        dSc = np.einsum("bxyo,xyio->bxyi", dUc, np.conj(R))
        dR = np.einsum("bxyi,bxyo->xyio", np.conj(Sc), dUc)
        dS2 = np.stack([dSc.real, dSc.imag], axis=2).reshape(B, 2 * KX, m2 * C)
        dS1 = np.einsum("rs,brj->bsj", self.D, dS2)              # [B, (x, reim), (ky, C)]
        dS1 = dS1.reshape(B, N, 2 * m2, C)
        dh = np.einsum("ky,bxkc->bxyc", self.F1, dS1)
        return dh, dR

    # -- network -------------------------------------------------------------
    def forward(self, p, x):
        L = p["W"].shape[0]
        c = {"x": x}
        h = x @ p["P"] + p["bp"]
        hs, zs, sc = [h], [], []
        for l in range(L):
            s, cache = self.spec_fwd(h, p["R"][l])
            z = s + h @ p["W"][l] + p["b"][l]
            zs.append(z)
            sc.append(cache)
            h = gelu(z) if l < L - 1 else z
            hs.append(h)
        z1 = h @ p["Q1"] + p["bq1"]
        y1 = gelu(z1)
        y = y1 @ p["Q2"] + p["bq2"]
        c.update(hs=hs, zs=zs, sc=sc, z1=z1, y1=y1)
        return y, c

    @staticmethod
    def loss(y, t, m):
        d = y - t
        den = 4.0 * max(m.sum(), 1.0)
        return float((m[..., None] * d * d).sum() / den), 2.0 * m[..., None] * d / den

    def backward(self, p, c, dy):
        L = p["W"].shape[0]
        g = {}
        flat = lambda a: a.reshape(-1, a.shape[-1])
        g["Q2"] = flat(c["y1"]).T @ flat(dy)
        g["bq2"] = flat(dy).sum(0)
        dz1 = (dy @ p["Q2"].T) * gelu_grad(c["z1"])
        hL = c["hs"][L]
        g["Q1"] = flat(hL).T @ flat(dz1)
        g["bq1"] = flat(dz1).sum(0)
        dh = dz1 @ p["Q1"].T
        gW = np.zeros_like(p["W"])
        gb = np.zeros_like(p["b"])
        gR = np.zeros_like(p["R"])
        for l in reversed(range(L)):
            z = c["zs"][l]
            dz = dh * gelu_grad(z) if l < L - 1 else dh
            h = c["hs"][l]
            gW[l] = flat(h).T @ flat(dz)
            gb[l] = flat(dz).sum(0)
            dh_s, gR[l] = self.spec_bwd(dz, p["R"][l], c["sc"][l])
            dh = dz @ p["W"][l].T + dh_s
        g["W"], g["b"], g["R"] = gW, gb, gR
        g["P"] = flat(c["x"]).T @ flat(dh)
        g["bp"] = flat(dh).sum(0)
        return g


def init_params(rng, cin, C, Cq, L, m1, m2):
    """Seeded initial parameters (uniform, fan-in scaled; spectral weights
    scaled by 1/(C C) as is usual for these operators)."""
    def u(shape, fan):
        a = 1.0 / np.sqrt(fan)
        return rng.uniform(-a, a, shape)
    s = 1.0 / (C * C)
    return {
        "P": u((cin, C), cin), "bp": u((C,), cin),
        "W": u((L, C, C), C), "b": u((L, C), C),
        "R": s * (rng.uniform(0, 1, (L, 2 * m1, m2, C, C)) + 1j * rng.uniform(0, 1, (L, 2 * m1, m2, C, C))),
        "Q1": u((C, Cq), C), "bq1": u((Cq,), C),
        "Q2": u((Cq, 4), Cq), "bq2": u((4,), Cq),
    }
