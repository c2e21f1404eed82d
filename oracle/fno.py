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

Both the forward map and its adjoint are written with numpy.fft from that
definition (no transform matrices):
    forward   out = irfft2(pad(R (x) trunc(rfft2(h))))
    adjoint   with g = d loss / d out (real), the gradient with respect to the
              kept half-spectrum Z of irfft2 is rfft2(g) c_ky / N^2
              (c_ky = 1 for ky = 0, 2 otherwise); through the mixing
              dS = conj(R) dU and dR = sum_b conj(S) dU; and the gradient
              with respect to h of H = rfft2(h) at the kept modes is
              Re(sum_kept dH exp(+i 2 pi (kx x + ky y) / N)), one term per
              kept (kx, ky) (an inverse 2-D FFT of the scattered modes).
The tests pin the forward against a brute-force double sum over sites and
modes, the adjoint by the identity <S h, g> = <h, S^T g>, and every gradient
of the network by central finite differences.
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


def spectral_conv_fft(h, R, m1):
    """The spectral convolution by its definition with numpy.fft.
    h [B, N, N, C] real, R complex [2 m1, m2, C, C] (kx order of kx_list)."""
    return spectral_fwd(h, R, m1)[0]


def spectral_fwd(h, R, m1):
    """Forward of the spectral convolution; returns (out, kept spectrum S)."""
    B, N, _, C = h.shape
    m2 = R.shape[1]
    kx = kx_list(N, m1)
    H = np.fft.rfft2(h, axes=(1, 2))                            # [B, N, N/2+1, C]
    S = H[:, kx][:, :, :m2]                                     # [B, 2 m1, m2, C]
    U = np.einsum("bxyi,xyio->bxyo", S, R)
    Z = np.zeros((B, N, N // 2 + 1, C), dtype=complex)
    Z[:, kx[:, None], np.arange(m2)[None, :]] = U
    return np.fft.irfft2(Z, s=(N, N), axes=(1, 2)), S


def spectral_bwd(g, R, S, m1):
    """Adjoint of spectral_fwd: gradients (dh, dR) of a real loss with
    d loss / d out = g, the kept spectrum S of the forward given."""
    B, N, _, C = g.shape
    m2 = R.shape[1]
    kx = kx_list(N, m1)
    c = np.where(np.arange(m2) == 0, 1.0, 2.0)
    dU = np.fft.rfft2(g, axes=(1, 2))[:, kx][:, :, :m2] * (c[None, None, :, None] / (N * N))
    dS = np.einsum("bxyo,xyio->bxyi", dU, np.conj(R))
    dR = np.einsum("bxyi,bxyo->xyio", np.conj(S), dU)
    full = np.zeros((B, N, N, C), dtype=complex)
    full[:, kx[:, None], np.arange(m2)[None, :]] = dS
    dh = np.real(np.fft.ifft2(full, axes=(1, 2))) * (N * N)
    return dh, dR


class Oracle:
    """Parameters: dict with P [cin, C], bp [C], W [L, C, C], b [L, C],
    R [L, 2 m1, m2, C, C] complex, Q1 [C, Cq], bq1 [Cq], Q2 [Cq, 4], bq2 [4]."""

    def __init__(self, N, m1, m2):
        self.N, self.m1, self.m2 = N, m1, m2

    # -- spectral convolution (numpy.fft, see the module docstring) ---------
    def spec_fwd(self, h, R):
        out, S = spectral_fwd(h, R, self.m1)
        return out, S

    def spec_bwd(self, dout, R, cache):
        return spectral_bwd(dout, R, cache, self.m1)

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
