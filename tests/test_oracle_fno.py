"""Pins for the oracle spectral neural operator (CPU).

* the spectral convolution equals a brute-force double sum over sites and
  kept modes (the definition: forward DFT, truncation, per-mode complex
  mixing, inverse real DFT with the ky = 0 column counted once);
* its adjoint satisfies <S h, g> = <h, S^T g> and <S h, g> is linear in R
  with the gradient the adjoint returns;
* every parameter gradient of the masked loss equals central finite
  differences of the loss.
"""
import numpy as np
import pytest

from oracle import fno


def tiny(seed=0, N=12, C=3, Cq=5, L=2, m1=2, m2=3, B=2):
    rng = np.random.default_rng(seed)
    p = fno.init_params(rng, 5, C, Cq, L, m1, m2)
    x = rng.standard_normal((B, N, N, 5))
    t = rng.standard_normal((B, N, N, 4))
    m = (rng.uniform(size=(B, N, N)) < 0.7).astype(float)
    return fno.Oracle(N, m1, m2), p, x, t, m


def brute_force_spectral_conv(h, R, m1):
    """out(x, y) = sum over kept (kx, ky) of c_ky Re(U(kx, ky) e^{+i th}) / N^2,
    U = sum_i S_i R_io, S(kx, ky) = sum_{x', y'} h(x', y') e^{-i th'},
    th = 2 pi (kx x + ky y) / N, c_ky = 1 for ky = 0 and 2 otherwise."""
    B, N, _, C = h.shape
    m2 = R.shape[1]
    kxs = list(range(m1)) + list(range(N - m1, N))
    out = np.zeros_like(h)
    xs = np.arange(N)
    for a, kx in enumerate(kxs):
        for ky in range(m2):
            ph = np.exp(-2j * np.pi * (kx * xs[:, None] + ky * xs[None, :]) / N)   # [x, y]
            S = np.einsum("bxyi,xy->bi", h, ph)
            U = S @ R[a, ky]                                                        # [B, C]
            c = 1.0 if ky == 0 else 2.0
            out += c * np.real(U[:, None, None, :] * np.conj(ph)[None, :, :, None]) / (N * N)
    return out


def test_spectral_conv_equals_brute_force_definition():
    rng = np.random.default_rng(1)
    N, C, m1, m2 = 10, 3, 3, 4
    h = rng.standard_normal((2, N, N, C))
    R = rng.standard_normal((2 * m1, m2, C, C)) + 1j * rng.standard_normal((2 * m1, m2, C, C))
    a = fno.spectral_conv_fft(h, R, m1)
    b = brute_force_spectral_conv(h, R, m1)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


def test_spectral_adjoint_identity():
    rng = np.random.default_rng(2)
    N, C, m1, m2, B = 16, 4, 3, 5, 2
    h = rng.standard_normal((B, N, N, C))
    g = rng.standard_normal((B, N, N, C))
    R = rng.standard_normal((2 * m1, m2, C, C)) + 1j * rng.standard_normal((2 * m1, m2, C, C))
    out, S = fno.spectral_fwd(h, R, m1)
    dh, dR = fno.spectral_bwd(g, R, S, m1)
    lhs = (out * g).sum()
    assert abs(lhs - (h * dh).sum()) < 1e-12 * np.abs(out * g).sum()
    # <S h, g> is real-linear in R: its derivative along a direction E is
    # Re(sum conj(dR) E) (gradient convention d/dRe + i d/dIm)
    E = rng.standard_normal(R.shape) + 1j * rng.standard_normal(R.shape)
    t = 1e-3
    lin = ((fno.spectral_fwd(h, R + t * E, m1)[0] * g).sum() - lhs) / t
    assert abs(lin - np.real(np.sum(np.conj(dR) * E))) < 1e-9 * max(1.0, abs(lin))


def test_gradients_match_finite_differences():
    o, p, x, t, m = tiny()
    y, c = o.forward(p, x)
    _, dy = o.loss(y, t, m)
    g = o.backward(p, c, dy)
    rng = np.random.default_rng(2)
    h = 1e-6
    for name, val in p.items():
        flat = val.reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            for part in ((1.0,) if not np.iscomplexobj(val) else (1.0, 1j)):
                q = {k: v.copy() for k, v in p.items()}
                q[name].reshape(-1)[idx] += h * part
                lp = o.loss(o.forward(q, x)[0], t, m)[0]
                q[name].reshape(-1)[idx] -= 2 * h * part
                lm = o.loss(o.forward(q, x)[0], t, m)[0]
                fd = (lp - lm) / (2 * h)
                an = g[name].reshape(-1)[idx]
                an = an.real if part == 1.0 else an.imag
                assert abs(fd - an) <= 1e-6 * max(1e-3, abs(fd)), (name, idx, part, fd, an)
