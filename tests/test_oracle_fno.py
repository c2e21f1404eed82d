"""Pins for the oracle spectral neural operator (CPU).

* the DFT-matrix form of the spectral convolution equals its definition with
  numpy.fft (rfft2 / truncation / per-mode mixing / irfft2);
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


def test_matrix_spectral_conv_equals_fft_definition():
    rng = np.random.default_rng(1)
    N, C, m1, m2 = 16, 4, 3, 5
    o = fno.Oracle(N, m1, m2)
    h = rng.standard_normal((2, N, N, C))
    R = rng.standard_normal((2 * m1, m2, C, C)) + 1j * rng.standard_normal((2 * m1, m2, C, C))
    a, _ = o.spec_fwd(h, R)
    b = fno.spectral_conv_fft(h, R, m1)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()


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
