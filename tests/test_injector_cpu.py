"""Host-side analysis of the potential near an injector (injector.py), on
synthetic fields whose answer is known (no GPU)."""
import numpy as np
import pytest

from paper_1804_02418_gb300 import injector


def test_bilinear_is_exact_on_linear_fields():
    y, x = np.mgrid[0:20, 0:30].astype(float)
    a = 0.3 + 0.02 * x - 0.05 * y
    xs, ys = np.array([3.25, 10.5, 27.9]), np.array([1.5, 17.75, 4.1])
    assert np.allclose(injector.bilinear(a, xs, ys), 0.3 + 0.02 * xs - 0.05 * ys, atol=1e-14)


def test_hop_average_is_the_box_mean():
    rng = np.random.default_rng(0)
    a = rng.standard_normal((12, 17))
    b = injector.hop_average(a)
    for (j, i) in [(0, 0), (5, 8), (11, 16), (2, 15)]:
        box = a[max(0, j - 2):j + 3, max(0, i - 2):i + 3]
        assert b[j, i] == pytest.approx(box.mean(), rel=1e-12)
    assert np.allclose(injector.hop_average(np.full((9, 9), 2.5)), 2.5)


def test_analyse_recovers_a_planted_cos2theta_over_r2_law():
    """U = A cos(2 theta) / r^2 + const about the injector (r in sites):
    every circle's fit returns A / r^2 and the constant, with no misfit."""
    s = injector.geometry(nx=400, ny=200, width=8)
    xc = s.contacts[0].x0 + s.contacts[0].length / 2.0 - 0.5
    y, x = np.mgrid[0:s.ny, 0:s.nx].astype(float)
    dx, dy = x - xc, y + 0.5
    r2 = dx * dx + dy * dy
    A, B = 3.0e-3, 0.7
    U = A * (dx * dx - dy * dy) / r2 / r2 + B           # cos(2 theta) = (dx^2 - dy^2) / r^2
    th, prof, fits, eta, pred = injector.analyse(s, U, I=1e-4, n0=1.5, T0=1.25,
                                                 radii=(20, 40, 60), smooth=False)
    for r in (20, 40, 60):
        a_fit, b_fit, rms = fits[r]
        # bilinear sampling of a smooth field: relative error ~ (1 / r)^2
        assert a_fit == pytest.approx(A / r ** 2, rel=5e-3)
        assert b_fit == pytest.approx(B, abs=1e-3 * A / r ** 2 + 1e-12)
        assert rms < 1e-2
    # the law's prediction uses eta = (3/4) n T (tau - 1/2)
    assert eta == pytest.approx(0.75 * 1.5 * 1.25 * (s.tau - 0.5))
    assert pred == pytest.approx(-2 * 1e-4 * eta / (np.pi * 1.5 ** 2))
