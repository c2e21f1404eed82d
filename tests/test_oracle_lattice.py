"""Pins for the oracle's streaming, boundaries and whole-run behaviour (CPU).

Independent references:
  * a literal per-site, per-population loop of the pull / wall / contact /
    periodic rules on tiny grids (brute force);
  * streaming with periodic wrap and bounce-back walls is a permutation of
    the post-collision values, so with F = 0 the global N^0 and T^00 are
    conserved exactly (and T^0i too when fully periodic);
  * the decay of a transverse shear wave at the rate nu k^2 with the lattice
    kinematic viscosity nu = (tau - 1/2) c^2 / 4, c = 5 sites per step, which
    at n = T = tau = 1 is the shear viscosity eta = nu (eps + P) = 3/8 quoted
    in the paper's commented calibration (Sec. 3).
"""
import numpy as np
import pytest

from oracle import lbm, quadrature
from paper_1804_02418_gb300 import workloads as W


def brute_force_stream(lat, post):
    t = lbm.tables()
    out = np.zeros_like(post)
    for y in range(lat.ny):
        for x in range(lat.nx):
            for i in range(48):
                dx, dy = (int(v) for v in t.hop[i])
                sx, sy = x - dx, y - dy
                if lat.px:
                    sx %= lat.nx
                if lat.py:
                    sy %= lat.ny
                if 0 <= sx < lat.nx and 0 <= sy < lat.ny:
                    out[i, y, x] = post[i, sy, sx]
                    continue
                owner = -1
                for k, c in enumerate(lat.contacts):
                    lo, hi = c.x0, c.x0 + c.length
                    hit = ((c.edge == 0 and sy < 0 and lo <= sx < hi)
                           or (c.edge == 1 and sy >= lat.ny and lo <= sx < hi)
                           or (c.edge == 2 and sx < 0 and lo <= sy < hi)
                           or (c.edge == 3 and sx >= lat.nx and lo <= sy < hi))
                    if hit:
                        owner = k
                        break
                if owner >= 0:
                    out[i, y, x] = lat.ghost[owner, i]
                else:
                    out[i, y, x] = post[t.opposite[i], y, x]
    return out


def tiny_samples():
    C = W.Contact
    return [
        W.Sample(13, 12, contacts=[C(0, 0, 4, u_n=0.01), C(3, 3, 5, n=1.1, T=0.9),
                                   C(1, 6, 7, u_n=-0.02)]),
        W.Sample(11, 14, periodic_x=True, contacts=[C(0, 2, 6, u_n=0.03), C(1, 0, 11)]),
        W.Sample(12, 11, periodic_y=True, contacts=[C(2, 1, 9, u_n=0.01, T=1.2)]),
        W.Sample(12, 12, periodic_x=True, periodic_y=True),
        W.Sample(11, 11),
    ]


@pytest.mark.parametrize("k", range(5))
def test_stream_matches_brute_force(k):
    s = tiny_samples()[k]
    lat = lbm.Lattice(s)
    rng = np.random.default_rng(10 + k)
    post = rng.standard_normal((48, s.ny, s.nx))
    assert np.array_equal(lat.stream(post), brute_force_stream(lat, post))


@pytest.mark.parametrize("k", [3, 4])
def test_stream_without_contacts_is_a_permutation(k):
    s = tiny_samples()[k]
    lat = lbm.Lattice(s)
    post = np.random.default_rng(20).standard_normal((48, s.ny, s.nx))
    out = lat.stream(post)
    assert np.array_equal(np.sort(out.ravel()), np.sort(post.ravel()))


def test_closed_box_conserves_mass_and_energy():
    s = W.Sample(24, 20, tau=0.9)
    lat = lbm.Lattice(s)
    n, ux, uy, T = W.random_fields(s, seed=3)
    post = lbm.init(lat, n, ux, uy, T)
    t = lbm.tables()
    def totals(p):
        return np.tensordot(t.P[0], p, axes=(0, 0)).sum(), np.tensordot(t.P[0] ** 2, p, axes=(0, 0)).sum()
    m0, e0 = totals(post)
    post = lbm.run(lat, post, 40)
    m1, e1 = totals(post)
    sites = s.nx * s.ny
    assert abs(m1 - m0) < 1e-13 * sites
    assert abs(e1 - e0) < 1e-13 * 2 * sites


def _shear_run(tau, steps, n=64):
    s = W.shear_wave(n, tau)
    lat = lbm.Lattice(s)
    fields = W.shear_wave_fields(s)
    post = lbm.init(lat, *fields)
    t = lbm.tables()
    y = np.arange(n)
    basis = np.sin(2 * np.pi * y / n)
    amps, cons = [], []
    for k in range(steps):
        ux = lbm.macroscopic(lat, post)[1]
        amps.append(2.0 / (n * n) * np.sum(ux * basis[:, None]))
        cons.append([np.tensordot(t.P[0], post, axes=(0, 0)).sum(),
                     np.tensordot(t.P[0] * t.P[1], post, axes=(0, 0)).sum(),
                     np.tensordot(t.P[0] * t.P[2], post, axes=(0, 0)).sum(),
                     np.tensordot(t.P[0] ** 2, post, axes=(0, 0)).sum()])
        post = lbm.step(lat, post)
    return np.array(amps), np.array(cons), s


def _decay_ratio(amps, tau, n, t0, t1):
    tt = np.arange(len(amps))[t0:t1]
    slope = np.polyfit(tt, np.log(amps[t0:t1]), 1)[0]
    nu = (tau - 0.5) * 25.0 / 4.0
    k = 2 * np.pi / n
    return -slope / (nu * k * k)


def test_shear_wave_64_decay_and_global_invariants():
    """64^2 doubly periodic, tau = 0.8, u_x = 0.01 sin(2 pi y / 64), 500 steps."""
    amps, cons, s = _shear_run(0.8, 500)
    ratio = _decay_ratio(amps, 0.8, 64, 50, 500)
    assert abs(ratio - 1.0) < 0.01, ratio
    sites = s.nx * s.ny
    drift = np.abs(cons - cons[0]).max(axis=0)
    assert drift[0] < 1e-13 * sites          # N^0
    assert drift[1] < 1e-13 * sites          # T^0x
    assert drift[2] < 1e-13 * sites          # T^0y
    assert drift[3] < 1e-13 * 2 * sites      # T^00


def test_viscosity_three_eighths_at_unit_tau():
    amps, _, _ = _shear_run(1.0, 300)
    ratio = _decay_ratio(amps, 1.0, 64, 40, 300)
    eta = ratio * (1.0 - 0.5) / 4.0 * 3.0        # nu (eps + P), n = T = 1
    assert abs(eta - 3.0 / 8.0) < 0.01 * 3.0 / 8.0, eta


def _strip_decay_ratio(ny, steps, tau=0.8, nx=16):
    """Shear wave u_x = 0.01 sin(2 pi y / ny) on a doubly periodic strip (the
    wave is uniform along x, so 16 columns suffice): decay rate over the
    Chapman-Enskog rate nu k^2, nu = (tau - 1/2) c^2 / 4, c = 5 sites."""
    s = W.Sample(nx, ny, periodic_x=True, periodic_y=True, tau=tau)
    lat = lbm.Lattice(s)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    basis = np.sin(2 * np.pi * y / ny)
    o = np.ones_like(basis)
    post = lbm.init(lat, o, 0.01 * basis, 0 * o, o)
    amps = []
    for _ in range(steps):
        ux = lbm.macroscopic(lat, post)[1]
        amps.append((ux * basis).sum() / (basis * basis).sum())
        post = lbm.step(lat, post)
    tt = np.arange(steps)
    slope = np.polyfit(tt[steps // 10:], np.log(amps[steps // 10:]), 1)[0]
    return -slope / ((tau - 0.5) * 25.0 / 4.0 * (2 * np.pi / ny) ** 2)


def test_shear_decay_converges_at_second_order():
    """Doubling the wavelength brings the decay rate about 4x closer to the
    Chapman-Enskog value (lattice error ~ k^2)."""
    e64 = abs(_strip_decay_ratio(64, 500) - 1)
    e128 = abs(_strip_decay_ratio(128, 2000) - 1)
    assert e64 < 0.01 and e128 < 0.0025
    assert 3.0 < e64 / e128 < 5.0, (e64, e128)
