"""Oracle pins of the Chapman-Enskog seed (oracle/lbm.py: chapman_enskog_init).

The seed is the stored state whose first pull-stream gives, at every site x
and population i whose source x - n_i lies inside the sample,
    f_i(x) = f^eq_i(x) - (f^eq_i(x) - f^eq_i(x - n_i)) / omega_i(x),
omega_i = gamma (1 - v_i.u) / tau (Eq. discrete-rbe): the equilibrium plus its
first-order Chapman-Enskog part of a steady flow.  Pinned here by
  * a brute-force loop over every site and population of small samples with
    walls, contacts and periodic axes (index arithmetic, wrap, boundary rule);
  * uniform fields, whose seed is the equilibrium itself;
  * the shear stress it carries: for a small linear shear u_x = a y the
    non-equilibrium T^xy is minus the Anderson-Witting (continuum) shear
    viscosity (3/4) n T tau times du_x/dy (reading 4: the gradient per length
    unit is 5 times the gradient per site), the Navier-Stokes stress of the
    relaxation-time model to first order.
"""
import math

import numpy as np
import pytest

from oracle import lbm
from paper_1804_02418_gb300 import workloads as W

HOPS = [(3, 4), (-3, -4), (-3, 4), (3, -4), (4, 3), (-4, -3), (-4, 3), (4, -3),
        (5, 0), (-5, 0), (0, 5), (0, -5)]


def smooth_fields(s, seed):
    rng = np.random.default_rng(seed)
    y, x = np.meshgrid(np.arange(s.ny), np.arange(s.nx), indexing="ij")
    ph = rng.uniform(0, 2 * np.pi, 4)
    n = 1 + 0.02 * np.sin(2 * np.pi * x / s.nx + ph[0]) * np.cos(2 * np.pi * y / s.ny)
    ux = 0.03 * np.sin(2 * np.pi * y / s.ny + ph[1])
    uy = 0.02 * np.cos(2 * np.pi * x / s.nx + ph[2])
    T = 1 + 0.01 * np.cos(2 * np.pi * (x / s.nx + y / s.ny) + ph[3])
    return n, ux, uy, T


CASES = {
    "walls_and_contacts": lambda: W.Sample(13, 12, tau=0.9, contacts=[
        W.Contact(0, 2, 5, u_n=0.01), W.Contact(3, 4, 5, n=1.01)]),
    "periodic_x": lambda: W.Sample(14, 11, periodic_x=True, tau=0.7),
    "doubly_periodic": lambda: W.Sample(12, 13, periodic_x=True, periodic_y=True, tau=1.3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_streamed_seed_is_equilibrium_plus_first_order_part_brute_force(name):
    s = CASES[name]()
    lat = lbm.Lattice(s)
    n, ux, uy, T = smooth_fields(s, 3)
    eq = lbm.init(lat, n, ux, uy, T)
    got = lat.stream(lbm.chapman_enskog_init(lat, n, ux, uy, T))
    checked = 0
    for i in range(48):
        hx, hy = HOPS[i // 4]
        for yy in range(s.ny):
            for xx in range(s.nx):
                sx, sy = xx - hx, yy - hy
                if s.periodic_x:
                    sx %= s.nx
                if s.periodic_y:
                    sy %= s.ny
                if not (0 <= sx < s.nx and 0 <= sy < s.ny):
                    continue          # a wall or contact supplies this population
                u_x, u_y = ux[yy, xx], uy[yy, xx]
                gamma = 1.0 / math.sqrt(1.0 - u_x * u_x - u_y * u_y)
                om = gamma * (1.0 - (hx * u_x + hy * u_y) / 5.0) / s.tau
                want = eq[i, yy, xx] - (eq[i, yy, xx] - eq[i, sy, sx]) / om
                assert abs(got[i, yy, xx] - want) <= 1e-15 + 1e-13 * abs(want), (i, xx, yy)
                checked += 1
    assert checked > 0


def test_uniform_fields_seed_is_the_equilibrium():
    s = CASES["walls_and_contacts"]()
    lat = lbm.Lattice(s)
    one = np.ones((s.ny, s.nx))
    f = (1.02 * one, 0.03 * one, -0.01 * one, 0.98 * one)
    assert np.array_equal(lbm.chapman_enskog_init(lat, *f), lbm.init(lat, *f))


@pytest.mark.parametrize("tau,n0,T0", [(0.8, 1.0, 1.0), (0.8, 1.3, 0.9), (1.2, 0.7, 1.4)])
def test_seed_carries_the_first_order_shear_stress(tau, n0, T0):
    nx, ny, a = 8, 64, 1e-6
    s = W.Sample(nx, ny, periodic_x=True, tau=tau)
    lat = lbm.Lattice(s)
    y = np.arange(ny)[:, None] * np.ones((1, nx))
    ux = a * (y - ny / 2)
    n, uy, T = n0 * np.ones_like(ux), 0 * ux, T0 * np.ones_like(ux)
    f = lat.stream(lbm.chapman_enskog_init(lat, n, ux, uy, T))
    t = lbm.tables()
    Txy = np.tensordot(t.P[1] * t.P[2], f - lbm.init(lat, n, ux, uy, T), axes=(0, 0))
    inner = Txy[6:-6]                       # sites whose sources all lie inside
    eta = 0.75 * n0 * T0 * tau              # Anderson-Witting, massless 2-D gas
    np.testing.assert_allclose(inner, -eta * 5 * a, rtol=1e-8)
    # a sign or direction error (downwind difference, omega at the source in
    # place of 1 / omega) would change this stress at first order
    assert np.all(inner < 0)
