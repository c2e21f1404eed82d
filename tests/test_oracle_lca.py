"""Oracle: electric force of the local capacitance approximation (Sec. 3,
Eq. lca), F_E = -(e^2 / C_g) grad n per particle from the previous step's
density.

Pins (none of them re-types the oracle's formula):
* the lattice gradient (over one hop, 5 sites = the length unit of c = 1) is
  exact on linear fields (central inside, forward / backward next to walled
  edges) and equals the discrete identity
  (sin(x + 5h) - sin(x - 5h)) / 2 = sin(5h) cos(x) on a periodic axis;
* the force points away from a density bump (repulsion), and density noise
  on the scale of single sites decays with it;
* with inv_cg = 0 the step is the plain step, bit for bit;
* with a site-dependent force the collision still conserves N^0 and changes
  T^0i by F^i N^0 at every site;
* sound speed: linearising the massless fluid (eps = 2 n T, P = eps / 2,
  enthalpy w = 3 n T) with the force gives
      w d_t u = -d_x P - n (e^2 / C_g) d_x n,   d_t n = -n d_x u,
      d_t eps = -w d_x u   =>   c_s^2 = 1/2 + n (e^2 / C_g) / (3 T).
  A standing sound wave on a periodic lattice must oscillate with the ratio
  of frequencies this predicts (1 %), and at inv_cg = 0 with c_s = 1/sqrt(2)
  (2 %).
"""
import numpy as np
import pytest

from oracle import lbm, quadrature
from paper_1804_02418_gb300 import workloads as W


def lattice(nx, ny, px=False, py=False, inv_cg=0.0, tau=0.8):
    return lbm.Lattice(W.Sample(nx, ny, periodic_x=px, periodic_y=py, tau=tau, inv_cg=inv_cg))


@pytest.mark.parametrize("px,py", [(False, False), (True, False), (False, True)])
def test_gradient_is_exact_on_linear_fields(px, py):
    lat = lattice(13, 11, px, py)
    y, x = np.meshgrid(np.arange(11), np.arange(13), indexing="ij")
    a = 0.3 + 0.02 * x - 0.05 * y
    gx, gy = lat.grad(a)
    # a periodic axis wraps: check only the interior there
    ix = slice(5, -5) if px else slice(None)
    iy = slice(5, -5) if py else slice(None)
    assert np.allclose(gx[iy, ix], 5 * 0.02, rtol=0, atol=1e-13)
    assert np.allclose(gy[iy, ix], -5 * 0.05, rtol=0, atol=1e-13)


def test_gradient_on_a_periodic_axis_is_the_discrete_sine_identity():
    nx = 40
    lat = lattice(nx, 11, px=True, py=True)
    h = 2 * np.pi / nx
    x = np.arange(nx)
    a = np.tile(np.sin(h * x + 0.4), (11, 1))
    gx, gy = lat.grad(a)
    assert np.allclose(gx, np.sin(5 * h) * np.cos(h * x + 0.4)[None, :], atol=1e-14)
    assert np.abs(gy).max() < 1e-14


def test_force_pushes_away_from_a_density_bump():
    lat = lattice(31, 11, inv_cg=0.5)
    x = np.arange(31)
    dn = np.tile(1e-3 * np.exp(-0.1 * (x - 15.0) ** 2), (11, 1))
    fx, fy = lat.electric_force(dn)
    assert (fx[:, 17:30] > 0).all() and (fx[:, 1:14] < 0).all()
    assert np.abs(fy).max() == 0.0


def test_zero_coupling_is_the_plain_step():
    s = W.graphene_sample(nx=64, ny=32, contact_width=4, contact_spacing=16)
    lat0 = lbm.Lattice(s)
    fields = W.random_fields(s, 3, du=0.02, dn=0.01, dT=0.01)
    post = lbm.init(lat0, *fields)
    a = lbm.run(lat0, post, 3)
    b, _ = lbm.run_lca(lat0, post, fields[0] - 1.0, 3)
    assert np.array_equal(a, b)


def test_site_dependent_force_keeps_the_collision_invariants():
    rng = np.random.default_rng(8)
    shape = (30,)
    n = rng.uniform(0.8, 1.2, shape)
    T = rng.uniform(0.8, 1.2, shape)
    ux = rng.uniform(-0.2, 0.2, shape)
    uy = rng.uniform(-0.2, 0.2, shape)
    Fx = rng.uniform(-1e-3, 1e-3, shape)
    Fy = rng.uniform(-1e-3, 1e-3, shape)
    q = quadrature.quadrature()
    P = np.array([q["P0"], q["PX"], q["PY"]])
    delta = lbm.equilibrium_deviation(n, ux, uy, T)
    out = lbm.collide(delta, 0.9, Fx, Fy)
    d = out - delta
    g = 1 / np.sqrt(1 - ux ** 2 - uy ** 2)
    N0 = n * g
    assert np.abs(P[0] @ d).max() < 1e-15
    dT0 = np.einsum("i,ai,is->as", P[0], P, d)
    assert np.allclose(dT0[1], Fx * N0, rtol=1e-11, atol=1e-18)
    assert np.allclose(dT0[2], Fy * N0, rtol=1e-11, atol=1e-18)


@pytest.mark.parametrize("inv_cg", [0.1, 0.3])
def test_site_scale_noise_decays_with_the_force_on(inv_cg):
    """Density noise on the scale of single sites (not resolved by a hop)
    must decay, not grow, with the electric force on: at the paper's C_g = 10
    (0.1) and at 0.3 (tau = 0.8; the stable range of the lagged hop-scale
    force ends between 0.3 and 0.5 there)."""
    s = W.Sample(30, 30, periodic_x=True, periodic_y=True, tau=0.8, inv_cg=inv_cg)
    lat = lbm.Lattice(s)
    f = W.random_fields(s, 3, du=1e-4, dn=1e-4, dT=1e-4)
    post, dn = lbm.run_lca(lat, lbm.init(lat, *f), f[0] - 1.0, 300)
    assert np.abs(dn).max() < 1e-4


def sound_period(inv_cg, nx=160, steps=120):
    """Period (steps) of a standing sound wave of wavelength nx sites."""
    ny = 11
    lat = lattice(nx, ny, px=True, py=True, inv_cg=inv_cg, tau=0.6)
    k = 2 * np.pi / nx
    x = np.arange(nx)
    dn = np.tile(1e-4 * np.cos(k * x), (ny, 1))
    n = 1.0 + dn
    T = 1.0 + dn / 2            # pure acoustic mode: no static (entropy) part
    z = np.zeros_like(n)
    post = lbm.init(lat, n, z, z, T)
    dn_prev = dn
    basis = np.sin(k * x)
    amp = []
    for _ in range(steps):
        post, dn_prev = lbm.step_lca(lat, post, dn_prev)
        ux = lbm.macroscopic(lat, post)[1]
        amp.append(float((ux * basis[None, :]).mean()))
    a = np.array(amp)
    # zero crossings of the velocity amplitude, linearly interpolated
    z = [i + a[i] / (a[i] - a[i + 1]) for i in range(len(a) - 1) if a[i] * a[i + 1] < 0]
    assert len(z) >= 3, z
    return 2 * np.mean(np.diff(z))


def test_electric_force_stiffens_sound_as_linear_hydrodynamics_predicts():
    inv_cg = 0.3
    p0 = sound_period(0.0)
    p1 = sound_period(inv_cg)
    wavelength = 160 / 5.0                       # in the length unit of c = 1
    assert abs(wavelength / p0 / np.sqrt(0.5) - 1.0) < 0.02
    predicted = np.sqrt((0.5 + inv_cg / 3.0) / 0.5)
    assert abs((p0 / p1) / predicted - 1.0) < 0.01, (p0, p1, p0 / p1, predicted)
