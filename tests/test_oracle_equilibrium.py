"""Pins for the oracle's equilibrium (App. B, App. C, Eq. feq-expansion-discrete).

Fixed independently of the oracle by:
  * direct numerical projection of the exact Maxwell-Juttner distribution
    onto the App. A polynomials (continuum integral, Gauss-Laguerre x angle);
  * the App. C closed form (a separate transcription of the same function);
  * the ideal-fluid moments N_E = n U, T_E = (eps + P) U U - P eta with the
    massless equation of state eps = 2 P = 2 n T, and the massless 2-D third
    moment (n/T) T^3 [15 UUU - 3 (eta U + eta U + eta U)].
"""
import numpy as np
import pytest

from oracle import expansion, lbm, quadrature

STATES = [(1.0, 0.0, 0.0, 1.0), (1.3, 0.12, -0.07, 0.85), (0.8, -0.3, 0.2, 1.4),
          (1.5, 0.01, 0.02, 1.25), (1.1, 0.36, 0.0, 1.0), (0.9, -0.1, -0.33, 0.7)]
ETA = np.diag([1.0, -1.0, -1.0])


def U_of(ux, uy):
    g = 1.0 / np.sqrt(1 - ux * ux - uy * uy)
    return np.array([g, g * ux, g * uy])


@pytest.mark.parametrize("state", STATES)
def test_projections_match_continuum_integral(state):
    """a^(k) = (T/n) int f_MJ J^(k) d^2p/p0 with f_MJ = n/(2 pi T^2) exp(-p.U/T)."""
    n, ux, uy, T = state
    U = U_of(ux, uy)
    s, ws = np.polynomial.laguerre.laggauss(60)
    M = 256
    th = 2 * np.pi * np.arange(M) / M
    a_num = np.zeros(16)
    for t in th:
        lam = (U[0] - U[1] * np.cos(t) - U[2] * np.sin(t)) / T      # p.U / (T |p|)
        p = s / lam
        J = expansion.polynomials(p, p * np.cos(t), p * np.sin(t))
        for k in range(16):
            a_num[k] += np.sum(ws * J[k]) / lam / (2 * np.pi * T) * (2 * np.pi / M)
    a = np.array([np.asarray(x, float) for x in expansion.projections(ux, uy, T)])
    assert np.allclose(a, a_num, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("state", STATES)
def test_appendix_c_equals_expansion(state):
    n, ux, uy, T = state
    q = quadrature.quadrature()
    f_sum = lbm.equilibrium(np.float64(n), np.float64(ux), np.float64(uy), np.float64(T))
    f_c = expansion.feq_appendix_c(q["w"], q["P0"], q["PX"], q["PY"], n, ux, uy, T)
    assert np.allclose(f_sum, f_c, rtol=1e-12, atol=1e-15)


@pytest.mark.parametrize("state", STATES)
def test_equilibrium_moments_up_to_third_order(state):
    n, ux, uy, T = state
    q = quadrature.quadrature()
    f = lbm.equilibrium(np.float64(n), np.float64(ux), np.float64(uy), np.float64(T))
    P = np.array([q["P0"], q["PX"], q["PY"]])
    U = U_of(ux, uy)
    eps, pr = 2 * n * T, n * T
    N = P @ f
    T2 = np.einsum("ai,bi,i->ab", P, P, f)
    T3 = np.einsum("ai,bi,ci,i->abc", P, P, P, f)
    N_E = n * U
    T_E = (eps + pr) * np.outer(U, U) - pr * ETA
    T3_E = (n / T) * T**3 * (15 * np.einsum("a,b,c->abc", U, U, U)
                             - 3 * (np.einsum("ab,c->abc", ETA, U) + np.einsum("ac,b->abc", ETA, U)
                                    + np.einsum("bc,a->abc", ETA, U)))
    assert np.allclose(N, N_E, rtol=1e-13, atol=1e-14)
    assert np.allclose(T2, T_E, rtol=1e-13, atol=1e-14)
    assert np.allclose(T3, T3_E, rtol=1e-12, atol=1e-13)


def test_rest_equilibrium_is_the_weights():
    q = quadrature.quadrature()
    f = lbm.equilibrium(np.float64(1.0), np.float64(0.0), np.float64(0.0), np.float64(1.0))
    assert np.allclose(f, q["w"], rtol=1e-15, atol=0)
    d = lbm.equilibrium_deviation(np.float64(1.0), np.float64(0.0), np.float64(0.0), np.float64(1.0))
    assert np.all(d == 0.0)


@pytest.mark.parametrize("state", STATES)
def test_deviation_form_matches_full_form(state):
    n, ux, uy, T = (np.float64(x) for x in state)
    q = quadrature.quadrature()
    d = lbm.equilibrium_deviation(n, ux, uy, T)
    f = lbm.equilibrium(n, ux, uy, T)
    assert np.allclose(d + q["w"], f, rtol=1e-14, atol=1e-17)


def test_small_velocity_deviation_is_odd_and_accurate():
    """For |u| = 1e-7 the deviation's odd part (which carries the flux) is
    exactly linear in u to rounding: no O(1) cancellation remains."""
    q = quadrature.quadrature()
    d1 = lbm.equilibrium_deviation(np.float64(1.0), np.float64(1e-7), np.float64(0.0), np.float64(1.0))
    d2 = lbm.equilibrium_deviation(np.float64(1.0), np.float64(2e-7), np.float64(0.0), np.float64(1.0))
    Nx1 = np.sum(d1 * q["PX"])
    Nx2 = np.sum(d2 * q["PX"])
    assert abs(Nx1 - 1e-7) < 1e-20 + 1e-13 * 1e-7
    assert abs(Nx2 / Nx1 - 2.0) < 1e-12


def _appendix_b_mp(ux, uy, T, mp):
    """Literal App. B in 50-digit arithmetic (reference for the near-rest form)."""
    ux, uy, T = mp.mpf(ux), mp.mpf(uy), mp.mpf(T)
    g = 1 / mp.sqrt(1 - ux * ux - uy * uy)
    u0, uX, uY = g, g * ux, g * uy
    s3, s15, s32, s52 = mp.sqrt(3), mp.sqrt(15), mp.sqrt(mp.mpf(3) / 2), mp.sqrt(mp.mpf(5) / 2)
    Tu = T * u0 - 1
    return [
        mp.mpf(1), Tu, T * uX, T * uY,
        T**2 * (3 * u0**2 - 1) / 2 - 2 * T * u0 + 1,
        s3 * T * uX * Tu, s3 * T * uY * Tu,
        -s3 * T**2 * (u0**2 - 2 * uX**2 - 1) / 2,
        s3 * T**2 * uX * uY,
        Tu * (T**2 * (5 * u0**2 - 3) - 4 * T * u0 + 2) / 2,
        T * uX * (T**2 * (5 * uX**2 + 3) - 6 * T * u0 + 3) / 2,
        -s15 * T * uX * (T**2 * (-2 * u0**2 + uX**2 + 1) + 2 * T * u0 - 1) / 2,
        -s15 * T**2 * Tu * (u0**2 - 2 * uX**2 - 1) / 2,
        s32 * T * uY * (T**2 * (5 * u0**2 - 1) - 8 * T * u0 + 4) / 2,
        -s52 * T**3 * uY * (u0**2 - 4 * uX**2 - 1) / 2,
        s15 * T**2 * uX * uY * Tu,
    ]


@pytest.mark.parametrize("state", [(3e-7, -2e-7, 5e-8), (1e-4, 2e-5, -3e-6), (0.02, -0.01, 0.003),
                                   (0.3, 0.1, 0.2)])
def test_near_rest_projections_equal_appendix_b_in_high_precision(state):
    """The rearranged App. B used by the oracle equals the literal App. B
    evaluated in 50-digit arithmetic, coefficient by coefficient, to full
    double relative precision even where the literal double evaluation
    cancels catastrophically."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    ux, uy, dT = state
    ref = _appendix_b_mp(ux, uy, mp.mpf(1) + mp.mpf(dT), mp)
    got = expansion.projections_near_rest(np.float64(ux), np.float64(uy), np.float64(dT))
    for k in range(16):
        r = float(ref[k])
        assert abs(float(got[k]) - r) <= 1e-13 * abs(r) + 1e-300, (k, float(got[k]), r)


def test_landau_recovers_small_deviations_to_full_precision():
    rng = np.random.default_rng(9)
    shape = (100,)
    dn = rng.uniform(-1e-9, 1e-9, shape)
    dT = rng.uniform(-1e-9, 1e-9, shape)
    ux = rng.uniform(-1e-6, 1e-6, shape)
    uy = rng.uniform(-1e-6, 1e-6, shape)
    d = lbm.equilibrium_deviation(1.0 + dn, ux, uy, 1.0 + dT, dn=dn, dT=dT)
    dn2, ux2, uy2, dT2, _ = lbm.landau_dev(*lbm.moments(d))
    assert np.abs(dn2 - dn).max() < 1e-12 * np.abs(dn).max()
    assert np.abs(dT2 - dT).max() < 1e-12 * np.abs(dT).max()
    assert np.abs(ux2 - ux).max() < 1e-12 * np.abs(ux).max()
    assert np.abs(uy2 - uy).max() < 1e-12 * np.abs(uy).max()
