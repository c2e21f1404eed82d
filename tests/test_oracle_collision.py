"""Pins for the oracle's Landau solve, relaxation and forcing (CPU only).

Independent references:
  * numpy.linalg.eig of T^a_b (a generic non-symmetric eigen-routine);
  * the round trip f^eq(n, u, T) -> moments -> (n, u, T);
  * the collision invariants of the Anderson-Witting operator in the Landau
    frame: U_m (N^m - N_E^m) = 0 and U_m (T^ma - T_E^ma) = 0, which make
    N^0 and T^0a exact collision invariants;
  * integration by parts of -F.grad_p f: the source changes N^0 by 0,
    T^0i by F^i N^0 and T^00 by F.N (exact for the degree <= 6 quadrature).
"""
import numpy as np
import pytest

from oracle import lbm, quadrature

ETA = np.diag([1.0, -1.0, -1.0])


def random_nonequilibrium(rng, shape, du=0.2, amp=0.02):
    """Equilibrium at random (n, u, T) plus a random non-equilibrium part."""
    n = rng.uniform(0.8, 1.3, shape)
    T = rng.uniform(0.8, 1.3, shape)
    ang = rng.uniform(0, 2 * np.pi, shape)
    mag = rng.uniform(0, du, shape)
    ux, uy = mag * np.cos(ang), mag * np.sin(ang)
    q = quadrature.quadrature()
    d = lbm.equilibrium_deviation(n, ux, uy, T)
    noise = amp * q["w"].reshape((-1,) + (1,) * len(shape)) * rng.standard_normal((48,) + shape)
    return d + noise


def full_moments(delta):
    dN, dT = lbm.moments(delta)
    N = dN + lbm.N_REST.reshape((3,) + (1,) * (dN.ndim - 1))
    T = dT + lbm.T_REST.reshape((3, 3) + (1,) * (dT.ndim - 2))
    return N, T


def test_landau_matches_generic_eigen_routine():
    rng = np.random.default_rng(1)
    delta = random_nonequilibrium(rng, (50,), du=0.5, amp=0.05)
    N, T = full_moments(delta)
    dN, dT = lbm.moments(delta)
    n, ux, uy, Tt, eps = lbm.landau(dN, dT)
    for s in range(50):
        A = T[:, :, s] @ ETA                  # T^a_b acting on U^b
        vals, vecs = np.linalg.eig(A)
        k = int(np.argmax(vals.real))
        U = vecs[:, k].real
        U = U / np.sqrt(U @ ETA @ U) * np.sign(U[0])
        assert abs(vals[k].real - eps[s]) < 1e-13 * abs(eps[s])
        assert abs(U[1] / U[0] - ux[s]) < 1e-13
        assert abs(U[2] / U[0] - uy[s]) < 1e-13
        assert abs(U @ ETA @ N[:, s] - n[s]) < 1e-13 * n[s]


def test_landau_round_trip_of_equilibrium():
    rng = np.random.default_rng(2)
    shape = (200,)
    n = rng.uniform(0.5, 2.0, shape)
    T = rng.uniform(0.5, 2.0, shape)
    ux = rng.uniform(-0.4, 0.4, shape)
    uy = rng.uniform(-0.4, 0.4, shape)
    d = lbm.equilibrium_deviation(n, ux, uy, T)
    n2, ux2, uy2, T2, eps = lbm.landau(*lbm.moments(d))
    assert np.abs(n2 - n).max() < 1e-14 * 4
    assert np.abs(T2 - T).max() < 1e-14 * 4
    assert np.abs(ux2 - ux).max() < 1e-14
    assert np.abs(uy2 - uy).max() < 1e-14
    # massless closed form eps = 2 P = 2 n T
    assert np.allclose(eps, 2 * n * T, rtol=1e-14)


def test_energy_momentum_tensor_is_traceless_for_any_populations():
    rng = np.random.default_rng(3)
    delta = rng.standard_normal((48, 30))
    N, T = full_moments(delta)
    assert np.allclose(T[0, 0], T[1, 1] + T[2, 2], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("tau", [0.6, 1.0, 1.7])
def test_collision_invariants(tau):
    rng = np.random.default_rng(4)
    delta = random_nonequilibrium(rng, (100,))
    post = lbm.collide(delta, tau)
    N0, T0 = full_moments(delta)
    N1, T1 = full_moments(post)
    assert np.abs(N1[0] - N0[0]).max() < 1e-13 * np.abs(N0[0]).max()
    for a in range(3):
        assert np.abs(T1[0, a] - T0[0, a]).max() < 1e-13 * np.abs(T0[0, 0]).max()
    # N^i and T^ij are not invariants of this operator: check they did change
    assert np.abs(N1[1] - N0[1]).max() > 1e-8


def test_landau_matching_conditions():
    rng = np.random.default_rng(5)
    delta = random_nonequilibrium(rng, (60,))
    N, T = full_moments(delta)
    n, ux, uy, Tt, eps = lbm.landau(*lbm.moments(delta))
    Ueq = np.array([1 / np.sqrt(1 - ux**2 - uy**2)] * 3) * np.array([np.ones_like(ux), ux, uy])
    deq = lbm.equilibrium_deviation(n, ux, uy, Tt)
    NE, TE = full_moments(deq)
    Ul = ETA @ Ueq
    assert np.abs(np.einsum("as,as->s", Ul, N - NE)).max() < 1e-13
    assert np.abs(np.einsum("as,abs->bs", Ul, T - TE)).max() < 1e-13


@pytest.mark.parametrize("F", [(1e-3, 0.0), (0.0, -2e-3), (7e-4, 5e-4)])
def test_forcing_moments(F):
    rng = np.random.default_rng(6)
    shape = (40,)
    n = rng.uniform(0.8, 1.3, shape)
    T = rng.uniform(0.8, 1.3, shape)
    ux = rng.uniform(-0.3, 0.3, shape)
    uy = rng.uniform(-0.3, 0.3, shape)
    S = lbm.forcing(n, ux, uy, T, F[0], F[1])
    q = quadrature.quadrature()
    P = np.array([q["P0"], q["PX"], q["PY"]])
    g = 1 / np.sqrt(1 - ux**2 - uy**2)
    NE = n * g * np.array([np.ones_like(ux), ux, uy])            # N_E = n U
    dN0 = P[0] @ S
    dT0 = np.einsum("i,ai,is->as", P[0], P, S)
    assert np.abs(dN0).max() < 1e-16
    assert np.allclose(dT0[1], F[0] * NE[0], rtol=1e-12, atol=1e-18)
    assert np.allclose(dT0[2], F[1] * NE[0], rtol=1e-12, atol=1e-18)
    assert np.allclose(dT0[0], F[0] * NE[1] + F[1] * NE[2], rtol=1e-11, atol=1e-18)
