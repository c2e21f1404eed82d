"""Oracle: the minimal massless third-order quadrature (Sec. 2.3, Fig. m0-o3,
Eq. orthonormal, Eq. discrete-quadri-momentum with energy shells).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Shares no code with the
CUDA path.

The stencil is G = {(+-3, +-4)_FS, (+-5, 0)_FS}: 8 vectors of the first kind,
4 of the second, |n| = 5 for all.  Each of the 12 directions carries 4 energy
shells, so there are 48 discrete momenta p_{d,j} = p0_j (1, n_d / 5).

Population index: i = 4 * d + j, with the direction order
    d:  0 (3,4)   1 (-3,-4)   2 (-3,4)   3 (3,-4)
        4 (4,3)   5 (-4,-3)   6 (-4,3)   7 (4,-3)
        8 (5,0)   9 (-5,0)   10 (0,5)   11 (0,-5)
so the opposite direction of d is d ^ 1.  Directions 0..7 carry the weights
w_{1j}, directions 8..11 the weights w_{2j}.

Reading (ambiguity): the printed weights and shells are truncated to 12
digits and only satisfy Eq. orthonormal to about 3e-9, and the conditions
leave a 2-parameter family of exact solutions.  The oracle uses the exact
solution nearest to the printed values: Gauss-Newton steps of minimum
Euclidean norm in the 12 unscaled parameters (w_11..w_14, w_21..w_24,
p0_1..p0_4), applied to the residual G - I of Eq. orthonormal, where G is the
discrete Gram matrix of the 16 App. A polynomials.  Every parameter moves by
less than 1e-11, i.e. below the printed truncation.
"""
from __future__ import annotations

import numpy as np

from . import expansion

HOPS = np.array([(3, 4), (-3, -4), (-3, 4), (3, -4),
                 (4, 3), (-4, -3), (-4, 3), (4, -3),
                 (5, 0), (-5, 0), (0, 5), (0, -5)], dtype=np.int64)
NDIR = 12
NSHELL = 4
Q = NDIR * NSHELL
RADIUS = 5
OPPOSITE_DIR = np.arange(NDIR) ^ 1
DIR_KIND = np.array([0] * 8 + [1] * 4)     # 0: (3,4)-type, 1: (5,0)-type

# Values printed in Sec. 2.3 (12 digits, truncated).
PRINTED_W1 = np.array([0.003930503244, 0.008026424774, 0.000175706060, 0.042659667266])
PRINTED_W2 = np.array([0.054642060984, 0.013535762740, 0.000296310700, 0.071941262878])
PRINTED_P0 = np.array([0.000016359462, 3.305423649330, 7.758786843141, 0.935838587521])


def unit_directions():
    """v_d = n_d / |n_d| (massless shells: |v| = c = 1)."""
    return HOPS.astype(np.float64) / RADIUS


def nodes(w1, w2, p0):
    """Weights w_i and momenta (p0_i, px_i, py_i) of the 48 populations."""
    v = unit_directions()
    w = np.empty(Q, dtype=np.result_type(w1, w2))
    P0 = np.empty(Q, dtype=np.result_type(p0, 1.0))
    PX = np.empty(Q, dtype=P0.dtype)
    PY = np.empty(Q, dtype=P0.dtype)
    for d in range(NDIR):
        for j in range(NSHELL):
            i = NSHELL * d + j
            w[i] = w1[j] if DIR_KIND[d] == 0 else w2[j]
            P0[i] = p0[j]
            PX[i] = p0[j] * v[d, 0]
            PY[i] = p0[j] * v[d, 1]
    return w, P0, PX, PY


def gram(w1, w2, p0):
    """Discrete Gram matrix G_lk = sum_i w_i J_l(p_i) J_k(p_i) (Eq. orthonormal)."""
    w, P0, PX, PY = nodes(w1, w2, p0)
    J = np.array(expansion.polynomials(P0, PX, PY))          # [16, 48]
    return (J * w[None, :]) @ J.T


def _residual(x):
    G = gram(x[0:4], x[4:8], x[8:12])
    iu = np.triu_indices(expansion.NPOLY)
    return (G - np.eye(expansion.NPOLY))[iu]


def _jacobian(x, h=1e-30):
    """d residual / d x by the complex-step derivative (exact to rounding)."""
    cols = []
    for k in range(12):
        xc = x.astype(np.complex128)
        xc[k] += 1j * h
        cols.append(np.imag(_residual(xc)) / h)
    return np.array(cols).T


def refine(w1=PRINTED_W1, w2=PRINTED_W2, p0=PRINTED_P0, iterations=6):
    """Minimum-norm Gauss-Newton projection of the printed values onto the
    exact solutions of Eq. orthonormal.  Returns (w1, w2, p0)."""
    x = np.concatenate([w1, w2, p0]).astype(np.float64)
    for _ in range(iterations):
        r = _residual(x)
        Jm = _jacobian(x)
        dx, *_ = np.linalg.lstsq(Jm, -r, rcond=1e-9)
        x = x + dx
    return x[0:4].copy(), x[4:8].copy(), x[8:12].copy()


_CACHE = {}


def quadrature():
    """The refined quadrature used by the oracle: dict with w1, w2, p0 and the
    48-node arrays w, p0_i, px_i, py_i."""
    if "q" not in _CACHE:
        w1, w2, p0 = refine()
        w, P0, PX, PY = nodes(w1, w2, p0)
        _CACHE["q"] = dict(w1=w1, w2=w2, p0=p0, w=w, P0=P0, PX=PX, PY=PY)
    return _CACHE["q"]
