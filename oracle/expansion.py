"""Oracle: the third-order polynomial expansion of the massless 2-D
Maxwell-Juttner equilibrium (App. A, App. B, App. C; Eq. feq-expansion).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow FP64 CPU restatement
of the paper used to check the CUDA path; only tests/, __graft_entry__.smoke()
and bench.py's CPU-baseline / reference arm may import it.  It shares no code
with the CUDA path.

Conventions: momenta p = (p0, px, py) with c = k_B = 1 and metric
eta = diag(1, -1, -1) (Sec. 2.1).  Polynomials are orthonormal under the rest
frame weight omega(p0) = exp(-p0) / (2 pi) at the reference temperature T0 = 1
with measure d^2p / p0 (Eq. mj-poly-weighting-factor).

Index order of the 16 polynomials / projections (App. A and App. B order):
    0: J0      1: J1_0    2: J1_x    3: J1_y
    4: J2_00   5: J2_0x   6: J2_0y   7: J2_xx   8: J2_xy
    9: J3_000 10: J3_xxx 11: J3_00x 12: J3_0xx 13: J3_00y 14: J3_xxy 15: J3_0xy
"""
from __future__ import annotations

import numpy as np

NPOLY = 16
NAMES = ["J0", "J1_0", "J1_x", "J1_y", "J2_00", "J2_0x", "J2_0y", "J2_xx", "J2_xy",
         "J3_000", "J3_xxx", "J3_00x", "J3_0xx", "J3_00y", "J3_xxy", "J3_0xy"]

S3 = np.sqrt(3.0)
S15 = np.sqrt(15.0)
S53 = np.sqrt(5.0 / 3.0)
S6 = np.sqrt(6.0)
S23 = np.sqrt(2.0 / 3.0)
S25 = np.sqrt(2.0 / 5.0)
S10 = np.sqrt(10.0)
S32 = np.sqrt(3.0 / 2.0)
S52 = np.sqrt(5.0 / 2.0)


def polynomials(p0, px, py):
    """The 16 orthonormal polynomials J^(k)(p) of App. A (m = 0, order <= 3).

    Arguments may be arrays (real or complex); returns a list of 16 arrays.
    """
    one = np.ones_like(p0)
    return [
        one,                                                        # J0
        p0 - 1.0,                                                   # J1_0
        px * one,                                                   # J1_x
        py * one,                                                   # J1_y
        0.5 * p0**2 - 2.0 * p0 + 1.0,                               # J2_00
        p0 * px / S3 - S3 * px,                                     # J2_0x
        p0 * py / S3 - S3 * py,                                     # J2_0y
        px**2 / S3 - p0**2 / (2.0 * S3),                            # J2_xx
        px * py / S3,                                               # J2_xy
        p0**3 / 6.0 - 1.5 * p0**2 + 3.0 * p0 - 1.0,                 # J3_000
        -p0 * px + px**3 / 6.0 + 1.5 * px,                          # J3_xxx
        p0**2 * px / S15 - S53 * p0 * px - px**3 / (2.0 * S15) + 0.5 * S15 * px,   # J3_00x
        -p0**3 / (2.0 * S15) + 0.5 * S53 * p0**2 + p0 * px**2 / S15 - S53 * px**2,  # J3_0xx
        p0**2 * py / (2.0 * S6) - 2.0 * S23 * p0 * py + S6 * py,   # J3_00y
        S25 / 3.0 * px**2 * py - p0**2 * py / (6.0 * S10),          # J3_xxy
        p0 * px * py / S15 - S53 * px * py,                         # J3_0xy
    ]


def polynomial_gradients(p0, px, py):
    """Partial derivatives (d/dp0, d/dpx, d/dpy) of each App. A polynomial,
    with p0, px, py taken as independent variables.  Returns 16 triples."""
    z = np.zeros_like(p0)
    one = np.ones_like(p0)
    return [
        (z, z, z),
        (one, z, z),
        (z, one, z),
        (z, z, one),
        (p0 - 2.0, z, z),
        (px / S3, p0 / S3 - S3, z),
        (py / S3, z, p0 / S3 - S3),
        (-p0 / S3, 2.0 * px / S3, z),
        (z, py / S3, px / S3),
        (0.5 * p0**2 - 3.0 * p0 + 3.0, z, z),
        (-px, -p0 + 0.5 * px**2 + 1.5, z),
        (2.0 * p0 * px / S15 - S53 * px,
         p0**2 / S15 - S53 * p0 - 1.5 * px**2 / S15 + 0.5 * S15, z),
        (-1.5 * p0**2 / S15 + S53 * p0 + px**2 / S15,
         2.0 * p0 * px / S15 - 2.0 * S53 * px, z),
        (p0 * py / S6 - 2.0 * S23 * py, z,
         p0**2 / (2.0 * S6) - 2.0 * S23 * p0 + S6),
        (-p0 * py / (3.0 * S10), 2.0 * S25 / 3.0 * px * py,
         S25 / 3.0 * px**2 - p0**2 / (6.0 * S10)),
        (px * py / S15, p0 * py / S15 - S53 * py, p0 * px / S15 - S53 * px),
    ]


def projections(ux, uy, T):
    """The 16 projection coefficients a^(k)(U, T) of App. B.

    u^0, u^x, u^y in App. B are the components of the (2+1)-velocity
    U = gamma (1, u) (reading: App. C reproduces N_E = n U only with this
    choice).  The coefficients are those of the equilibrium divided by n/T,
    so a^(0) = 1.
    """
    g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy)
    u0, uX, uY = g, g * ux, g * uy
    Tu = T * u0 - 1.0
    return [
        np.ones_like(T),
        Tu,
        T * uX,
        T * uY,
        0.5 * T**2 * (3.0 * u0**2 - 1.0) - 2.0 * T * u0 + 1.0,
        S3 * T * uX * Tu,
        S3 * T * uY * Tu,
        -0.5 * S3 * T**2 * (u0**2 - 2.0 * uX**2 - 1.0),
        S3 * T**2 * uX * uY,
        0.5 * Tu * (T**2 * (5.0 * u0**2 - 3.0) - 4.0 * T * u0 + 2.0),
        0.5 * T * uX * (T**2 * (5.0 * uX**2 + 3.0) - 6.0 * T * u0 + 3.0),
        -0.5 * S15 * T * uX * (T**2 * (-2.0 * u0**2 + uX**2 + 1.0) + 2.0 * T * u0 - 1.0),
        -0.5 * S15 * T**2 * Tu * (u0**2 - 2.0 * uX**2 - 1.0),
        0.5 * S32 * T * uY * (T**2 * (5.0 * u0**2 - 1.0) - 8.0 * T * u0 + 4.0),
        -0.5 * S52 * T**3 * uY * (u0**2 - 4.0 * uX**2 - 1.0),
        S15 * T**2 * uX * uY * Tu,
    ]


def projections_near_rest(ux, uy, dT):
    """App. B rewritten for numerical accuracy near the rest state.

    Identical algebra to projections(), with every coefficient expressed
    through quantities that vanish at rest (n = T = 1, u = 0):
        Tu = T u^0 - 1 = (T - 1) gamma + (gamma - 1),  gamma - 1 = u^2 / (s (1 + s)),
        s = sqrt(1 - u^2),  T^2 - 1 = (T - 1)(T + 1),  (u^0)^2 - 1 = gamma^2 u^2,
    and combinations such as Tu - (T^2 - 1)/2 = (gamma - 1) T - (T - 1)^2 / 2
    written without the cancelling first-order parts, so that small
    coefficients keep full relative precision instead of rounding against
    O(1) terms.  dT is T - 1.
    """
    u2 = ux * ux + uy * uy
    s = np.sqrt(1.0 - u2)
    g = 1.0 / s
    gm1 = u2 / (s * (1.0 + s))
    T = 1.0 + dT
    uX, uY = g * ux, g * uy
    Tu = dT * g + gm1
    g2 = g * g
    xx = g2 * (uy * uy - ux * ux)            # (u^0)^2 - 2 (u^x)^2 - 1
    xxy = g2 * (uy * uy - 3.0 * ux * ux)     # (u^0)^2 - 4 (u^x)^2 - 1
    return [
        np.ones_like(T),
        Tu,
        T * uX,
        T * uY,
        1.5 * Tu * Tu + gm1 * T - 0.5 * dT * dT,
        S3 * T * uX * Tu,
        S3 * T * uY * Tu,
        -0.5 * S3 * T**2 * xx,
        S3 * T**2 * uX * uY,
        0.5 * Tu * (5.0 * Tu * Tu + 6.0 * gm1 * T - 3.0 * dT * dT),
        0.5 * T * uX * (5.0 * T**2 * uX * uX + 3.0 * dT * dT - 6.0 * gm1 * T),
        -0.5 * S15 * T * uX * (-2.0 * Tu * Tu + T**2 * uX * uX + dT * dT - 2.0 * gm1 * T),
        -0.5 * S15 * T**2 * Tu * xx,
        0.5 * S32 * T * uY * (5.0 * Tu * Tu + 2.0 * gm1 * T - dT * dT),
        -0.5 * S52 * T**3 * uY * xxy,
        S15 * T**2 * uX * uY * Tu,
    ]


def feq_appendix_c(w, p0, px, py, n, ux, uy, T):
    """The fully expanded discrete equilibrium printed in App. C (m = 0, N = 3).

    Used only as an independent cross-check of w (n/T) sum_k a^(k) J^(k).
    """
    g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy)
    u0, uX, uY = g, g * ux, g * uy
    Tu = T * u0 - 1.0
    t = (
        T**3 * uX * (px**3 - 0.75 * p0**2 * px) * (-3.0 * u0**2 + 4.0 * uX**2 + 3.0) / 6.0
        + py * T**3 * uY * (p0**2 - 4.0 * px**2) * (u0**2 - 4.0 * uX**2 - 1.0) / 24.0
        + 0.25 * T**2 * (p0**2 - 2.0 * px**2) * (u0**2 - 2.0 * uX**2 - 1.0)
        + (-2.0 * p0**2 + (p0 - 5.0) * px**2 + 9.0 * p0 - 3.0) * Tu
        * (T * (5.0 * T * uX**2 + T - 2.0 * u0) + 1.0) / 8.0
        + (4.0 * p0**3 - 30.0 * p0**2 - 3.0 * (p0 - 5.0) * px**2 + 45.0 * p0 - 15.0) * Tu
        * (T**2 * (4.0 * u0**2 - 3.0 * (uX**2 + 1.0)) - 2.0 * T * u0 + 1.0) / 24.0
        + (p0 - 5.0) * px * py * T**2 * uX * uY * Tu
        + (p0 - 6.0) * (p0 - 2.0) * px * T * uX * (T**2 * (5.0 * u0**2 - 1.0) - 8.0 * T * u0 + 4.0) / 8.0
        + (p0 - 3.0) * px * T * uX * Tu
        + (p0 - 6.0) * (p0 - 2.0) * py * T * uY * (T**2 * (5.0 * u0**2 - 1.0) - 8.0 * T * u0 + 4.0) / 8.0
        + (p0 - 3.0) * py * T * uY * Tu
        + 0.25 * ((p0 - 4.0) * p0 + 2.0) * (T**2 * (3.0 * u0**2 - 1.0) - 4.0 * T * u0 + 2.0)
        + (p0 - 1.0) * Tu
        + px * py * T**2 * uX * uY
        + px * T * uX
        + py * T * uY
        + 1.0
    )
    return w * n / T * t
