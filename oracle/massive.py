"""Oracle: the massive-particle variant of the method, rest mass m = 5 T0
(Sec. 2.3: Eq. discrete-quadri-momentum, Eq. discrete-p0, Eq. orthonormal,
Fig. m5-stencil; Sec. 2.2: Eq. feq-expansion-discrete, Eq. discrete-rbe).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy over
sites; the quadrature is solved in 60-digit decimal arithmetic.  Shares no
code with the CUDA path.

Units: T0 = 1 (the reference temperature of the weight function), so the
rest mass is m = 5; dt = 1; a population with stencil vector n_i moves n_i
sites per step with velocity v_i = v0 n_i, so one site is v0 length units.

Stencil (Fig. m5-stencil): G = {(0,0), (1,0)_FS, (1,1)_FS, (2,0)_FS, (2,1)_FS,
(2,2)_FS, (3,0)_FS, (3,2)_FS, (3,3)_FS, (4,0)_FS}, 45 vectors, FS = all sign
changes and the swap of the two components.  Population order: the 44 moving
vectors class by class in the order above, opposite vectors adjacent (the
opposite of i < 44 is i ^ 1), then the rest vector at i = 44.  Within a class
(a, 0): (a,0) (-a,0) (0,a) (0,-a); (a, a): (a,a) (-a,-a) (-a,a) (a,-a);
(a, b), 0 < b < a: (a,b) (-a,-b) (-a,b) (a,-b) (b,a) (-b,-a) (-b,a) (b,-a).

Discrete momenta (Eq. discrete-quadri-momentum, Eq. discrete-p0):
    p_i = p0_i (1, v0 n_i),   p0_i = m gamma_i = m / sqrt(1 - v0^2 |n_i|^2).

Weight function: the Maxwell-Juttner distribution at rest at T0,
    omega(p0) = exp(-(p0 - m)) / (2 pi),   int omega d^2p / p0 = 1,
where on the mass shell d^2p / p0 = dp0 dtheta (p0 from m to infinity).

Quadrature conditions.  Eq. orthonormal for every pair of polynomials of
degree <= 3 in p holds exactly when the quadrature integrates every product
of two of them, i.e. every monomial p0^a px^b py^c of degree <= 6, exactly.
On the mass shell p0^2 = m^2 + px^2 + py^2 (the nodes lie on it), so a <= 1
suffices; the stencil is symmetric under the 8 reflections of the square, so
odd b or c vanish on both sides and b, c may be swapped.  That leaves ten
conditions (a, b, c) = (0,0,0) (0,2,0) (0,4,0) (0,2,2) (0,6,0) (0,4,2)
(1,0,0) (1,2,0) (1,4,0) (1,2,2), linear in the ten class weights; their
right-hand sides are rational (closed forms below).

Reading (v0): the paper leaves v0 free (|v_i| <= 1, i.e. v0 <= 1/sqrt(18))
and asks for non-negative weights but gives no v0.  For each v0 the ten
conditions fix the ten weights; all ten are non-negative only on one narrow
interval of v0 (near 0.2211, about 1.4e-5 wide; w_(1,0) >= 0 sets its lower
end, w_(1,1) >= 0 its upper end).  The oracle takes v0 = the midpoint of that
interval, rounded to FP64, and the weights and p0 at that v0 from the
decimal solve, rounded to FP64.

Polynomials J^(k): Gram-Schmidt of the 16 monomials listed in MONOMIALS
(a basis of the polynomials of degree <= 3 on the mass shell), in that order,
under <f, g> = int omega f g d^2p / p0 (exact rational Gram matrix).

Equilibrium (Eq. feq-expansion-discrete):
    f^eq_i = w_i sum_k a^(k) J^(k)(p_i),   a^(k) = int f_MJ J^(k) d^2p / p0,
    f_MJ = A exp(-p.U / T),   A = n / (2 pi T (m + T) exp(-m/T))  (N = n U).
The moments of f_MJ are those of its rest frame, boosted by U.  Precision:
the Gram-Schmidt coefficients reach 170 and the nodes' monomials 3e3, so the
moments enter the projection as deviations from their rest values, formed in
numpy longdouble, and J^(k)(p_i) is tabulated from the 60-digit solve; f^eq
is then within ~4e-14 of a 40-digit evaluation (FP64 throughout would leave
~1e-12).

Equation of state (2-D massive ideal gas; the same rest integrals):
    P = n T,   eps = n (m^2 + 2 m T + 2 T^2) / (m + T),
so T follows from eps / n by the root of 2T^2 + (2m - e)T + m^2 - e m = 0.

Collision (Eq. discrete-rbe), Landau frame as in the massless case:
  eps U^a = T^ab U_b (timelike eigenvector), n = U_a N^a, T from the EOS;
  f*_i = f_i - (p_i.U / (p0_i tau)) (f_i - f^eq_i) + F_i^ext.
Forcing (reading, as for the massless stencil): force F per particle,
    F_i^ext = -F.grad_p (omega P)|_{p_i} / omega * w_i
            = w_i [ (F.v_i) P(p_i) - F.grad_p P(p_i) ],
P = sum_k a^(k) J^(k), grad_p along the mass shell (grad_p p0 = v), from the
pre-force n, u, T.
Walls: on-site bounce-back (a pull from outside the rectangle takes the
post-collision opposite population of the destination site).
"""
from __future__ import annotations

import decimal
from fractions import Fraction
from functools import lru_cache
from math import comb, factorial

import numpy as np

MASS = 5
Q = 45
CLASSES = [(1, 0), (1, 1), (2, 0), (2, 1), (2, 2), (3, 0), (3, 2), (3, 3), (4, 0), (0, 0)]

# monomials p0^a px^b py^c spanning degree <= 3 on the mass shell (a <= 1)
MONOMIALS = [(0, 0, 0),
             (1, 0, 0), (0, 1, 0), (0, 0, 1),
             (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1), (0, 0, 2),
             (1, 2, 0), (1, 1, 1), (1, 0, 2), (0, 3, 0), (0, 2, 1), (0, 1, 2), (0, 0, 3)]

CONDITIONS = [(0, 0, 0), (0, 2, 0), (0, 4, 0), (0, 2, 2), (0, 6, 0), (0, 4, 2),
              (1, 0, 0), (1, 2, 0), (1, 4, 0), (1, 2, 2)]


def class_vectors(c):
    a, b = c
    if a == 0:
        return [(0, 0)]
    if b == 0:
        return [(a, 0), (-a, 0), (0, a), (0, -a)]
    if a == b:
        return [(a, a), (-a, -a), (-a, a), (a, -a)]
    return [(a, b), (-a, -b), (-a, b), (a, -b), (b, a), (-b, -a), (-b, a), (b, -a)]


def stencil():
    """(45, 2) integer vectors n_i, (45,) class index, (45,) opposite index."""
    vec, cls = [], []
    for k, c in enumerate(CLASSES):
        for v in class_vectors(c):
            vec.append(v)
            cls.append(k)
    vec = np.array(vec, dtype=np.int64)
    opp = np.array([i ^ 1 for i in range(Q - 1)] + [Q - 1])
    return vec, np.array(cls), opp


# ---------------------------------------------------------------------------
# Rest-frame integrals (closed forms)
# ---------------------------------------------------------------------------
def _dfact(k):
    """(k)!! for k >= -1."""
    r = 1
    while k > 1:
        r *= k
        k -= 2
    return r


def angular_fraction(b, c):
    """(1 / 2 pi) int_0^{2 pi} cos^b sin^c dtheta (0 unless b, c even)."""
    if b % 2 or c % 2:
        return Fraction(0)
    return Fraction(_dfact(b - 1) * _dfact(c - 1), _dfact(b + c))


def shell_power_integral(k, T=Fraction(1), m=MASS):
    """exp(m/T) int_m^inf exp(-p0/T) p0^k dp0 = T sum_j C(k,j) j! m^(k-j) T^j."""
    return T * sum(comb(k, j) * factorial(j) * m ** (k - j) * T ** j for j in range(k + 1))


def omega_moment(a, b, c):
    """int omega p0^a px^b py^c d^2p / p0 (exact rational), omega at T0 = 1:
    (1 / 2 pi) int_m^inf exp(-(p0 - m)) p0^a |p|^(b+c) dp0 int cos^b sin^c,
    with |p|^2 = p0^2 - m^2."""
    ang = angular_fraction(b, c)
    if ang == 0:
        return Fraction(0)
    h = (b + c) // 2
    rad = sum(comb(h, l) * (-MASS * MASS) ** (h - l) * shell_power_integral(a + 2 * l)
              for l in range(h + 1))
    return rad * ang


# ---------------------------------------------------------------------------
# Quadrature (Sec. 2.3)
# ---------------------------------------------------------------------------
def _solve_decimal(A, b):
    """Gaussian elimination with partial pivoting (lists of Decimal)."""
    n = len(b)
    A = [row[:] for row in A]
    b = b[:]
    for col in range(n):
        piv = max(range(col, n), key=lambda r: abs(A[r][col]))
        A[col], A[piv] = A[piv], A[col]
        b[col], b[piv] = b[piv], b[col]
        for r in range(col + 1, n):
            f = A[r][col] / A[col][col]
            for k in range(col, n):
                A[r][k] -= f * A[col][k]
            b[r] -= f * b[col]
    x = [None] * n
    for r in range(n - 1, -1, -1):
        s = b[r] - sum(A[r][k] * x[k] for k in range(r + 1, n))
        x[r] = s / A[r][r]
    return x


def _pw(x, k):
    """x^k for a Decimal (0^0 = 1)."""
    return x ** k if k else decimal.Decimal(1)


def _ctx():
    return decimal.Context(prec=60)


def class_weights(v0):
    """The ten class weights fixed by the ten conditions at a given v0
    (Decimal or float), as Decimals, and the ten class energies p0."""
    with decimal.localcontext(_ctx()):
        D = decimal.Decimal
        v0 = D(v0)
        m = D(MASS)
        rhs = [D(omega_moment(*c).numerator) / D(omega_moment(*c).denominator) for c in CONDITIONS]
        A = [[D(0)] * len(CLASSES) for _ in CONDITIONS]
        p0c = []
        for k, c in enumerate(CLASSES):
            n2 = c[0] ** 2 + c[1] ** 2
            p0 = m / (D(1) - v0 * v0 * n2).sqrt()
            p0c.append(p0)
            for (nx, ny) in class_vectors(c):
                px, py = p0 * v0 * nx, p0 * v0 * ny
                for r, (a, b, cc) in enumerate(CONDITIONS):
                    A[r][k] += _pw(p0, a) * _pw(px, b) * _pw(py, cc)
        return _solve_decimal(A, rhs), p0c


def _nonneg(v0):
    w, _ = class_weights(v0)
    return min(w) >= 0


def _window_float():
    """Coarse scan (FP64 solves, step 1e-6) for the interval of v0 where all
    ten weights are non-negative; returns grid points bracketing its ends."""
    vec, cls, _ = stencil()
    rhs = np.array([float(omega_moment(*c)) for c in CONDITIONS])
    vmax = 1.0 / np.sqrt(18.0)
    grid = np.arange(0.01, vmax, 1e-6)
    ok = np.zeros(len(grid), bool)
    for s in range(0, len(grid), 20000):
        v0 = grid[s:s + 20000]
        A = np.zeros((len(v0), len(CONDITIONS), len(CLASSES)))
        for (nx, ny), k in zip(vec, cls):
            vx, vy = v0 * nx, v0 * ny
            p0 = MASS / np.sqrt(1.0 - vx * vx - vy * vy)
            px, py = p0 * vx, p0 * vy
            for r, (a, b, c) in enumerate(CONDITIONS):
                A[:, r, k] += p0 ** a * px ** b * py ** c
        w = np.linalg.solve(A, np.broadcast_to(rhs, (len(v0), len(rhs)))[..., None])[..., 0]
        ok[s:s + 20000] = (w >= 0).all(axis=1)
    idx = np.flatnonzero(ok)
    if len(idx) == 0:
        raise RuntimeError("no v0 with non-negative weights")
    lo, hi = idx[0], idx[-1]
    if np.any(~ok[lo:hi + 1]):
        raise RuntimeError("the non-negative window is not one interval")
    return (grid[lo - 1], grid[lo]), (grid[hi], grid[hi + 1])


def _bisect(bad, good, iters=90):
    with decimal.localcontext(_ctx()):
        D = decimal.Decimal
        bad, good = D(bad), D(good)
        for _ in range(iters):
            mid = (bad + good) / 2
            if _nonneg(mid):
                good = mid
            else:
                bad = mid
        return (bad + good) / 2


@lru_cache(maxsize=None)
def quadrature():
    """dict: v0, the interval ends, class weights / energies, and per
    population n (45, 2), class, opp, w (45,), p (45, 3) = (p0, px, py)."""
    (lo_bad, lo_good), (hi_good, hi_bad) = _window_float()
    with decimal.localcontext(_ctx()):
        lo = _bisect(lo_bad, lo_good)
        hi = _bisect(hi_bad, hi_good)
        v0 = float((lo + hi) / 2)
        wd, p0d = class_weights(v0)
        wc = np.array([float(x) for x in wd])
        p0c = np.array([float(x) for x in p0d])
        vec, cls, opp = stencil()
        D = decimal.Decimal
        p = np.zeros((Q, 3))
        for i, ((nx, ny), k) in enumerate(zip(vec, cls)):
            p[i, 0] = p0c[k]
            p[i, 1] = float(p0d[k] * D(v0) * nx)
            p[i, 2] = float(p0d[k] * D(v0) * ny)
    return {"v0": v0, "window": (float(lo), float(hi)), "w_class": wc, "p0_class": p0c,
            "n": vec, "cls": cls, "opp": opp, "w": wc[cls], "p": p}


# ---------------------------------------------------------------------------
# Orthonormal polynomials (Eq. orthonormal) by Gram-Schmidt
# ---------------------------------------------------------------------------
def monomial_values(p):
    """(16, ...) values of MONOMIALS at momenta p = (p0, px, py) (leading axis 3)."""
    return np.array([p[0] ** a * p[1] ** b * p[2] ** c for (a, b, c) in MONOMIALS])


def _gram_schmidt_decimal(G):
    """Lower-triangular C = L^-1 with G = L L^T (Decimal, current context)."""
    n = len(G)
    D = decimal.Decimal
    Gd = [[D(g.numerator) / D(g.denominator) for g in row] for row in G]
    L = [[D(0)] * n for _ in range(n)]
    for i in range(n):
        for j in range(i + 1):
            s = Gd[i][j] - sum(L[i][k] * L[j][k] for k in range(j))
            L[i][j] = s.sqrt() if i == j else s / L[j][j]
    C = [[D(0)] * n for _ in range(n)]
    for col in range(n):
        for i in range(n):
            s = (D(1) if i == col else D(0)) - sum(L[i][k] * C[k][col] for k in range(i))
            C[i][col] = s / L[i][i]
    return C


@lru_cache(maxsize=None)
def polynomials():
    """(16, 16) lower-triangular C with J^(k) = sum_b C[k, b] MONOMIALS[b]:
    Gram-Schmidt (Cholesky of the exact Gram matrix, in 60 digits)."""
    G = [[omega_moment(a1 + a2, b1 + b2, c1 + c2) for (a2, b2, c2) in MONOMIALS]
         for (a1, b1, c1) in MONOMIALS]
    with decimal.localcontext(_ctx()):
        return np.array([[float(x) for x in row] for row in _gram_schmidt_decimal(G)])


# ---------------------------------------------------------------------------
# Maxwell-Juttner moments, equation of state
# ---------------------------------------------------------------------------
def eos_energy(n, T):
    return n * (MASS ** 2 + 2 * MASS * T + 2 * T * T) / (MASS + T)


def temperature(n, eps):
    e = eps / n
    return (e - 2 * MASS + np.sqrt(e * e + 4 * e * MASS - 4 * MASS * MASS)) / 4


def _rest_tensor(order, n, T):
    """Rest-frame moments int f_MJ p^a1 .. p^a_order d^2p/p0 of f_MJ(n, T) as
    an array of shape (3,)*order + T.shape (components 0, x, y)."""
    T = np.asarray(T, np.longdouble)
    n = np.asarray(n, np.longdouble)
    m = MASS
    A = n / (2 * np.pi * T * (m + T))                  # A exp(-m/T), the exp cancels
    out = np.zeros((3,) * order + T.shape, np.longdouble)
    for idx in np.ndindex(*((3,) * order)):
        a = idx.count(0)
        b = idx.count(1)
        c = idx.count(2)
        ang = angular_fraction(b, c)
        if ang == 0:
            continue
        h = (b + c) // 2
        rad = 0.0
        for l in range(h + 1):
            k = a + 2 * l
            s = T * sum(comb(k, j) * factorial(j) * m ** (k - j) * T ** j for j in range(k + 1))
            rad = rad + comb(h, l) * (-m * m) ** (h - l) * s
        out[idx] = 2 * np.pi * A * rad * (np.longdouble(ang.numerator) / ang.denominator)
    return out


def boost(ux, uy):
    """Lorentz boost Lambda^a_b taking the rest frame to velocity u: (3, 3, ...)."""
    ux = np.asarray(ux, np.longdouble)
    uy = np.asarray(uy, np.longdouble)
    u2 = ux * ux + uy * uy
    g = 1 / np.sqrt(1 - u2)
    k = g * g / (g + 1)                                # (gamma - 1) / u^2
    L = np.empty((3, 3) + ux.shape, np.longdouble)
    L[0, 0] = g
    L[0, 1] = L[1, 0] = g * ux
    L[0, 2] = L[2, 0] = g * uy
    L[1, 1] = 1 + k * ux * ux
    L[2, 2] = 1 + k * uy * uy
    L[1, 2] = L[2, 1] = k * ux * uy
    return L


def mj_monomial_moments(n, ux, uy, T):
    """(16, ...) int f_MJ m_b(p) d^2p/p0 for the MONOMIALS, f_MJ(n, U, T), in
    numpy longdouble: the component of the boosted rest-frame tensor,
        M^{a1..ak} = Lambda^a1_d1 .. Lambda^ak_dk R^{d1..dk}."""
    L = boost(ux, uy)
    R = [_rest_tensor(k, n, T) for k in range(4)]
    out = []
    for (a, b, c) in MONOMIALS:
        idx = (0,) * a + (1,) * b + (2,) * c
        acc = np.zeros_like(R[0])
        for d in np.ndindex(*((3,) * len(idx))):
            if not np.any(R[len(idx)][d]):
                continue
            term = R[len(idx)][d]
            for ai, di in zip(idx, d):
                term = term * L[ai, di]
            acc = acc + term
        out.append(acc)
    return np.array(out)


@lru_cache(maxsize=None)
def _rest_projection_and_nodes():
    """a^(k) at rest (n = T = 1, u = 0) and the table J^(k)(p_i) (16, 45), both
    from the 60-digit Gram-Schmidt, rounded to FP64.  At rest f_MJ = omega / (m + 1)."""
    n = len(MONOMIALS)
    G = [[omega_moment(a1 + a2, b1 + b2, c1 + c2) for (a2, b2, c2) in MONOMIALS]
         for (a1, b1, c1) in MONOMIALS]
    q = quadrature()
    with decimal.localcontext(_ctx()):
        D = decimal.Decimal
        C = _gram_schmidt_decimal(G)
        Mr = [D(omega_moment(*mon).numerator) / D(omega_moment(*mon).denominator) / D(MASS + 1)
              for mon in MONOMIALS]
        a_rest = np.array([float(sum(C[k][b] * Mr[b] for b in range(n))) for k in range(n)])
        v0 = D(q["v0"])
        J = np.zeros((n, Q))
        for i in range(Q):
            k = q["cls"][i]
            n2 = int(q["n"][i, 0]) ** 2 + int(q["n"][i, 1]) ** 2
            p0 = D(MASS) / (D(1) - v0 * v0 * n2).sqrt()
            p = (p0, p0 * v0 * int(q["n"][i, 0]), p0 * v0 * int(q["n"][i, 1]))
            mv = [_pw(p[0], a) * _pw(p[1], b) * _pw(p[2], c) for (a, b, c) in MONOMIALS]
            for kk in range(n):
                J[kk, i] = float(sum(C[kk][b] * mv[b] for b in range(n)))
    return a_rest, J


def projections(n, ux, uy, T):
    """a^(k) = int f_MJ J^(k) d^2p/p0, (16, ...): the rest value (exact) plus
    C times the moments' deviation from rest, taken in longdouble before the
    FP64 product (so the large entries of C never multiply rounded O(1)
    moments)."""
    C = polynomials()
    a_rest, _ = _rest_projection_and_nodes()
    nd = np.ndim(n)
    dM = (mj_monomial_moments(n, ux, uy, T) - _rest_moments().reshape((-1,) + (1,) * nd)).astype(float)
    return a_rest.reshape((-1,) + (1,) * nd) + np.einsum("kb,b...->k...", C, dM)


@lru_cache(maxsize=None)
def _rest_moments():
    one = np.ones(1)
    return mj_monomial_moments(one, 0 * one, 0 * one, one)[:, 0]


def equilibrium(n, ux, uy, T, a=None):
    """f^eq_i (45, ...) (Eq. feq-expansion-discrete); `a` may pass the
    projections already computed for these fields."""
    q = quadrature()
    if a is None:
        a = projections(n, ux, uy, T)
    _, J = _rest_projection_and_nodes()               # (16, 45): J^(k)(p_i)
    return q["w"].reshape((Q,) + (1,) * np.ndim(n)) * np.einsum("ki,k...->i...", J, a)


def rest_populations():
    """f^eq at n = T = 1, u = 0: the reference the library's deviations are taken from."""
    return equilibrium(np.ones(1), np.zeros(1), np.zeros(1), np.ones(1))[:, 0]


# ---------------------------------------------------------------------------
# Moments, Landau frame, collision
# ---------------------------------------------------------------------------
def moments(f):
    """N^a (3, ...) and T^ab (3, 3, ...) of populations f (45, ...)."""
    p = quadrature()["p"]
    N = np.einsum("ia,i...->a...", p, f)
    Tab = np.einsum("ia,ib,i...->ab...", p, p, f)
    return N, Tab


ETA = np.diag([1.0, -1.0, -1.0])


def landau(N, Tab):
    """n, ux, uy, T from N^a, T^ab: eps U^a = T^a_b U^b, the eigenvector of
    the largest eigenvalue (the timelike one), U.U = 1, U^0 > 0."""
    shape = N.shape[1:]
    Tm = np.einsum("ac...,cb->...ab", Tab, ETA).reshape(-1, 3, 3)
    lam, vec = np.linalg.eig(Tm)
    k = np.argmax(lam.real, axis=1)
    eps = lam.real[np.arange(len(k)), k]
    U = vec.real[np.arange(len(k)), :, k]
    U = U / np.sqrt(U[:, 0] ** 2 - U[:, 1] ** 2 - U[:, 2] ** 2)[:, None]
    U = U * np.sign(U[:, 0])[:, None]
    Nf = N.reshape(3, -1)
    n = U[:, 0] * Nf[0] - U[:, 1] * Nf[1] - U[:, 2] * Nf[2]
    T = temperature(n, eps)
    ux, uy = U[:, 1] / U[:, 0], U[:, 2] / U[:, 0]
    return n.reshape(shape), ux.reshape(shape), uy.reshape(shape), T.reshape(shape)


def macroscopic(f):
    return landau(*moments(f))


def force_term(n, ux, uy, T, Fx, Fy, a=None):
    """F_i^ext = w_i [ (F.v_i) P(p_i) - F.grad_p P(p_i) ], (45, ...)."""
    q = quadrature()
    C = polynomials()
    if a is None:
        a = projections(n, ux, uy, T)
    coef = np.einsum("kb,k...->b...", C, a)           # P in MONOMIALS
    p = q["p"].T
    v = p[1:] / p[0]
    d0 = np.zeros((len(MONOMIALS), Q))
    dx = np.zeros_like(d0)
    dy = np.zeros_like(d0)
    for b, (a, bx, by) in enumerate(MONOMIALS):
        if a:
            d0[b] = a * p[0] ** (a - 1) * p[1] ** bx * p[2] ** by
        if bx:
            dx[b] = bx * p[0] ** a * p[1] ** (bx - 1) * p[2] ** by
        if by:
            dy[b] = by * p[0] ** a * p[1] ** bx * p[2] ** (by - 1)
    P = np.einsum("bi,b...->i...", monomial_values(p), coef)
    dP0 = np.einsum("bi,b...->i...", d0, coef)
    gx = np.einsum("bi,b...->i...", dx, coef) + v[0].reshape((Q,) + (1,) * np.ndim(n)) * dP0
    gy = np.einsum("bi,b...->i...", dy, coef) + v[1].reshape((Q,) + (1,) * np.ndim(n)) * dP0
    Fx = np.asarray(Fx, float)
    Fy = np.asarray(Fy, float)
    Fv = Fx * v[0].reshape((Q,) + (1,) * np.ndim(n)) + Fy * v[1].reshape((Q,) + (1,) * np.ndim(n))
    w = q["w"].reshape((Q,) + (1,) * np.ndim(n))
    return w * (Fv * P - Fx * gx - Fy * gy)


def collide(f, tau, Fx=0.0, Fy=0.0):
    """f* = f - (p.U / (p0 tau)) (f - f^eq) + F^ext (Eq. discrete-rbe)."""
    q = quadrature()
    n, ux, uy, T = macroscopic(f)
    a = projections(n, ux, uy, T)
    feq = equilibrium(n, ux, uy, T, a)
    g = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy)
    v = q["p"][:, 1:] / q["p"][:, :1]
    om = g * (1.0 - np.einsum("i,...->i...", v[:, 0], ux) - np.einsum("i,...->i...", v[:, 1], uy)) / tau
    out = f - om * (f - feq)
    if Fx != 0.0 or Fy != 0.0:
        out = out + force_term(n, ux, uy, T, Fx, Fy, a)
    return out


# ---------------------------------------------------------------------------
# Lattice, streaming
# ---------------------------------------------------------------------------
class Lattice:
    def __init__(self, nx, ny, periodic_x=False, periodic_y=False, tau=1.0, Fx=0.0, Fy=0.0):
        self.nx, self.ny = nx, ny
        self.periodic_x, self.periodic_y = periodic_x, periodic_y
        self.tau, self.Fx, self.Fy = tau, Fx, Fy


def stream(lat, post):
    """Pull: f_i(x) = f*_i(x - n_i); periodic axes wrap, a source outside a
    walled axis bounces back: f_i(x) = f*_opp(i)(x)."""
    q = quadrature()
    ny, nx = lat.ny, lat.nx
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    out = np.empty_like(post)
    for i in range(Q):
        sx = x - q["n"][i, 0]
        sy = y - q["n"][i, 1]
        inside = np.ones_like(sx, dtype=bool)
        if lat.periodic_x:
            sx = sx % nx
        else:
            inside &= (sx >= 0) & (sx < nx)
        if lat.periodic_y:
            sy = sy % ny
        else:
            inside &= (sy >= 0) & (sy < ny)
        out[i] = np.where(inside, post[i][np.clip(sy, 0, ny - 1), np.clip(sx, 0, nx - 1)],
                          post[q["opp"][i]])
    return out


def init(lat, n, ux, uy, T):
    """Stored post-collision state at t = 0: f^eq of the fields."""
    return equilibrium(np.asarray(n, float), np.asarray(ux, float),
                       np.asarray(uy, float), np.asarray(T, float))


def step(lat, post):
    return collide(stream(lat, post), lat.tau, lat.Fx, lat.Fy)


def run(lat, post, nsteps):
    for _ in range(nsteps):
        post = step(lat, post)
    return post


def fields(lat, post):
    """n, ux, uy, T at the current time: moments of the streamed populations."""
    return macroscopic(stream(lat, post))
