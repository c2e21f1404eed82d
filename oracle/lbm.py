"""Oracle: the (2+1)-D relativistic lattice Boltzmann step for a massless fluid.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain FP64 numpy,
vectorised over sites, no blocking or fusion beyond what the method states.

Per time step and site (the per-site algorithm that closes Sec. 2, kept in
the source as a commented-out subsection, and Eq. discrete-rbe):
  1. pull-stream: f_i(x, t+1) = f*_i(x - n_i, t), with the boundary rules below;
  2. moments N^a = sum_i f_i p_i^a, T^ab = sum_i f_i p_i^a p_i^b;
  3. Landau frame: eps U^a = T^ab U_b gives eps and U = gamma (1, u);
  4. n = U_a N^a;
  5. massless equation of state eps = 2 P = 2 n T, so T = eps / (2 n);
  6. f_i^eq = w_i (n/T) sum_k a^(k)(U, T) J^(k)(p_i)   (Eq. feq-expansion-discrete);
  7. forcing term F_i^ext (Sec. 2.4, reading below);
  8. f*_i = f_i - (p_i^m U_m / (p_i^0 tau)) (f_i - f_i^eq) + F_i^ext.

Storage reading: the state holds deviations delta_i = f_i - w_i from the rest
equilibrium (n = T = 1, u = 0, where f^eq_i = w_i exactly).  This is the same
arithmetic as storing f, except that moment sums over small deviations do not
round against the O(1) rest values:
  * N = (1, 0, 0) + sum_i delta_i p_i and T = diag(2, 1, 1) + sum_i delta_i p_i p_i,
    the rest values being the equilibrium moments n U and (eps + P) U U - P eta
    at n = T = 1, u = 0, which the quadrature reproduces exactly;
  * f^eq_i - w_i = w_i [ (n/T) (Q_i - 1) + (n - T) / T ], Q_i = sum_k a^(k) J^(k)(p_i),
    with Q_i - 1 summed over k >= 1 (a^(0) J^(0) = 1).

Readings of points the paper leaves open (each also listed in the design notes):
  * Units: dt = 1, a hop is 5 sites, so c = 5 sites per step.
  * Relaxation sign: relax towards f^eq as in Eq. discrete-rbe.
  * Equation of state: massless, eps = 2 n T.
  * Eigenvalue: the timelike eigenvector (largest eigenvalue) of T^a_b,
    found by Newton's method on eps - E + M.u(eps) = 0 with
    u(eps) = (Pi + eps I)^-1 M, E = T^00, M = T^0i, Pi = T^ij, from eps0 = E.
  * Forcing: force F per particle, on-shell kinetic equation
    d_t f + v.grad f + F.grad_p f = C; with f ~ f^eq = omega (n/T) Q the
    source is S_i = w_i (n/T) [ (F.v_i)(Q_i - dQ/dp0) - F.grad_xy Q ] evaluated
    at p_i (grad_p omega = -omega v for omega ~ exp(-p0)).  It is added after
    relaxation, computed from the same (pre-force) n, u, T.
  * Walls: a pull whose source lies outside the rectangle (and not in a
    contact strip) takes the post-collision population of the opposite
    direction, same shell, at the destination site (on-site bounce-back).
  * Contacts: a strip 5 sites deep outside the edge, over the contact span,
    whose populations are fixed at the equilibrium of (n_c, u_n * inward
    normal, T_c); a pull from the strip takes that value.  A contact wins
    over the wall.
  * Initial state: the stored post-collision state at t = 0 is f^eq of the
    initial fields; step 1 starts with streaming.
  * Macroscopic fields at time t are the moments of the streamed populations
    at t (the values the next collision uses).
  * Electric force, local capacitance approximation (Sec. 3, Eq. lca):
    phi = -e n / C_g.  Reading: the force pushes electrons away from high
    density (like charges repel), F_E = -(e^2 / C_g) grad n per particle; the
    printed E = -rho_e grad phi, taken literally with e > 0, would point the
    other way.  e = 1, and inv_cg = e^2 / C_g.  The gradient is taken over
    one hop (5 sites, the length unit of c = 1) of the density of the
    previous time step: (n(x + 5) - n(x - 5)) / 2 where both exist, the
    forward or backward difference over 5 sites next to a walled edge,
    wrapped on periodic axes; at the first step the initial density field.
    (A difference over neighbouring sites couples to density structure finer
    than a hop, which the lattice does not resolve, and grows site-scale noise
    beyond e^2 / C_g of about 0.12; with the hop-scale difference the lagged
    force is stable to about 0.3 at tau = 0.8, measured.  The paper's
    C_g = 10 is e^2 / C_g = 0.1.)  F_E adds to the uniform force F of the
    sample.
"""
from __future__ import annotations

import numpy as np

from . import expansion, quadrature

N_REST = np.array([1.0, 0.0, 0.0])
T_REST = np.diag([2.0, 1.0, 1.0])


class Tables:
    """Per-population constants derived from the refined quadrature."""

    def __init__(self):
        q = quadrature.quadrature()
        self.w = q["w"]
        self.P = np.array([q["P0"], q["PX"], q["PY"]])             # p_i^a, [3, 48]
        self.v = self.P[1:] / self.P[0]                              # unit velocities, [2, 48]
        J = expansion.polynomials(self.P[0], self.P[1], self.P[2])
        self.J = np.array(J)                                         # [16, 48]
        grads = expansion.polynomial_gradients(self.P[0], self.P[1], self.P[2])
        self.dJ = np.array([[np.broadcast_to(g[c], (quadrature.Q,)) for g in grads]
                            for c in range(3)])                     # [3, 16, 48]
        d = np.repeat(np.arange(quadrature.NDIR), quadrature.NSHELL)
        j = np.tile(np.arange(quadrature.NSHELL), quadrature.NDIR)
        self.opposite = quadrature.NSHELL * quadrature.OPPOSITE_DIR[d] + j
        self.hop = quadrature.HOPS[d]                                # [48, 2]


_TABLES = None


def tables() -> Tables:
    global _TABLES
    if _TABLES is None:
        _TABLES = Tables()
    return _TABLES


# ---------------------------------------------------------------------------
# Local (per-site) operations; fields have any trailing shape.
# ---------------------------------------------------------------------------

def _contract(M, v):
    """sum_i M[..., i] v[i, ...]: a per-site sum over the last index of the
    constant table M (numpy.einsum without contraction-path optimisation).
    Unlike a BLAS matrix product, whose blocking may depend on the number of
    sites, it gives every site the same result whatever the shape of the
    array the site sits in (the slab-decomposition test relies on that)."""
    lead = "abcdefgh"[:M.ndim - 1]
    return np.einsum(f"{lead}i,i...->{lead}...", M, v, optimize=False)


def moments(delta):
    """Deviations of N^a and T^ab from their rest values: (dN [3,...], dT [3,3,...])."""
    t = tables()
    dN = _contract(t.P, delta)
    PP = t.P[:, None, :] * t.P[None, :, :]
    dT = _contract(PP, delta)
    return dN, dT


def landau(dN, dT, max_iter=60):
    """Solve eps U^a = T^ab U_b; returns (n, ux, uy, T, eps).

    Works on the deviations from rest: eps = 2 + deps with Newton on deps,
    n - 1 and T - 1 formed without subtracting O(1) numbers, so fields near
    rest keep full relative precision in their deviations (see landau_dev).
    """
    dn, ux, uy, dTT, deps = landau_dev(dN, dT, max_iter)
    return 1.0 + dn, ux, uy, 1.0 + dTT, 2.0 + deps


def landau_dev(dN, dT, max_iter=60):
    """Landau frame in deviation variables: returns (n - 1, ux, uy, T - 1, eps - 2).

    E = T^00 = 2 + dE, M = T^0i, Pi = T^ij = I + dPi (rest values diag(2, 1, 1)).
    u(eps) = (Pi + eps I)^-1 M, g(eps) = eps - E + M.u(eps), g'(eps) = 1 - u.u,
    Newton from eps0 = E.  Then n = U_a N^a = gamma (N^0 - u.N) and the
    massless equation of state gives T = eps / (2 n).
    """
    dE = dT[0, 0]
    Mx, My = dT[0, 1], dT[0, 2]
    dPxx, Pxy, dPyy = dT[1, 1], dT[1, 2], dT[2, 2]

    def velocity(deps):
        a, c = 3.0 + dPxx + deps, 3.0 + dPyy + deps      # Pi + eps I, eps = 2 + deps
        det = a * c - Pxy * Pxy
        return (c * Mx - Pxy * My) / det, (a * My - Pxy * Mx) / det

    deps = np.array(dE, dtype=np.float64, copy=True)
    for _ in range(max_iter):
        ux, uy = velocity(deps)
        g = deps - dE + Mx * ux + My * uy
        step = g / (1.0 - ux * ux - uy * uy)
        deps = deps - step
        if np.all(np.abs(step) <= 1e-17 * (2.0 + np.abs(deps))):
            break
    ux, uy = velocity(deps)
    u2 = ux * ux + uy * uy
    s = np.sqrt(1.0 - u2)
    gm1 = u2 / (s * (1.0 + s))                      # gamma - 1
    dpar = dN[0] - ux * dN[1] - uy * dN[2]          # N^0 - u.N - 1
    dn = gm1 * (1.0 + dpar) + dpar                  # n - 1 = gamma (1 + dpar) - 1
    dTT = (deps - 2.0 * dn) / (2.0 * (1.0 + dn))     # T - 1 = eps / (2 n) - 1
    return dn, ux, uy, dTT, deps


def equilibrium_deviation(n, ux, uy, T, dn=None, dT=None):
    """f^eq_i - w_i for the fields (n, u, T); returns [48, ...].

    dn = n - 1 and dT = T - 1 may be given for full relative precision of
    deviations near rest (otherwise they are formed from n and T)."""
    t = tables()
    if dn is None:
        dn = n - 1.0
    if dT is None:
        dT = T - 1.0
    a = np.array(expansion.projections_near_rest(ux, uy, dT))       # [16, ...]
    Qm1 = _contract(t.J[1:].T, a[1:])                              # sum_{k>=1} a_k J_k(p_i)
    nT = (1.0 + dn) / (1.0 + dT)
    return t.w.reshape((-1,) + (1,) * np.ndim(dn)) * (nT * Qm1 + (dn - dT) / (1.0 + dT))


def equilibrium(n, ux, uy, T):
    """Full f^eq_i = w_i (n/T) sum_k a^(k) J^(k)(p_i) (Eq. feq-expansion-discrete)."""
    t = tables()
    a = np.array(expansion.projections(ux, uy, T))
    Qf = _contract(t.J.T, a)
    return t.w.reshape((-1,) + (1,) * np.ndim(n)) * (n / T) * Qf


def forcing(n, ux, uy, T, Fx, Fy):
    """F_i^ext for a force F per particle and dt = 1; returns [48, ...]."""
    t = tables()
    a = np.array(expansion.projections(ux, uy, T))
    ex = (1,) * np.ndim(n)
    Q = _contract(t.J.T, a)
    dQ0 = _contract(t.dJ[0].T, a)
    dQx = _contract(t.dJ[1].T, a)
    dQy = _contract(t.dJ[2].T, a)
    Fv = Fx * t.v[0].reshape((-1,) + ex) + Fy * t.v[1].reshape((-1,) + ex)
    return t.w.reshape((-1,) + ex) * (n / T) * (Fv * (Q - dQ0) - (Fx * dQx + Fy * dQy))


def collide(delta, tau, Fx=0.0, Fy=0.0, return_dn=False):
    """Relaxation + forcing of Eq. discrete-rbe on streamed deviations [48, ...].
    Fx, Fy: force per particle, scalars or per-site arrays.  With return_dn,
    also returns n - 1 of the streamed populations."""
    t = tables()
    dN, dT = moments(delta)
    dn, ux, uy, dTT, _ = landau_dev(dN, dT)
    n, T = 1.0 + dn, 1.0 + dTT
    deq = equilibrium_deviation(n, ux, uy, T, dn=dn, dT=dTT)
    ex = (1,) * np.ndim(n)
    gamma = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy)
    # p_i^m U_m / (p_i^0 tau), U_m = gamma (1, -u) (indices lowered with eta)
    pU = gamma * (t.P[0].reshape((-1,) + ex) - t.P[1].reshape((-1,) + ex) * ux
                  - t.P[2].reshape((-1,) + ex) * uy)
    omega = pU / (t.P[0].reshape((-1,) + ex) * tau)
    out = delta - omega * (delta - deq)
    if np.any(np.asarray(Fx) != 0.0) or np.any(np.asarray(Fy) != 0.0):
        out = out + forcing(n, ux, uy, T, Fx, Fy)
    return (out, dn) if return_dn else out


# ---------------------------------------------------------------------------
# Geometry and streaming
# ---------------------------------------------------------------------------

class Lattice:
    """Rectangle [0, nx) x [0, ny), periodic or walled per axis, plus contacts.

    `sample` is any object with nx, ny, periodic_x, periodic_y, tau, Fx, Fy
    and a list `contacts` of objects with edge, x0, length, u_n, n, T.
    """

    def __init__(self, sample):
        self.nx, self.ny = int(sample.nx), int(sample.ny)
        self.px, self.py = bool(sample.periodic_x), bool(sample.periodic_y)
        self.tau = float(sample.tau)
        self.Fx, self.Fy = float(sample.Fx), float(sample.Fy)
        self.inv_cg = float(getattr(sample, "inv_cg", 0.0))   # e^2 / C_g; 0: no electric force
        self.contacts = list(sample.contacts)
        for c in self.contacts:
            if c.edge in (0, 1) and self.py or c.edge in (2, 3) and self.px:
                raise ValueError("contact on a periodic edge")
        self._build_pull_tables()

    def contact_deviation(self, c):
        normal = {0: (0.0, 1.0), 1: (0.0, -1.0), 2: (1.0, 0.0), 3: (-1.0, 0.0)}[c.edge]
        ux, uy = c.u_n * normal[0], c.u_n * normal[1]
        return equilibrium_deviation(np.float64(c.n), np.float64(ux), np.float64(uy),
                                     np.float64(c.T))

    def _contact_of(self, sx, sy):
        """Index of the contact whose ghost strip holds (sx, sy), else -1."""
        owner = np.full(sx.shape, -1, dtype=np.int64)
        for k, c in enumerate(self.contacts):
            lo, hi = c.x0, c.x0 + c.length
            if c.edge == 0:
                m = (sy < 0) & (sx >= lo) & (sx < hi)
            elif c.edge == 1:
                m = (sy >= self.ny) & (sx >= lo) & (sx < hi)
            elif c.edge == 2:
                m = (sx < 0) & (sy >= lo) & (sy < hi)
            else:
                m = (sx >= self.nx) & (sy >= lo) & (sy < hi)
            owner = np.where((owner < 0) & m, k, owner)
        return owner

    def _build_pull_tables(self):
        t = tables()
        Y, X = np.meshgrid(np.arange(self.ny), np.arange(self.nx), indexing="ij")
        self.pull = []
        for i in range(quadrature.Q):
            dx, dy = t.hop[i]
            sx, sy = X - dx, Y - dy
            if self.px:
                sx = np.mod(sx, self.nx)
            if self.py:
                sy = np.mod(sy, self.ny)
            inside = (sx >= 0) & (sx < self.nx) & (sy >= 0) & (sy < self.ny)
            owner = np.where(inside, -1, self._contact_of(sx, sy))
            wall = ~inside & (owner < 0)
            self.pull.append((inside, np.clip(sx, 0, self.nx - 1),
                              np.clip(sy, 0, self.ny - 1), owner, wall))
        self.ghost = np.array([self.contact_deviation(c) for c in self.contacts]) \
            if self.contacts else np.zeros((0, quadrature.Q))

    def grad(self, a):
        """(d/dx, d/dy) of a site field [ny, nx] over one hop (5 sites = the
        length unit of c = 1): central differences over +-5 sites, forward /
        backward over 5 sites next to a walled edge, wrapped on periodic axes."""
        h = 5

        def d(axis, periodic):
            m = a.shape[axis]
            if periodic:
                return (np.roll(a, -h, axis) - np.roll(a, h, axis)) / 2.0
            g = np.empty_like(a)
            sl = lambda i: tuple(slice(None) if k != axis else i for k in range(2))
            g[sl(slice(h, m - h))] = (a[sl(slice(2 * h, m))] - a[sl(slice(0, m - 2 * h))]) / 2.0
            g[sl(slice(0, h))] = a[sl(slice(h, 2 * h))] - a[sl(slice(0, h))]
            g[sl(slice(m - h, m))] = a[sl(slice(m - h, m))] - a[sl(slice(m - 2 * h, m - h))]
            return g
        return d(1, self.px), d(0, self.py)

    def electric_force(self, dn_prev):
        """F_E = -(e^2 / C_g) grad n per particle from the previous step's n - 1."""
        gx, gy = self.grad(dn_prev)
        return -self.inv_cg * gx, -self.inv_cg * gy

    def stream(self, post):
        """Pull-streaming with periodic wrap, contacts and bounce-back walls."""
        t = tables()
        out = np.empty_like(post)
        for i in range(quadrature.Q):
            inside, sx, sy, owner, wall = self.pull[i]
            v = post[i][sy, sx]
            if len(self.contacts):
                v = np.where(owner >= 0, self.ghost[np.maximum(owner, 0), i], v)
            v = np.where(wall, post[t.opposite[i]], v)
            out[i] = v
        return out


# ---------------------------------------------------------------------------
# Driver
# ---------------------------------------------------------------------------

def init(lat: Lattice, n, ux, uy, T):
    """Post-collision state at t = 0: f^eq of the initial fields (deviations)."""
    n, ux, uy, T = (np.asarray(a, np.float64) for a in (n, ux, uy, T))
    return equilibrium_deviation(n, ux, uy, T, dn=n - 1.0, dT=T - 1.0)


def relaxation_rates(ux, uy, tau):
    """omega_i = p_i^m U_m / (p_i^0 tau) = gamma (1 - v_i.u) / tau per
    population and site (Eq. discrete-rbe); returns [48, ...]."""
    t = tables()
    ex = (1,) * np.ndim(ux)
    gamma = 1.0 / np.sqrt(1.0 - ux * ux - uy * uy)
    vu = t.v[0].reshape((-1,) + ex) * ux + t.v[1].reshape((-1,) + ex) * uy
    return gamma * (1.0 - vu) / tau


def chapman_enskog_init(lat: Lattice, n, ux, uy, T):
    """Post-collision state at t = 0 that streams to f^eq plus its first-order
    Chapman-Enskog part (a seed for steady flows; the paper gives no seed, this
    is the reading used for warm starts).

    Steady BGK, Eq. discrete-rbe, with f = f^eq + f^neq and f^neq small and
    slowly varying gives f^neq_i(x) = -(f^eq_i(x) - f^eq_i(x - n_i)) / omega_i(x):
    the streaming derivative of the equilibrium over one hop, divided by the
    relaxation rate at the site where the population arrives.  So the stored
    value at a source site s, whose population i arrives at d = s + n_i
    (wrapped on periodic axes), is
        f*_i(s) = f^eq_i(d) - (f^eq_i(d) - f^eq_i(s)) / omega_i(d),
    and f*_i(s) = f^eq_i(s) where d lies outside the sample (such a population
    is only read by the bounce-back at s).  Deviations f - w, [48, ny, nx]."""
    n, ux, uy, T = (np.asarray(a, np.float64) for a in (n, ux, uy, T))
    t = tables()
    eq = init(lat, n, ux, uy, T)
    om = relaxation_rates(ux, uy, lat.tau)
    out = eq.copy()
    Y, X = np.meshgrid(np.arange(lat.ny), np.arange(lat.nx), indexing="ij")
    for i in range(quadrature.Q):
        dx, dy = t.hop[i]
        tx, ty = X + dx, Y + dy
        if lat.px:
            tx = np.mod(tx, lat.nx)
        if lat.py:
            ty = np.mod(ty, lat.ny)
        inside = (tx >= 0) & (tx < lat.nx) & (ty >= 0) & (ty < lat.ny)
        tx, ty = np.clip(tx, 0, lat.nx - 1), np.clip(ty, 0, lat.ny - 1)
        ed = eq[i][ty, tx]
        seed = ed - (ed - eq[i]) / om[i][ty, tx]
        out[i] = np.where(inside, seed, eq[i])
    return out


def step(lat: Lattice, post):
    """One time step: stream then collide.  Returns the new post-collision state."""
    if lat.inv_cg != 0.0:
        raise ValueError("a sample with an electric force steps with step_lca")
    return collide(lat.stream(post), lat.tau, lat.Fx, lat.Fy)


def run(lat: Lattice, post, nsteps):
    for _ in range(nsteps):
        post = step(lat, post)
    return post


def step_lca(lat: Lattice, post, dn_prev):
    """One time step with the electric force of the local capacitance
    approximation: F = (Fx, Fy) + F_E(grad of the previous step's density).
    Returns (post-collision state, n - 1 of this step)."""
    ex, ey = lat.electric_force(dn_prev)
    return collide(lat.stream(post), lat.tau, lat.Fx + ex, lat.Fy + ey, return_dn=True)


def run_lca(lat: Lattice, post, dn_prev, nsteps):
    for _ in range(nsteps):
        post, dn_prev = step_lca(lat, post, dn_prev)
    return post, dn_prev


def macroscopic(lat: Lattice, post):
    """(n, ux, uy, T) at the current time: moments of the streamed populations."""
    dN, dT = moments(lat.stream(post))
    dn, ux, uy, dTT, _ = landau_dev(dN, dT)
    return 1.0 + dn, ux, uy, 1.0 + dTT


def residual(u_prev, u_now):
    """r = ||u(t) - u(t-1)||_2 / ||u(t)||_2 over all sites (the paper defines no
    convergence measure; this is the reading used throughout)."""
    dx = u_now[0] - u_prev[0]
    dy = u_now[1] - u_prev[1]
    num = np.sqrt(np.sum(dx * dx + dy * dy))
    den = np.sqrt(np.sum(u_now[0] ** 2 + u_now[1] ** 2))
    return num / den if den > 0 else (0.0 if num == 0 else np.inf)
