"""Seeded synthetic workloads: sample geometries and initial fields.

This module only describes inputs (domain sizes, boundary kinds, contact
spans, relaxation time, body force, initial macroscopic fields).  It holds
none of the method's arithmetic, so both the CUDA path and the CPU oracle
may take their inputs from it.

Lattice conventions used by every workload:
  * sites are indexed (x, y), 0 <= x < nx, 0 <= y < ny, stored row-major
    as [ny][nx];
  * one time step is dt = 1 and a hop of the stencil is 5 sites, so the
    speed of light is c = 5 sites per step (Sec. 2.3, massless shells);
  * a body force (Fx, Fy) is the momentum given to one particle per step.

Contacts (injector / collector, Sec. 3, Fig. geom caption) sit on one edge of
the rectangle.  edge = 0 is the y = 0 edge, 1 the y = ny-1 edge, 2 the x = 0
edge and 3 the x = nx-1 edge; the contact covers `length` sites starting at
`x0` along that edge.  Its sites never evolve: they hold the equilibrium of
(n, u_n * inward normal, T).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import List

import numpy as np

EDGE_Y0, EDGE_Y1, EDGE_X0, EDGE_X1 = 0, 1, 2, 3
MAX_CONTACTS = 4
HOP_RADIUS = 5


@dataclass
class Contact:
    edge: int
    x0: int
    length: int
    u_n: float = 0.0
    n: float = 1.0
    T: float = 1.0


@dataclass
class Sample:
    nx: int
    ny: int
    periodic_x: bool = False
    periodic_y: bool = False
    tau: float = 1.0
    Fx: float = 0.0
    Fy: float = 0.0
    contacts: List[Contact] = field(default_factory=list)
    # electric force of the local capacitance approximation: e^2 / C_g (0: none)
    inv_cg: float = 0.0

    @property
    def sites(self) -> int:
        return self.nx * self.ny


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def shear_wave(n: int = 64, tau: float = 0.8) -> Sample:
    """Doubly periodic n x n box for the transverse shear wave."""
    return Sample(nx=n, ny=n, periodic_x=True, periodic_y=True, tau=tau)


def shear_wave_fields(s: Sample, amplitude: float = 0.01):
    """n = T = 1 everywhere, u_x = amplitude * sin(2 pi y / ny), u_y = 0."""
    y = np.arange(s.ny, dtype=np.float64)
    ux = np.repeat((amplitude * np.sin(2.0 * math.pi * y / s.ny))[:, None], s.nx, axis=1)
    n = np.ones((s.ny, s.nx))
    return n, ux, np.zeros_like(ux), np.ones_like(n)


def graphene_sample(nx: int = 1024, ny: int = 512, contact_width: int = 32,
                    contact_spacing: int = 256, force: float = 1e-6,
                    tau: float = 1.0, u_in: float = 0.0) -> Sample:
    """Rectangle with no-slip walls and two contacts on the y = 0 long edge.

    The contacts are `contact_width` sites wide with centres `contact_spacing`
    apart, placed symmetrically about the middle of the edge.  The uniform
    body force points along the edge from the injector (left) to the
    collector (right).  `u_in` is the inward normal velocity held at the
    injector; the collector holds -u_in (outflow).
    """
    c0 = nx // 2 - contact_spacing // 2
    c1 = nx // 2 + contact_spacing // 2
    half = contact_width // 2
    contacts = [Contact(EDGE_Y0, c0 - half, contact_width, u_n=u_in),
                Contact(EDGE_Y0, c1 - half, contact_width, u_n=-u_in)]
    return Sample(nx=nx, ny=ny, tau=tau, Fx=force, Fy=0.0, contacts=contacts)


def rest_fields(s: Sample, n0: float = 1.0, T0: float = 1.0):
    n = np.full((s.ny, s.nx), n0)
    return n, np.zeros_like(n), np.zeros_like(n), np.full_like(n, T0)


def random_fields(s: Sample, seed: int, du: float = 0.05, dn: float = 0.05, dT: float = 0.05):
    """Smooth-free random perturbation around n = T = 1, u = 0 (seeded)."""
    rng = np.random.default_rng(seed)
    shape = (s.ny, s.nx)
    n = 1.0 + dn * rng.uniform(-1, 1, shape)
    T = 1.0 + dT * rng.uniform(-1, 1, shape)
    ux = du * rng.uniform(-1, 1, shape)
    uy = du * rng.uniform(-1, 1, shape)
    return n, ux, uy, T


def ensemble(count: int = 256, seed0: int = 1234, w_lo: int = 128, w_hi: int = 1024,
             max_aspect: float = 4.0) -> List[Sample]:
    """Uneven graphene-like samples, one seeded generator per sample.

    Short side W ~ U[w_lo, w_hi], long side L = round(a W) with a ~ U[1, max_aspect],
    tau ~ U[0.6, 2.0], contact width ~ U{8..64}, |F| ~ logU[1e-7, 1e-5].
    The contacts sit on the long (x) edge at y = 0, centres L/4 apart.
    """
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        W = int(rng.integers(w_lo, w_hi + 1))
        a = float(rng.uniform(1.0, max_aspect))
        L = max(W, int(round(a * W)))
        tau = float(rng.uniform(0.6, 2.0))
        cw = int(rng.integers(8, 65))
        F = float(10.0 ** rng.uniform(-7.0, -5.0))
        spacing = max(cw + 2 * HOP_RADIUS, L // 4)
        # narrow samples with wide contacts: move the contacts closer until
        # both lie on the edge (the contacts of every other sample are as drawn)
        while spacing > cw and (L // 2 - spacing // 2 - cw // 2 < 0 or
                                L // 2 + spacing // 2 - cw // 2 + cw > L):
            spacing -= 1
        s = graphene_sample(nx=L, ny=W, contact_width=cw, contact_spacing=spacing,
                            force=F, tau=tau)
        out.append(s)
    return out
