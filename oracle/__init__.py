"""CPU oracle for the (2+1)-D relativistic lattice Boltzmann method of
Gabbana, Mendoza, Succi, Tripiccione (arXiv:1804.02418).

TEST INFRASTRUCTURE ONLY.  A plain, slow, FP64 numpy restatement of the
paper, written to check the CUDA path.  Only tests/, __graft_entry__.smoke()
and bench.py (its CPU-baseline leg and its reference arm) may import it; the
product library never calls it and shares no code, header, table or constant
generator with it.

Modules:
  expansion   App. A polynomials (and their partial derivatives), App. B
              projections, App. C expanded equilibrium
  quadrature  the 48-velocity massless order-3 stencil of Sec. 2.3, refined
              onto the exact solutions of Eq. orthonormal
  lbm         streaming with walls / contacts / periodic wrap, moments,
              Landau-frame solve, equilibrium, forcing, relaxation (Sec. 2,
              Eq. discrete-rbe, Sec. 3)
  massive     the massive-particle variant (m = 5 T0, the 45-vector stencil
              of Fig. m5-stencil): quadrature solve, Gram-Schmidt
              polynomials, equilibrium, Landau frame with the massive
              equation of state, forcing, walls (Sec. 2.3)

Every function is pinned by tests/test_oracle_*.py against what the paper and
the mathematics fix (continuum integrals, exact rational moment sums, closed
forms, invariants, brute force on tiny grids).  The steady states of the
walled / contact geometries have no closed form: for those only the
invariants and the GPU-vs-oracle comparison apply.
"""
