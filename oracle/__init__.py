"""Plain, slow FP64 CPU oracle of one ADER-DG + a-posteriori subcell-limiter step.

TEST INFRASTRUCTURE ONLY.  This package is the independent checker of the CUDA
library: only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import it.  The product path never calls into it, and it
shares no code, tables or helpers with the CUDA library.

It follows Dumbser, Zanotti, Loubere, Diot, "A posteriori subcell limiting of
the discontinuous Galerkin finite element method for hyperbolic conservation
laws" (arXiv 1406.7416):

  basis.py     Sec. 2.1 / 2.2 Gauss-Legendre nodal basis, space-time operators
  euler.py     Sec. 5 Euler flux and ideal-gas EOS; Rusanov flux of Sec. 2.3
  dg.py        Sec. 2.2 Eq. (pde.nc.dg2) predictor, Sec. 2.3 Eq. (pde.nc.gw2)
               corrector, Sec. 2.4 Eq. (cfl) time step
  subcell.py   Sec. 4.2 Eqs. (subcell.p), (subcell.r), (subcell.r.constraint)
  detect.py    Sec. 4.3 Eqs. (positivity), (dmp), (relax)
  weno.py      Sec. 4.3 Eq. (aderweno): third-order subcell ADER-WENO FV
  step.py      Sec. 4.4 five-act step with the neighbour flux correction
  problems.py  Sec. 5 initial data (explosion, quadrant Riemann data, vortex)
  ic.py        Sec. 4.4 L2 projection of the initial data and its detection

Array conventions: a DG field on a d-dimensional grid has shape
``(nvar, n_1, ..., n_d, n, ..., n)`` -- variable first, then the cell index per
axis (x first), then one nodal index per axis (x first).  A space-time field
appends the time-node axis last.  Everything is float64.

Functions whose parity is not pinned against something other than themselves
say so in their docstring ("parity unpinned").
"""
