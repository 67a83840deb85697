"""Plain FP64 CPU oracle for the generalized-polynomial lattice Boltzmann
method (Coelho, Ilha, Doria, arXiv:1510.07328).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py``'s ``cpu_baseline`` and ``--impl reference`` legs may import or run
anything here.  The CUDA library never calls it and this package imports
nothing from the library; the two share no code, tables or constants.  Inputs
that both sides consume come from ``paper_1510_07328_gb300.inputs``, which
holds only seeded random draws and field shapes, none of the method.

Modules:
  fd      complete Fermi-Dirac integrals, J_2(x), J_4(x), t <-> x
  gpoly   moments I_2N, polynomial coefficients, P_0..P_4, A_0..A_3,
          quadrature weights, tensor-contraction equilibrium
  lbm     lattice state, pull streaming with bounce-back, moments, bisection
          FD inversion, BGK step (d2v9)
  lbm1d   the d1v3 lattice with the zero-temperature and Maxwell-Boltzmann
          closures
  porous  rigid obstacles (halfway bounce-back) and a constant body force
          (exact difference method)
  riemann exact isothermal Riemann solution (the Fig. 1 comparison)
  mlp     the learned inversion's features, targets, forward pass and gradient
"""
