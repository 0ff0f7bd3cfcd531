"""FP64 CPU oracle of the parallel iDMRG (Hida's iDMRG with wavefunction prediction).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or call
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it.

* ``oracle.idmrg`` -- the algorithm of Sec. 2 (Steps 1-7) with the parallel
  replacements of Sec. 3 (Steps 2', 3', 5'), written plainly with dense numpy
  arrays in float64.  U(1) charges are carried as labels on every basis state
  and used only where the method needs charge-definite bases (the SVD of
  Step 4); the arithmetic is the plain dense definition.
* ``oracle.ed`` -- exact diagonalisation of open clusters straight from a bond
  list, and the free-fermion energies of XX chains.  It shares nothing with
  ``oracle.idmrg`` and pins it.
* ``oracle.observables`` -- the uniform MPS of Eq. mps2 built from a
  converged state, its transfer matrix (dense, ``numpy.linalg.eig``), bond
  strengths, spin-spin correlations, Delta+- (Eqs. diff1, diff2) and the
  correlation length.
* ``oracle.extrapolate`` -- the m scan of Sec. 4.4: runs to convergence and the
  quadratic eps -> 0 fit.
* ``oracle.rng`` -- the counter-based generator (SplitMix64) of the Lanczos
  start vectors for n = 1, 2.

Parity status of each function is stated in its docstring; every function
listed here is pinned by a ``-m "not gpu"`` test against exact
diagonalisation, a closed form, a dense textbook construction or an invariant.
"""
