"""CPU FP64 oracle for the KPM observable engine of the RMFT vortex solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, links or runs
this package: only the tests, the smoke check and the benchmark's CPU-baseline
leg do. It shares no code with the CUDA library; the two meet only through
the seeded input arrays, whose layout both implement independently.

Every routine is written to be read against the paper (arXiv:2212.05685):

  lattice.py  Peierls phases in the Landau gauge A = B(0, x), B = 2 Phi0/(Nx Ny)
              (Sec. II, App. C)
  rmft.py     Gutzwiller factors, the variational energy W and its derivatives,
              the effective fields T, D, eps (App. A, Eqs. Tij, Dij, mu_i)
  bdg.py      the Nambu matrix h_IJ (App. B) as dense and CSR matrices, and the
              spectral bounds used to rescale it
  kpm.py      Jackson damping, Chebyshev coefficients of the T=0 step and of
              the grand-potential function (Eqs. rho_KPM, F_KPM), three routes
              to the density matrix: ED step (O0), spectral KPM (O1) and the
              naive Chebyshev recursion on unit vectors (O2, Eq. alpha)
  kspace.py   the zero-field translation-invariant case in momentum space
  fock.py     many-body brute force on clusters of a few sites
  adjoint.py  reverse-mode gradients of the KPM observables (Eqs. dFdH,
              dalphadH), checked against finite differences and exact
              matrix-function derivatives

Parity status: every function listed above is pinned by tests in tests/
against closed forms, brute force or invariants, except the paper's physics
numbers (vortex size, residual magnetisation), which the oracle does not
claim to reproduce.
"""
