"""CPU oracle for the three-region FEM-BEM nonlinear Poisson-Boltzmann Newton solve.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, float64 restatement
of the method of Guerrero-Montero, Bosy and Cooper, "A Self-Adjusting FEM-BEM
Coupling Scheme for the Nonlinear Poisson-Boltzmann Equation" (arXiv
2511.21713).  Only the test-suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it.  The CUDA library never calls
into it and shares no code, tables or constants with it; the only module both
sides use is the seeded input generator ``paper_2511_21713_gb300.inputs``.

Modules:
  quadrature  -- 14-point tetrahedron, 6-point triangle, Gauss-Legendre and
                 Sauter-Schwab rules (Sec. 3 "fourth-order Gaussian quadrature").
  fem         -- P1 stiffness, nonlinear load N(u), Jacobian J(u), second
                 directional derivative, the Omega_i energy integral.
  bem         -- dense Galerkin Laplace/Yukawa single- and double-layer
                 matrices, surface mass matrices, the Coulomb right-hand side.
  pb          -- the coupled block operator (Eq. fembem_matrix in its
                 three-region form), GMRES, the Newton-Raphson loop with the
                 optimal relaxation factor (Eqs. NR_main, Ec_NL_NR, fd=0,
                 Appendix A), and the solvation energy (Eqs. Esolv,
                 Potential_in_Omega_m).
  solute      -- the paper's own formulation: FEM over Omega_m and Omega_i
                 with the charges as point loads, Yukawa BEM on Gamma_s
                 (Eq. fembem_matrix), and the reaction potential from the
                 Gamma_m boundary integral equation (Sec. 2.3.1).

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, a library routine used as an independent check, an invariant or
brute force; no function here is "parity unpinned".
"""
