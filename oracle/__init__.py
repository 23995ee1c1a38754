"""CPU oracle for the LREI hot path -- TEST INFRASTRUCTURE ONLY.

Plain, slow, FP64 NumPy/SciPy restatements of what the paper's method
computes.  Only the test-suite, the package smoke check and the timed CPU
baseline of the benchmark may import this package; the product path never
does, and this package never imports the product.

Modules:
  model     -- dense spin operators and the spin Hamiltonian (Sec. 3.6, eq. H1)
  dense_ei  -- the dense eigenmode-integration (EI) scheme: q-LL / q-LLG
               right-hand sides, the spectrum projection, EI-RK and EI-AB
               (Sec. 2, eqs. eigendecom .. x_ell_sol; Sec. 3.7-3.8)
  lowrank   -- the plain low-rank LREI scheme as the paper states it:
               Householder reflectors for the complement (Sec. 3.4), the
               Z/W right-hand side (Sec. 3.5, eq. q-LLG-low-rank), stage
               matrices in factored form (eqs. K-expand, rho-expand) and an
               ARPACK partial eigensolver on the operator g (eq. g-func)
  exact     -- closed-form references: rank-one pure-state solution
               (eq. exact_q-LL, corrected reading) and the kappa=0 unitary flow
  reduced   -- two-spin reduced density matrices R_kl (partial trace and the
               paper's 16-expectation route) with concurrence and negativity
               (Sec. 3.6)
  werner    -- Werner-state initial data through the shifted low-rank
               problem kappa -> (1-p) kappa (Sec. 5, eq. werner-sol)
  mlp       -- FP64 reference of the step-controller network (forward,
               backward, Adam) used to check the GPU training kernels

Every function cites the passage it follows.
"""
