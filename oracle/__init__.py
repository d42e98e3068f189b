"""CPU oracle for IBSN (arXiv 2603.07156) -- TEST INFRASTRUCTURE ONLY.

A plain, slow, float64 numpy restatement of the paper's method, used to check
the CUDA path.  Only the test-suite, the package smoke check and the CPU
baseline leg of the benchmark may import it; the solver library never does.

It shares no code with the CUDA path: it keeps log X^k explicitly (Alg. 2),
forms H_rho densely (Alg. 1), evaluates L^k directly for Armijo, and rounds
with Alg. 3 literally.

Modules
  ibsn  -- Eqs. 4-7, Alg. 1, Alg. 2, Alg. 3, D_phi, c-transform, Delta_kkt.
  lp    -- exact LP references used to pin the oracle: permutation
           enumeration, a network simplex, the 1-D monotone coupling and the
           separable-cost closed form.

Parity status per function is listed in each module's header.
"""
