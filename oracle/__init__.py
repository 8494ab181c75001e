"""FP64 CPU oracle for the full-TDDFT (Tsiper p/q) operator and its preconditioned CG solver.

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports this package: only the tests, the
smoke check of the entry module and the CPU-baseline leg of the benchmark may import or run it.
It shares no code with the CUDA library; both take their inputs from the seeded synthetic
generator and nothing else.

Two levels (all arithmetic in float64, numpy/scipy):

* ``casida`` (O1) -- the plain definition. Kohn-Sham states from the generalised eigenproblems of
  the synthetic Hamiltonians, the coupling matrix K of Sec. II A built from KS products on the
  full grid, and the dense matrix [[A, B], [-B, -A]] of Eq. (1) diagonalised directly. Tiny
  systems only.
* ``operator`` + ``solver`` (O2) -- the paper's algorithm in the mixed chi/phi representation:
  Eq. operator_RPA for the operator (with the response density, Hartree + f_xc response potential
  and the <chi|V|phi> integrals of ``grid``), the trace functionals of Eqs. functional_RPA,
  tsip_grad and ortho, the preconditioner linear system of Eq. precond solved by CG, the
  auxiliary-matrix map of Eq. auxiliary, Gram-Schmidt with the sign flip of Sec. III C, and the
  subspace matrix Q of Sec. III C.

Pins that tie each function to something other than itself live in tests/test_oracle_*.py.
"""
