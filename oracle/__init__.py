"""CPU FP64 oracle for the nonnested augmented subspace method (test infrastructure).

This package is TEST INFRASTRUCTURE.  Only the tests, the smoke check and the
benchmark's CPU-baseline / reference leg may import it.  The GPU library never
calls it, and it shares no code with the GPU library: every formula here is
restated from the paper (arXiv 2404.19249, "A Nonnested Augmented Subspace
Method for Kohn-Sham Equation") in plain NumPy/SciPy, FP64 throughout.

Modules and the passages they follow:
  quadrature   tetrahedral quadrature (the paper leaves the rule open; Sec. 2)
  fem          P1/P2 spaces on tetrahedra, assembly of K, M and potential
               mass matrices (Sec. 2 discretisation; Sec. 3.3, A_h^L and A_h^NL)
  lda          Slater exchange + Perdew-Zunger correlation and the
               energy formula (Sec. 3.1)
  hartree      Poisson problem for V_Har with multipole boundary values
               (Sec. 3.1)
  transfer     nonnested interpolation I_H^h (Sec. 3.2, Algorithm 1)
  anderson     Anderson density mixing (Sec. 4, Anderson mixing)
  nas          Algorithm 3 (augmented subspace step of Sec. 3.3: the
               linear problems and the blocks of F_A, F_B) with its inner SCF, plus the direct fine-space SCF used
               as the plain definition of the discrete ground state.
  spmm_omp.c   (C, OpenMP; built by build_c.py) the plain CSR product with N
               interleaved right-hand sides of Algorithm 3 step 1's block
               solves, timed on all host cores as the CPU baseline's SpMM
"""
