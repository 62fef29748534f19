"""Plain FP64 CPU oracle for the backward-Euler Richards step (TEST INFRASTRUCTURE).

This package is a slow, obviously-correct restatement of the method of
Bertaccini, D'Ambra, Durastante and Filippone, "Why diffusion-based
preconditioning of Richards equation works" (arXiv 2112.05051).  It exists
only to check the CUDA path: the tests, the package smoke check and the
bench's CPU-baseline leg may import it; the product path never does.  It
shares no code with the CUDA library (only the seeded input generators of
``paper_2112_05051_gb300.synth``, which hold no arithmetic of the method).

Modules
  constitutive   s(p), K(p) and their derivatives (eqs. (s(p)), (K(p)),
                 (derivativeofcoefficients)).
  discretization face means, residual Phi (eq. (dynamic_of_the_problem)),
                 Jacobian J (Supplementary A/C entries, exact derivative),
                 diffusion-only preconditioner matrix (Sec. 4, after
                 Theorem (spectraldescription)).
  amg            strength, MIS-2 aggregation, smoothed prolongation,
                 Galerkin products, l1-Jacobi V-cycle (eq. (Vcycle), Sec. 5.2).
  krylov         flexible CG and flexible GMRES(m) with right
                 preconditioning (eq. (precsystem)).
  newton         inexact Newton with Armijo backtracking (Sec. 3).

Every array is float64 unless stated.  Cell c = i + nx (j + ny k).
"""
