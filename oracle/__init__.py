"""CPU oracle for the relativistic space-charge BLDTT-FMM (arXiv 2302.07567).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement
of what the paper computes, written to check the CUDA library against.  It
is used by the test-suite, by the smoke check and by the CPU-baseline leg of
the benchmark, and by nothing else: the library never imports it and shares
no code, table or helper with it.

Modules
-------
physics   relativistic kernel g (Eq. 3.2), pair fields (Eq. 3.1), gamma-bar
          (Section 3), the brute-force direct sum (Alg. 10 with S_t=S_s=S,
          i != j, Section 5) and the exact uniform-motion field.
interp    Chebyshev points and the Lagrange basis of Eq. 2.2.
tree      Algs. 1-2 with the median split of Appendix B and the breadth-first
          node numbering of Section 8.
bldtt     the serial FMM: P2M/M2M (Algs. 3-5), diam/dist/admissible
          (Algs. 6-8), M2L/P2P (Algs. 9-10), the dual tree traversal
          (Algs. 11/17), L2L/L2P (Algs. 13-15) and the driver (Alg. 12).
metrics   the error of Eq. 5.1.
gradient  reference gradients: autograd through the frozen-plan FMM and
          through the direct sum.

Every floating-point quantity is float64.  Where the paper is silent or
ambiguous the reading taken is stated at the function that needs it.
"""
