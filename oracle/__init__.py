"""FP64 CPU oracle for the PolyCLEAN hot path (test infrastructure only).

This package is a plain, slow, obviously-correct restatement of what the paper
defines: the discrete measurement operator and its adjoint (Sect. 2.2, the
discrete forward equation and its adjoint), the LASSO objective (Sect. 4.1),
the dual certificate (Sect. 4.2), lambda_max (Sect. 5.3) and the Polyatomic
Frank-Wolfe loop (Algorithm 2) with an accelerated proximal-gradient
sub-solver (Sect. 4.4 / Sect. 5.1), over pixels or over the atoms of the
multi-scale synthesis dictionary (Sect. 4.3, diffuse experiment of Sect. 6).

It is test infrastructure. Only the test-suite, the smoke check of the
package entry file and the CPU-baseline leg of the benchmark may import it.
The GPU library never calls it, and it shares no code with the GPU library:
the only common module is the seeded input generator, which holds none of the
method's arithmetic.

Every floating-point computation here is float64 / complex128.

Parity status per function (what pins it, see tests/test_oracle_pins.py):
  operators.forward / adjoint      adjoint identity, lattice case == numpy.fft,
                                   point source == shifted PSF (w = 0) and != (w != 0)
  operators.lambda_max             x == 0 exactly for lambda >= lambda_max
  lasso.apgd                       single-atom closed form, brute force on 3x3 grids,
                                   independent coordinate descent
  pfw.solve                        KKT conditions, monotone objective, alpha identity,
                                   brute force on tiny grids
  pfw.duality_gap                  gap >= 0 and -> 0 at the optimum (KKT test)
  dictionary.kernel / synthesize   closed form, scipy.signal convolve2d / correlate2d,
    / analyze                      adjoint identity, single-atom placement and border crop
  dictionary.columns / forward     composite adjoint identity, sigma = 0 column == Phi column
    / adjoint / lambda_max
  dictionary.solve                 one-scale sigma = 0 dictionary == pfw.solve, theta = 0 at
                                   lambda_max, coordinate descent on the full dictionary
                                   (also non-negative), optimality conditions
"""
