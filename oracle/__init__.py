"""FP64 CPU oracle of the two-level nonlinear Schwarz method (test infrastructure only).

This package is the independent reference that the CUDA path is checked against.
It is test infrastructure: only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import it.  It shares no code with the CUDA path; the only
module both sides use is the seeded input generator ``paper_2410_24138_gb300.inputs``,
which holds no arithmetic of the method.

Every routine is written plainly, in FP64, in the order and notation of the paper
(Heinlein, Ho, Klawonn, Lanser: "Nonlinear Two-Level Schwarz Methods: A Parallel
Implementation in FROSch", arXiv 2410.24138):

* ``fem``           Eq. 1 (nonlinear diffusion) and Eq. 2 (compressible Neo-Hooke),
                    element residuals/tangents and the global F(u), DF(u) of Eq. 3.
* ``decomposition`` overlapping element subdomains, the restriction R_i, extension
                    P_i and the restricted extension P~_i of Eq. 8.
* ``coarse``        the RGDSW coarse space (option 2.2, with the paper's Dirichlet-edge
                    modification, Section 2) and its energy-minimising extension.
* ``schwarz``       local corrections T_i (Eq. 4), F_1 (Eq. 5), the coarse correction T_0
                    (Eq. 9), F_a (Eq. 10), F_h (Eq. 11), their exact tangents (Eqs. 6, 7, 12),
                    GMRES on the tangent system (Eq. 13), the outer Newton loop, load
                    stepping and a plain global Newton used as the definition of F(u) = 0.
"""
