"""FP64 CPU oracle for the convolution-product expansion (test infrastructure).

This package is test infrastructure.  Only the test suite, the smoke check
and the CPU-baseline leg of the benchmark may import it; the product path
(the CUDA library and its binding) never does, and shares no code with it.

It is deliberately plain and slow: every function evaluates the definition it
cites, in float64, with no FFT blocking, fusion or reordering beyond what that
definition states.

Contents (each function cites the passage it follows):

* ``dft``          -- O4, the naive DFT with the sign of the Fourier atoms e_k
                      (Section 2) and the unnormalised-forward / 1/n-inverse
                      reading of the FFT identity of Section 3.5.
* ``expansion``    -- O1/O2/O3/O5: H_m u = sum_k h_k * (w_k . u) (Eq. 1.4) by
                      direct circular convolution, its adjoint, direct
                      quadrature of the integral operator (Eq. 1.1), and the
                      gradients of <H_m u, r>.
* ``construct``    -- the paper's example TVIRs (Examples 3.1-3.3, Fig. 1) and
                      the two constructions of (h_k, w_k) on hat spaces
                      (L2 projection, Corollary 4.3; interpolation, Section 4).

Every function is pinned by a CPU test (tests/test_oracle_*.py) against
values the paper prints, closed forms, invariants or brute force.
"""
