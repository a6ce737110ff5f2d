"""CPU oracle for periodic LR-CCSD (test infrastructure only).

Plain, slow, FP64/complex128 implementations of what the GPU path computes, written
from the method's equations.  Only the test-suite, the smoke check and the CPU
baseline leg of the benchmark may import this package; the library itself never
does, and shares no code with it.

Modules:
  spinorb   dense spin-orbital collective-index CCSD residual and energy in the
            arrangement of Eqs. 6-8 (tiny sizes).
  fci       brute force in determinant space (similarity-transformed Hamiltonian
            projections, FCI sum-over-states polarizability).
  rcc       closed-shell, k-blocked CCSD: dressed residual, Jacobian products by
            exact polynomial stencils, transpose products, ground-state, Lambda and
            perturbed-amplitude solvers, linear-response polarizability.
"""
