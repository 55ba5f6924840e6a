"""FP64 CPU oracle for Grover-QAOA on 3-SAT (arXiv:2402.02585).

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct reference that
the CUDA library is checked against. Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import it. It shares no code with the CUDA
path and never imports the product package.

Modules:
  statevector  full 2^n complex128 statevector (plain C via ctypes):
               cost table, histogram, evolution, readout, sampling, Philox.
  reduced      the exact (m+1)-dimensional cost-class model of Appendix C,
               its readouts and its adjoint gradient (numpy).
  mlp          FP64 forward/backward/Adam of the angle-proposer MLP (numpy).

Parity status of every function is stated in its module header.
"""
