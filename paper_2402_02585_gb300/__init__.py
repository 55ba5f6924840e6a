"""GB300 (sm_103a) Grover-QAOA statevector library for random 3-SAT.

Method: arXiv:2402.02585 (Grover-QAOA for 3-SAT). The compute path is the
CUDA library libgqaoa.so behind the C ABI of include/gqaoa.h; this package
holds its build script, the ctypes binding (`_capi`), thin torch wrappers
(`core`), the synthetic input generator (`instances`) and the host-side
drivers built on the kernels.

Importing the package does not load the CUDA library; the first call does,
and fails loudly if it cannot.
"""

__all__ = ["instances"]
