"""GB300-native (sm_103a) multilevel Monte Carlo estimator of E[AB] for random matrices
(Wu & Polydorides, arXiv:1904.00429).

The compute path is the CUDA library ``libmlmc.so`` behind the C ABI declared in
``include/mlmc.h``; ``binding`` marshals arguments to it through ctypes.  Importing this
package loads nothing: the library is opened on first use of the binding, and every
entry point fails loudly when it is missing.
"""

__all__ = ["autograd", "binding", "inputs"]
