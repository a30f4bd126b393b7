"""GB300-native (sm_103a) hot path of matrix-free natural gradient descent for PINNs
with a randomized Nystrom preconditioner (Bioli, Marcati, Sangalli, arXiv 2505.11638).

The compute path lives in the CUDA shared library ``libngd.so`` built from ``csrc/``;
``paper_2505_11638_gb300.ngd`` is the thin ctypes binding over its C ABI
(``include/ngd.h``).  ``paper_2505_11638_gb300.inputs`` holds the seeded synthetic
problem generators.  Importing this package loads nothing: the binding opens the
library on first use and raises if it is missing.
"""

__all__ = ["inputs", "ngd", "build"]
