"""GB300-native multilevel decomposition / recomposition of structured grids.

The hot path (coefficients, mass-transfer load vector, tridiagonal correction
solves, correction update, recomposition, their adjoints, the mixed-precision
and batched variants) runs as hand-written sm_103a CUDA kernels behind the C
ABI declared in ``include/mgard.h``.  Python modules:

* ``mgard``     -- ctypes binding of the C ABI (argument marshalling only)
* ``autograd``  -- torch.autograd.Function wrappers over the adjoint kernels
* ``autotune``  -- tile-shape autotuner for the batched path
* ``synth``     -- seeded synthetic input fields
* ``build``     -- nvcc build of the shared library

Importing the package loads nothing; ``mgard`` loads the CUDA library and
raises if it is missing.
"""
