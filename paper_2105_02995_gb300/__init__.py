"""GB300-native apply of the approximate inverse of discrete Fourier integral operators.

Layout:
  builder/   host factor builder (butterfly, peeling, hierarchical interpolative factorisation)
             and the stage-major packer; runs once per operator.
  csrc/      CUDA kernels for sm_103a and the C ABI (libfio).
  binding.py ctypes binding of the C ABI (argument marshalling only).
  inputs.py  seeded synthetic inputs (random right-hand sides), no method arithmetic.

Importing the package does not load the CUDA library; ``binding.load()`` does, and fails loudly
when it is missing.
"""

__all__ = ["builder", "binding", "inputs"]
