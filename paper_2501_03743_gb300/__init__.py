"""sscg: preconditioned s-step Conjugate Gradient (Chronopoulos and Gear) on
one NVIDIA GB300, after arXiv 2501.03743.

Modules
-------
sscg    ctypes binding of the C-ABI library ``_build/libsscg.so``
        (include/sscg.h); the CUDA kernels live in ``csrc/``.
inputs  seeded synthetic workloads (Poisson-type CSR matrices, right-hand sides).
build   nvcc build of the library for sm_103a.

Importing the package has no side effects; the library loads on first use.
"""

__version__ = "0.1.0"
