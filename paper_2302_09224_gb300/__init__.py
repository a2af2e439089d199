"""HISQ staggered stencil with reduced-bit storage formats and mixed-precision
Krylov solvers on NVIDIA GB300 (sm_103a).

The compute path is the C-ABI library ``libhisq.so`` (hand-written CUDA,
declared in ``include/hisq.h``); ``paper_2302_09224_gb300.hisq`` is its thin
ctypes binding and ``paper_2302_09224_gb300.synth`` makes the seeded inputs.
Importing the package loads nothing; the library is opened on first use and a
missing build raises instead of falling back to anything else.
"""

__all__ = ["hisq", "synth"]
