"""GB300-native explicit relativistic particle-in-cell step.

The hot path (field gather, Boris push, Esirkepov deposition, Yee update,
supercell frame maintenance) runs in the CUDA kernels of libpic, reached
through its C ABI (include/pic.h); ``pic`` is the thin ctypes binding and
``workloads`` the seeded synthetic inputs.  Build the library with
``build.build()``.
"""
from . import workloads  # noqa: F401

__all__ = ["workloads", "pic", "build"]
