"""GB300-native locally adaptive non-hydrostatic shallow-water library.

The compute path is the CUDA shared library built from ``csrc/`` (C ABI in
``include/nhswe.h``); ``nhswe`` is its thin ctypes binding.  Importing this
package does not load the library; ``nhswe.load()`` does, and it raises if the
library is missing -- there is no CPU fallback.
"""

__all__ = ["nhswe", "workloads"]
