"""GB300-native MAPA allocation engine (arXiv 2110.03214).

The compute path lives in the C-ABI library built from ``csrc/`` (see
``include/mapa.h``); ``mapa`` is its ctypes binding.  Importing the package
does not load the library; ``paper_2110_03214_gb300.mapa`` does, and raises if
it is missing.
"""

__all__ = ["workloads", "mapa", "build"]
