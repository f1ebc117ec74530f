"""GB300-native Cartesian-grid Active Flux method with AMR (arXiv 2205.07572).

The compute path is the CUDA library libaf.so (C ABI in include/af.h); this
package holds its sources (csrc/), its build script and a thin binding (af).
"""
from . import af  # noqa: F401
