"""GB300-native affinity propagation (Xia et al.: AP, partition AP, landmark AP).

The compute path is the CUDA library ``libapgb.so`` (C ABI in include/apgb.h);
``capi`` is its Python binding, ``synth`` the seeded workload generators.
"""
from . import synth  # noqa: F401

__all__ = ["capi", "synth", "build"]
