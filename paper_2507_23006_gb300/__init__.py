"""GB300-native differentiable tile-based Gaussian rasterizer.

The CUDA library (libgsr.so, C ABI in include/gsr.h) is loaded on first use by
``paper_2507_23006_gb300.native``; importing this package loads nothing, so the scene
generators in ``scenes`` can be used without a GPU.
"""

__all__ = ["scenes", "native", "build"]
