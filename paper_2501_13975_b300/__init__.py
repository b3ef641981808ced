"""gs2: B300-native hot path of near-second-order (local Newton) 3D Gaussian
Splatting training (arXiv 2501.13975).

Submodules:
  synth    seeded synthetic scenes and cameras (inputs only)
  gs2      ctypes binding of the CUDA library libgs2.so (imported lazily so
           that input generation works without the compiled library)
"""
__all__ = ["synth", "gs2"]
