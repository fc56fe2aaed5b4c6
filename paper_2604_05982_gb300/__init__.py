"""GB300-native GPU-resident fork-join task runtime (GTaP method, arXiv 2604.05982).

The compute path is the native library libgtap.so (hand-written CUDA for
sm_103a) behind the C ABI declared in include/gtap.h; ``gtap`` is its ctypes
binding and ``runner`` a thin convenience layer.  ``inputs`` holds the seeded
synthetic input generators.  Importing the package does not load the native
library; the first call does, and fails loudly if it was not built.
"""
__all__ = ["gtap", "runner", "inputs", "build"]
