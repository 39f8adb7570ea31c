"""GB300-native Fourier PlenOctree renderer.

Rendering runs in libfpo.so (hand-written sm_103a CUDA kernels behind the C
ABI of include/fpo.h); `fpo` is its ctypes binding and `synth` draws seeded
synthetic inputs.  Importing the package loads nothing; the library is
loaded on first use and its absence is an error.
"""

__all__ = ["fpo", "synth", "build"]
