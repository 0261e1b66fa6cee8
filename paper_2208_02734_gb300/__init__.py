"""GB300-native MASK: multilevel k-means index build and top-down approximate
k-NN query (Ortega et al., "Unconventional application of k-means for
distributed approximate similarity search", §3.1-§3.3).

The compute path lives in ``libmask_gb300.so`` (CUDA for sm_103a, C ABI in
``include/mask.h``).  ``paper_2208_02734_gb300.mask`` is the thin ctypes
binding over it; ``paper_2208_02734_gb300.synth`` holds the seeded synthetic
input generators.  Importing this package loads nothing: the shared library is
opened on first use and a missing library is an error, never a fallback.
"""

__all__ = ["mask", "synth"]
