"""GB300-native plane-evaluation Gaussian beamlet decomposition (arXiv 2404.12454).

``gbd`` is the thin ctypes binding of the CUDA library ``libgbd.so`` (C ABI in
``include/gbd.h``); ``workloads`` describes the seeded synthetic inputs; ``build``
compiles the library in-tree for sm_103a.  Importing the package loads nothing: the
library is opened on first use and its absence is an error, never a fallback.
"""
