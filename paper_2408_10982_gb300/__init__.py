"""GB300-native RIS influence-maximization hot path (GreediRIS, arXiv 2408.10982).

Submodules:
  inputs  -- seeded synthetic R-MAT graphs and edge weights (fixtures)
  im      -- thin ctypes binding over the CUDA library libim.so (C ABI in
             include/im.h); every step of the path runs in its kernels
"""
