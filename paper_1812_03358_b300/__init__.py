"""B300-native light-transport camera model (McGaffin et al., arXiv 1812.03358).

Submodules:
  inputs  -- seeded synthetic volumes, cameras and noise (no model arithmetic)
  lt      -- ctypes binding of the C ABI in include/lt.h (liblt.so, sm_103a)
  build   -- nvcc build of the in-tree library
"""
