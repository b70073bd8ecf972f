"""GB300-native BURA solver for A^alpha u = f (multi-shift multigrid-PCG in CUDA for sm_103a).

Submodules:
  bura       ctypes binding of the C ABI (include/bura.h); loads libbura.so
  build_lib  in-tree nvcc build of libbura.so
  workloads  seeded synthetic inputs (grids, right-hand sides, coefficient fields)
"""
