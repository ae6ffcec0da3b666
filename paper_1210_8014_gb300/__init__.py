"""GB300-native octree-AMR volume ray casting (Labadens et al., "Volume Rendering
of AMR Simulations", Sec. 2.2): exact-integer octree traversal and FP32
compensated / FP64 accumulation in hand-written sm_103a CUDA kernels behind the
C-ABI library ``libamr`` (declared in ``include/amr.h``).

Modules:
  amr     ctypes binding of libamr (same names as the C entry points)
  inputs  seeded synthetic octrees and cameras (input generation only)
"""
