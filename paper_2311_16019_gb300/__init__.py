"""GB300 (sm_103a) implementation of the sketched-and-truncated polynomial
Krylov method (s-PKSM) for A X + X B = C1 C2^T.

Submodules (imported on demand so that the problem generators can be used
without the CUDA library):
  inputs    seeded synthetic problems (no solver arithmetic)
  build     in-tree nvcc build of libspk.so
  spk       ctypes binding of the C ABI (include/spk.h)
  autograd  torch.autograd.Function for gradients through the solve
"""
__all__ = ["inputs", "build", "spk", "autograd"]
