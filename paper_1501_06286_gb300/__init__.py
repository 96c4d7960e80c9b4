"""GB300 (sm_103a) fast QMC matrix product B = Y·A (arXiv 1501.06286).

Submodules
  capi       ctypes declarations of the C ABI (include/qmc.h)
  qmc        Plan / Batch: products, adjoint, point generation
  autograd   QmcMatmul and ExpMeanLoss autograd functions
  workloads  seeded synthetic inputs (no method arithmetic)
  build      nvcc build of libqmcfft.so

The CUDA library is loaded on first use; a missing library raises.
"""

__all__ = ["capi", "qmc", "autograd", "workloads", "build"]
