"""GB300-native consensus-ADMM trajectory optimiser (TOP, arXiv 2507.10290).

Submodules:
  top        ctypes binding of the CUDA library's C ABI (top_create,
             top_solve, top_grad, top_destroy); importing it loads the
             compiled library and fails loudly if it is missing.
  autograd   torch.autograd.Function around top_solve / top_grad.
  workloads  seeded synthetic inputs (no optimiser arithmetic).

Nothing is imported eagerly, so `workloads` can be used without loading the
CUDA library.
"""
