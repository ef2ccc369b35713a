"""GB300-native (sm_103a) local-energy hot path of the NNQS-Transformer
method (arXiv 2306.16705).

Submodules:
  inputs   seeded synthetic molecules, samples and ansatz parameters
  binding  ctypes binding of include/nnqs.h (libnnqs.so)
  vmc      the VMC step built from the binding (sampling, E_loc, gradient,
           Adam) and its torch.autograd.Function
"""
__all__ = ["inputs", "binding"]
