"""B300-native gradient-guided SAT hot path (TurboSAT, arXiv 2511.07737).

Submodules:
  turbosat  -- ctypes binding of the C-ABI library ``libturbosat.so``
  autograd  -- ``SatObjective``, a torch.autograd.Function over the library
  cnfgen    -- seeded synthetic CNF generators (inputs only)
Importing the package does not load the CUDA library; ``turbosat`` does, and
fails loudly when the library is missing.
"""
__all__ = ["turbosat", "autograd", "cnfgen"]
