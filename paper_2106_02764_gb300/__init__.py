"""GB300-native aMFP phonon-BTE sweep solver (OpenBTE, arXiv 2106.02764).

Submodules:
  inputs   -- seeded synthetic inputs (masks, MFP bins, quadratures)
  binding  -- ctypes binding to the CUDA C-ABI library ``libobte``
  autograd -- torch.autograd.Function for d kappa_eff / d s(x)
The binding is imported lazily so that ``inputs`` stays importable alone.
"""
__all__ = ["inputs", "binding", "autograd"]
