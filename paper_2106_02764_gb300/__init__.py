"""GB300-native aMFP phonon-BTE sweep solver (OpenBTE, arXiv 2106.02764).

Submodules:
  inputs   -- seeded synthetic inputs (masks, MFP bins, quadratures)
  binding  -- ctypes binding to the CUDA C-ABI library ``libobte``
  autograd -- torch.autograd.Function for d kappa_eff / d s(x)
The binding is imported lazily so that ``inputs`` stays importable alone; the
main names are reachable from the package itself (``Solver``,
``solve_batch``, ``measure_fma_rate``, ``ObteError`` from the binding,
``KappaEff`` from autograd), each imported on first use.
"""
__all__ = ["inputs", "binding", "autograd", "Solver", "solve_batch", "measure_fma_rate",
           "ObteError", "KappaEff"]

_FROM_BINDING = ("Solver", "solve_batch", "measure_fma_rate", "ObteError")


def __getattr__(name):
    if name in _FROM_BINDING:
        from . import binding
        return getattr(binding, name)
    if name == "KappaEff":
        from .autograd import KappaEff
        return KappaEff
    raise AttributeError(f"module {__name__!r} has no attribute {name!r}")
