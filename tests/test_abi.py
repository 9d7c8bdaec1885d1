"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares; the binding's signature table covers them all (CPU, no
compute call)."""
import ctypes
import glob
import os
import re

import pytest

from paper_2106_02764_gb300 import binding, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"\b(obte_[A-Za-z_0-9]+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("obte_create", "obte_create_mesh", "obte_set_material", "obte_solve",
              "obte_solve_batch", "obte_get_T_L", "obte_get_flux", "obte_get_kappa_eff",
              "obte_kappa_grad_s", "obte_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_signatures_match_header():
    assert {n for n, _, _ in binding.SIGNATURES} == _declared()


def test_struct_sizes_are_consistent(lib):
    # obte_default_opts writes the whole struct: run it into an oversized buffer
    buf = (ctypes.c_ubyte * (ctypes.sizeof(binding.SolveOpts) + 64))()
    lib.obte_default_opts.argtypes = [ctypes.c_void_p]
    lib.obte_default_opts(ctypes.cast(buf, ctypes.c_void_p))
    assert all(b == 0 for b in buf[ctypes.sizeof(binding.SolveOpts):])
    o = binding.SolveOpts.from_buffer(buf)
    assert o.precision == binding.OBTE_FP64 and o.max_iter == 2000 and o.use_graph == 1


def test_solver_refuses_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    with pytest.raises(RuntimeError):
        binding.Solver()


def test_package_level_names():
    """The package exposes the binding's main names and the autograd Function
    without importing them at package import."""
    import importlib
    import sys
    pkg = importlib.import_module("paper_2106_02764_gb300")
    from paper_2106_02764_gb300 import binding
    assert pkg.Solver is binding.Solver and pkg.solve_batch is binding.solve_batch
    assert pkg.ObteError is binding.ObteError
    from paper_2106_02764_gb300.autograd import KappaEff
    assert pkg.KappaEff is KappaEff
    assert "paper_2106_02764_gb300" in sys.modules
