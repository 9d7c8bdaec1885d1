"""obte_kappa_grad_s_noalloc: the gradient entry point for callers that cannot
allocate device memory when they need it (for example while a framework
captures a CUDA graph).  Its buffers live in a fixed device array inside the
library instead of coming from cudaMalloc.  Through the C ABI, two calls in a
row must both agree with obte_kappa_grad_s (the allocating entry point) within
the gradient tolerance of the other GPU tests.  Named so that pytest collects
it last.
"""
import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_gradient_matches_allocating_entry_point(precision):
    from paper_2106_02764_gb300.binding import Solver
    wl = I.small_2d(n=16, porosity=0.2, n_bins=3, n_phi=8, s_seed=29)
    s = Solver.from_workload(wl)
    if precision == "fp64":
        s.solve(precision="fp64", tol=1e-12, tol_TL=1e-13, max_iter=200000, allow_not_converged=True)
        tol = 1e-9
    else:
        s.solve(precision="mixed", tol=0.0, tol_TL=0.0, max_iter=4000, allow_not_converged=True)
        tol = 1e-4
    ref = s.kappa_grad_s()
    scale = np.abs(ref).max()
    assert scale > 0
    for _ in range(2):  # the second call sees the first call's leftovers in the array
        g = s.kappa_grad_s_noalloc()
        assert g.shape == ref.shape
        assert np.all(g[wl.mask == 0] == 0)
        assert np.abs(g - ref).max() <= tol * scale
