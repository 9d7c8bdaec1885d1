"""obte_kappa_grad_s_noalloc: the gradient entry point for callers that cannot
allocate device memory when they need it (a service that reserved its whole
device-memory budget at start-up, or a loop sharing a full GPU with other
jobs).  Its buffers live in a fixed device array inside the library instead
of coming from cudaMalloc.  Through the C ABI, two calls in a row must both
agree with obte_kappa_grad_s (the allocating entry point) within the gradient
tolerance of the other GPU tests, also when the problem runs as several
batches of ordinate pairs whose fields leave their contents in the array.
Named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


def _solved(wl, precision):
    from paper_2106_02764_gb300.binding import Solver
    s = Solver.from_workload(wl)
    if precision == "fp64":
        s.solve(precision="fp64", tol=1e-12, tol_TL=1e-13, max_iter=200000, allow_not_converged=True)
        return s, 1e-9
    s.solve(precision="mixed", tol=0.0, tol_TL=0.0, max_iter=4000, allow_not_converged=True)
    return s, 1e-4


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_gradient_matches_allocating_entry_point(precision):
    wl = I.small_2d(n=16, porosity=0.2, n_bins=3, n_phi=8, s_seed=29)
    s, tol = _solved(wl, precision)
    ref = s.kappa_grad_s()
    scale = np.abs(ref).max()
    assert scale > 0
    for _ in range(2):  # the second call sees the first call's leftovers in the array
        g = s.kappa_grad_s_noalloc()
        assert g.shape == ref.shape
        assert np.all(g[wl.mask == 0] == 0)
        assert np.abs(g - ref).max() <= tol * scale


def test_noalloc_gradient_in_several_batches():
    """Config 5 in FP64 (128 x 128 cells, 640 ordinates): the 32 MiB hold 127
    reversed pairs of fields against the 320 pairs of the material, so the
    gradient runs as three batches and is summed across them.  Compared with
    the allocating entry point with its default field budget (one batch) and
    with a budget of 4 pairs (80 batches), two calls in a row."""
    wl = I.config5()
    s, tol = _solved(wl, "fp64")
    ref = s.kappa_grad_s()
    small = s.kappa_grad_s(max_field_bytes=2 * 4 * 8 * wl.mask.size)
    scale = np.abs(ref).max()
    assert np.abs(small - ref).max() <= tol * scale
    for _ in range(2):
        g = s.kappa_grad_s_noalloc()
        assert np.all(g[wl.mask == 0] == 0)
        assert np.abs(g - ref).max() <= tol * scale
