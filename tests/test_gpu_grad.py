"""d kappa_eff / d s(x) on the GPU vs the FP64 oracle adjoint and central
finite differences of the GPU's own converged kappa (GPU)."""
import copy

import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I
from gpu_common import gpu, solid_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


def _case():
    return I.small_2d(n=8, porosity=0.2, n_bins=3, n_phi=8, s_seed=21)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_grad_vs_oracle_adjoint(precision):
    from oracle import adjoint, bte
    wl = _case()
    pr = bte.Problem.from_workload(wl)
    g_ref, _ = adjoint.kappa_grad_s(pr, rtol=1e-13)
    s, _ = gpu(wl, precision)
    g = solid_vector(pr, s.kappa_grad_s())
    tol = 1e-6 if precision == "fp64" else 1e-3
    assert np.abs(g - g_ref).max() <= tol * np.abs(g_ref).max()
    assert np.all(s.kappa_grad_s()[wl.mask == 0] == 0)


def test_grad_bounded_memory_batches_agree():
    """Recording one reversed pair of ordinates at a time gives the same gradient."""
    wl = _case()
    s, _ = gpu(wl, "fp64")
    g_all = s.kappa_grad_s()
    n_cells = wl.mask.size
    g_small = s.kappa_grad_s(max_field_bytes=2 * 8 * n_cells)
    assert np.abs(g_all - g_small).max() <= 1e-12 * np.abs(g_all).max()


def test_grad_vs_gpu_finite_differences():
    wl = I.small_2d(n=16, porosity=0.2, n_bins=3, n_phi=8, s_seed=5)
    s, _ = gpu(wl, "fp64", tol=1e-14, tol_TL=1e-15)
    g = s.kappa_grad_s()
    rng = np.random.default_rng(17)
    solid = np.argwhere(wl.mask[0] == 1)
    h = 1e-4
    for (y, x) in solid[rng.choice(len(solid), size=6, replace=False)]:
        kk = []
        for sgn in (1, -1):
            w2 = copy.deepcopy(wl)
            w2.s = wl.s.copy()
            w2.s[0, y, x] += sgn * h
            s2, _ = gpu(w2, "fp64", tol=1e-14, tol_TL=1e-15)
            kk.append(s2.kappa_eff)
        fd = (kk[0] - kk[1]) / (2 * h)
        assert abs(fd - g[0, y, x]) <= 1e-5 * np.abs(g).max(), (fd, g[0, y, x])


def test_autograd_function():
    torch = pytest.importorskip("torch")
    from paper_2106_02764_gb300.autograd import KappaEff
    wl = _case()
    s_t = torch.tensor(wl.s, dtype=torch.float64, requires_grad=True)
    k = KappaEff.apply(s_t, wl, "fp64")
    k.backward()
    from paper_2106_02764_gb300.binding import Solver
    sol = Solver.from_workload(wl)
    sol.solve(precision="fp64", tol=1e-12, tol_TL=1e-13, max_iter=200000, allow_not_converged=True)
    g = sol.kappa_grad_s()
    assert abs(float(k) - sol.kappa_eff) < 1e-9 * sol.kappa_eff
    assert np.abs(s_t.grad.numpy() - g).max() <= 1e-8 * np.abs(g).max()
