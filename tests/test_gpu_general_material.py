"""General per-ordinate material (obte_set_material_ordinates) on the GPU vs
the FP64 oracle (GPU).

Anisotropic synthetic materials (MFP and weight depending on direction) on 2D
and 3D meshes, both precisions, the gradient along y, the pore-free closed
form, the Fourier model with the anisotropic bulk tensor, the adjoint
gradient, the per-bin spectrum, the isotropic limit and the input checks.
"""
import numpy as np
import pytest

from gpu_common import KAPPA_RTOL, TL_ATOL, gpu, oracle, solid_vector
from paper_2106_02764_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


def _swap_xy(wl):
    import copy
    w = copy.deepcopy(wl)
    w.mask = np.ascontiguousarray(np.transpose(wl.mask, (0, 2, 1)))
    w.shape = (wl.shape[1], wl.shape[0], wl.shape[2])
    w.lengths = (wl.lengths[1], wl.lengths[0], wl.lengths[2])
    w.grad_axis = 1
    d = np.array(wl.ords["dirs"], float)
    d[:, [0, 1]] = d[:, [1, 0]]
    w.ords = dict(wl.ords, dirs=d)
    return w


L = 100e-9
CASES = {
    "2d_circle_12": lambda: I.anisotropic(I.small_2d(n=12, porosity=0.25, n_bins=2, n_phi=12), 0.3, 0.5),
    "2d_square_16_proj": lambda: I.anisotropic(
        I.make_2d("sq", 16, L, [I.square_pore(L, L, 0.15, x=0.35 * L, y=0.6 * L)], 3,
                  I.projected_quadrature(8, 4)), 0.35, 0.6),
    "2d_swapped": lambda: _swap_xy(I.anisotropic(
        I.make_2d("sq", 12, L, [I.square_pore(L, L, 0.12, x=0.3 * L, y=0.6 * L)], 2,
                  I.circle_quadrature(8)), 0.3, 0.5)),
    "3d_film": lambda: I.anisotropic(I.small_film(n=8, nz=4, porosity=0.15, n_bins=2, n_phi=8, n_mu=4),
                                     0.3, 0.4),
    "2d_32_warp": lambda: I.anisotropic(I.config1(), 0.25, 0.5),
}
_REF = {}


def _ref(name):
    if name not in _REF:
        wl = CASES[name]()
        _REF[name] = (wl,) + oracle(wl)
    return _REF[name]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", sorted(CASES))
def test_general_material_parity(name, precision):
    wl, pr, ref = _ref(name)
    s, st = gpu(wl, precision)
    k = s.kappa_eff
    assert abs(k - ref.kappa) <= KAPPA_RTOL[precision] * abs(ref.kappa), (k, ref.kappa)
    TL = solid_vector(pr, s.T_L())
    assert np.abs(TL - ref.T_L).max() <= TL_ATOL
    if precision == "fp64":
        assert abs(k - ref.kappa) < 1e-9 * abs(ref.kappa)
    # the per-bin spectrum (from one more sweep of the final state) adds up to
    # kappa; in mixed precision that sweep moves kappa by float rounding
    assert abs(s.kappa_bins().sum() - k) <= (1e-9 if precision == "fp64" else 1e-6) * abs(k)


def test_isotropic_limit_matches_separable_entry_point():
    wl = I.small_2d(n=12, porosity=0.2, n_bins=3, n_phi=8)
    s1, _ = gpu(wl, "fp64")
    s2, _ = gpu(I.anisotropic(wl, 0.0, 0.0), "fp64")
    assert abs(s1.kappa_eff - s2.kappa_eff) < 1e-11 * s1.kappa_eff
    a, b = s1.T_L(), s2.T_L()
    ok = wl.mask == 1
    assert np.abs(a[ok] - b[ok]).max() < 1e-11


def test_porefree_closed_form_anisotropic():
    wl = I.anisotropic(I.make_2d("pf", 8, L, [], 3, I.circle_quadrature(8)), 0.4, 0.6)
    from oracle import bte
    pr = bte.Problem.from_workload(wl)
    s, _ = gpu(wl, "fp64", tol=1e-14, tol_TL=1e-15)
    assert abs(s.kappa_eff - bte.kappa_bulk_discrete(pr)) < 1e-9 * bte.kappa_bulk_discrete(pr)


@pytest.mark.parametrize("name", ["2d_square_16_proj", "2d_swapped", "3d_film"])
def test_fourier_anisotropic(name):
    from oracle import fourier
    wl, pr, _ = _ref(name)
    ref = fourier.solve_fourier(pr.mesh, pr.ords.kappa_axes)
    from paper_2106_02764_gb300.binding import Solver
    r = Solver.from_workload(wl).solve_fourier(tol=1e-13)
    assert abs(r["kappa"] - ref["kappa"]) <= 1e-9 * abs(ref["kappa"])
    T = r["T"]
    c = pr.mesh.coords
    assert np.abs(T[c[:, 2], c[:, 1], c[:, 0]] - ref["T"]).max() <= 1e-9


def test_gradient_anisotropic():
    from oracle import adjoint, bte
    wl = I.anisotropic(I.small_2d(n=8, porosity=0.2, n_bins=3, n_phi=8, s_seed=21), 0.3, 0.5)
    pr = bte.Problem.from_workload(wl)
    g_ref, _ = adjoint.kappa_grad_s(pr, rtol=1e-13)
    s, _ = gpu(wl, "fp64")
    g = solid_vector(pr, s.kappa_grad_s())
    assert np.abs(g - g_ref).max() <= 1e-6 * np.abs(g_ref).max()


def test_general_material_input_checks():
    from paper_2106_02764_gb300.binding import ObteError, Solver
    wl = I.anisotropic(I.small_2d(n=8, porosity=0.2, n_bins=2, n_phi=8), 0.3, 0.5)
    o = wl.ords
    s = Solver()
    s.create_mesh(wl.mask, wl.lengths, wl.periodic, wl.grad_axis, wl.delta_T, wl.dim)

    def expect(code, **kw):
        args = dict(lam=o["lambda"], dirs=o["dirs"], weight=o["weight"], bins=o["bin"])
        args.update(kw)
        with pytest.raises(ObteError) as e:
            s.set_material_ordinates(**args)
        assert code in str(e.value)

    w = o["weight"].copy()
    w[3] = -1.0
    expect("EINVAL", weight=w)
    expect("EINVAL", weight=np.zeros_like(o["weight"]))
    lam = o["lambda"].copy()
    lam[0] = 0.0
    expect("EINVAL", lam=lam)
    lam[0] = np.nan
    expect("ENONFINITE", lam=lam)
    b = o["bin"].copy()
    b[1] = 7
    expect("EINVAL", bins=b, n_bins=2)
    # one direction without its mirror image: walls would not conserve energy
    d = np.array(o["dirs"], float)
    d[0] = [0.9, 0.1, 0.0]
    expect("EINVAL", dirs=d)
    # a valid call after the failures
    s.set_material_ordinates(o["lambda"], o["dirs"], o["weight"], o["bin"])
    st = s.solve(precision="fp64", tol=1e-10, max_iter=20000)
    assert st["converged"]
