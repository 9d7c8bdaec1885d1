"""The Fourier model alone (App. B) through obte_solve_fourier vs the FP64 oracle (GPU).

kappa_fourier and the temperature field against ``oracle.fourier.solve_fourier``
(a sparse direct solve) on small meshes: circular and square pores, a pore
across the hot contact, a rectangular cell, the gradient along y and a 3D film
with z walls; the oracle values stored for the full-size workloads; the
pore-free closed form; and the Eucken-Maxwell limit over a porosity sweep
(the comparison of Sec. 8).
"""
import numpy as np
import pytest

from gpu_common import SMALL, golden, rect_2d, transposed
from paper_2106_02764_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# FP64 conjugate gradients to |r| <= 1e-13 |b| against a direct solve
KF_RTOL = 1e-9
T_ATOL = 1e-9
CG_TOL = 1e-13


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


def _solver(wl):
    from paper_2106_02764_gb300.binding import Solver
    return Solver.from_workload(wl)


def _oracle(wl):
    from oracle import bte, fourier
    mesh = bte.Problem.from_workload(wl).mesh
    return mesh, fourier.solve_fourier(mesh, float(np.sum(wl.kappa_m)))


def _hot_contact_pore():
    L = 100e-9
    return I.make_2d("hotpore", 24, L, [I.square_pore(L, L, 0.12, x=0.0, y=0.4 * L)], 2,
                     I.circle_quadrature(8))


CASES = {
    "2d_circle_12_ragged": SMALL["2d_circle_12_ragged"],
    "2d_square_16": SMALL["2d_square_16"],
    "3d_film": SMALL["3d_film"],
    "rect": rect_2d,
    "rect_transposed": lambda: transposed(rect_2d()),
    "hot_contact_pore": _hot_contact_pore,
    "circle_64": lambda: I.make_2d("c64", 64, 100e-9, [I.circle_pore(100e-9, 100e-9, 0.2)], 2,
                                   I.circle_quadrature(8)),
    "film_24x24x10": lambda: I.small_film(n=24, nz=10, porosity=0.2, n_bins=2, n_phi=8, n_mu=4),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_fourier_parity(name):
    wl = CASES[name]()
    mesh, ref = _oracle(wl)
    s = _solver(wl)
    r = s.solve_fourier(tol=CG_TOL)
    assert r["converged"] and r["iterations"] > 0
    assert abs(r["kappa"] - ref["kappa"]) <= KF_RTOL * abs(ref["kappa"]), (r["kappa"], ref["kappa"])
    T = r["T"]
    c = mesh.coords
    assert np.abs(T[c[:, 2], c[:, 1], c[:, 0]] - ref["T"]).max() <= T_ATOL
    assert np.all(np.isnan(T[wl.mask == 0])) and np.all(np.isfinite(T[wl.mask == 1]))


@pytest.mark.parametrize("name", ["1", "5", "4_1", "4_2"])
def test_fourier_stored_oracle_values(name):
    """Full-size workloads: the oracle's kappa_fourier stored beside its
    kappa_eff (tests/golden/make_golden.py)."""
    g = golden(name)
    if g is None:
        pytest.skip(f"no stored oracle value for {name}")
    if name.startswith("4_"):
        wl = I.config4()[int(name.split("_")[1])]
    else:
        wl = I.CONFIGS[int(name)]()
    assert wl.name == g["workload"]
    r = _solver(wl).solve_fourier(tol=CG_TOL)
    assert r["converged"]
    assert abs(r["kappa"] - g["kappa_fourier"]) <= KF_RTOL * abs(g["kappa_fourier"]), (
        r["kappa"], g["kappa_fourier"])


def test_fourier_porefree_closed_form():
    """No pores: the linear profile solves the system exactly, kappa_fourier =
    kappa_bulk (App. B)."""
    wl = SMALL["2d_porefree"]()
    r = _solver(wl).solve_fourier(tol=CG_TOL)
    kb = float(np.sum(wl.kappa_m))
    assert abs(r["kappa"] - kb) <= 1e-12 * kb
    n = wl.mask.shape[-1]
    x = (np.arange(n) + 0.5) / n
    prof = -wl.delta_T * (x - x.mean())
    assert np.abs(r["T"][0] - prof[None, :]).max() <= 1e-12


def test_fourier_eucken_maxwell_sweep():
    """Porosity sweep of the Fourier model (the data-free experiment of Sec. 8):
    kappa_fourier / kappa_bulk follows (1 - phi) / (1 + phi) within 1 % at
    128 x 128 up to phi = 0.25 (the dilute limit: at 0.3 the next term of the
    square-array expansion already moves it by about 1 %) and falls
    monotonically with phi."""
    L = 100e-9
    ratios = []
    for phi in (0.05, 0.1, 0.15, 0.2, 0.25):
        wl = I.make_2d("em", 128, L, [I.circle_pore(L, L, phi)], 1, I.circle_quadrature(4))
        r = _solver(wl).solve_fourier(tol=1e-12)
        k = r["kappa"] / float(np.sum(wl.kappa_m))
        ph = wl.porosity
        assert abs(k / ((1 - ph) / (1 + ph)) - 1) < 0.01, (phi, k)
        ratios.append(k)
    assert all(a > b for a, b in zip(ratios, ratios[1:]))


def test_fourier_errors_and_cap():
    from paper_2106_02764_gb300.binding import ObteError, Solver
    wl = SMALL["2d_circle_8"]()
    s = Solver()
    s.create_mesh(wl.mask, wl.lengths, wl.periodic, wl.grad_axis, wl.delta_T, wl.dim)
    with pytest.raises(ObteError) as e:
        s.solve_fourier()
    assert "ESTATE" in str(e.value)
    s.set_material(wl.kappa_m, wl.lambda_m, wl.quad.dirs, wl.quad.weights, wl.quad.angular_dim)
    with pytest.raises(ObteError) as e:
        s.solve_fourier(tol=-1.0)
    assert "EINVAL" in str(e.value)
    r = s.solve_fourier(tol=1e-14, max_iter=1, allow_not_converged=True)
    assert not r["converged"] and r["iterations"] == 1 and np.isfinite(r["kappa"])
    with pytest.raises(ObteError):
        s.solve_fourier(tol=1e-14, max_iter=1)
    # the transport solve is unaffected by a Fourier-only call before it
    st = s.solve(precision="fp64", tol=1e-10, max_iter=20000)
    assert st["converged"]
