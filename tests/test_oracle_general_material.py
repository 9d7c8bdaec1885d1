"""Pins of the oracle's general per-ordinate material (Sec. 5, App. A) (CPU).

The general form gives every ordinate its own MFP Lambda_o, direction s_o and
weight W_o (a_o = W_o / sum W, K_o = W_o Lambda_o s_o).  Pinned against: the
bin x direction material it generalises, the pore-free closed form with the
anisotropic bulk tensor, a brute-force dense solve, conservation of energy,
the x <-> y transposition symmetry, and finite differences of the adjoint
gradient.
"""
import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I
from oracle import adjoint, bte, dense, fourier


def _solve(wl, **kw):
    pr = bte.Problem.from_workload(wl)
    return pr, bte.solve_mode_B(pr, **kw)


@pytest.mark.parametrize("make", [lambda: I.small_2d(n=8, porosity=0.2, n_bins=3, n_phi=8),
                                  lambda: I.small_film(n=6, nz=3, porosity=0.15, n_bins=2,
                                                       n_phi=4, n_mu=2)])
def test_isotropic_limit_is_the_separable_material(make):
    """eps = 0: the per-ordinate form with W_o = d_ang w_s kappa_m / Lambda_m^2
    reproduces the bin x direction material's weights and fixed point."""
    wl = make()
    wg = I.anisotropic(wl, 0.0, 0.0)
    pr, sol = _solve(wl, rtol=1e-13)
    pg, solg = _solve(wg, rtol=1e-13)
    assert np.abs(pr.ords.a - pg.ords.a).max() < 1e-15
    assert np.abs(pr.ords.K - pg.ords.K).max() < 1e-13 * np.abs(pr.ords.K).max()
    assert abs(sol.kappa - solg.kappa) < 1e-11 * sol.kappa
    assert np.abs(sol.T_L - solg.T_L).max() < 1e-11


@pytest.mark.parametrize("quad", [I.circle_quadrature(8), I.projected_quadrature(8, 4)])
def test_porefree_closed_form_anisotropic(quad):
    """Pore-free periodic cell: T_o = T_L - Lambda_o s_ox a solves E1 exactly for
    a linear T_L of slope a = -dT/L as long as sum_o a_o Lambda_o s_ox = 0
    (time reversal); the upwinded hot-face flux is then
    kappa_xx + (h/2) sum_o |K_ox| with kappa_xx = sum_o W_o Lambda_o^2 s_ox^2."""
    L = 100e-9
    wl = I.anisotropic(I.make_2d("pf", 8, L, [], 3, quad), 0.4, 0.6)
    pr, sol = _solve(wl)
    o = wl.ords
    p = np.asarray(o["dirs"])
    kxx = float(np.sum(o["weight"] * o["lambda"] ** 2 * p[:, 0] ** 2))
    kyy = float(np.sum(o["weight"] * o["lambda"] ** 2 * p[:, 1] ** 2))
    assert abs(kxx / kyy - 1) > 0.2          # the material is anisotropic
    h = L / 8
    K = np.asarray(o["weight"] * o["lambda"])[:, None] * p
    expect = kxx + 0.5 * h * np.abs(K[:, 0]).sum()
    assert abs(sol.kappa - expect) < 1e-12 * expect
    x = (pr.mesh.coords[:, 0] + 0.5) * h
    assert np.abs(sol.T_L + (x - x.mean()) / L).max() < 1e-12


@pytest.mark.parametrize("case", ["2d", "3d"])
def test_dense_brute_force_anisotropic(case):
    if case == "2d":
        wl = I.small_2d(n=4, porosity=0, n_bins=2, n_phi=8)
        wl.mask = np.ones((1, 4, 4), np.uint8)
        wl.mask[0, 1:3, 1:3] = 0
    else:
        wl = I.small_film(n=4, nz=2, porosity=0, n_bins=2, n_phi=4, n_mu=2)
        wl.mask[:, 1:3, 1:3] = 0
    wl = I.anisotropic(wl, 0.35, 0.5)
    pr, sol = _solve(wl, rtol=1e-13)
    d = dense.dense_from_workload(wl)
    assert d["residual"] < 1e-10
    assert abs(sol.kappa - d["kappa"]) < 1e-9 * abs(d["kappa"])
    assert np.abs(sol.T_L - d["T_L"]).max() < 1e-9


def test_conservation_anisotropic():
    """Every x-section carries the same net heat flux at the fixed point."""
    L = 100e-9
    wl = I.anisotropic(I.make_2d("cons", 12, L, [I.square_pore(L, L, 0.12, x=0.4 * L, y=0.55 * L)],
                                 3, I.circle_quadrature(8)), 0.3, 0.5)
    pr, sol = _solve(wl, rtol=1e-13)
    phis = bte.fields(pr, sol)["phis"]
    assert np.abs(phis - phis[0]).max() < 1e-9 * abs(phis[0])


def _swap_xy(wl):
    """The same problem with x and y exchanged: mask transposed, gradient along
    y, every ordinate's direction with its x and y components exchanged."""
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


def test_transposition_symmetry_anisotropic():
    L = 100e-9
    wl = I.anisotropic(I.make_2d("asym", 8, L, [I.square_pore(L, L, 0.1, x=0.3 * L, y=0.6 * L)], 2,
                                 I.circle_quadrature(8)), 0.3, 0.5)
    _, sol = _solve(wl, rtol=1e-13)
    _, solr = _solve(_swap_xy(wl), rtol=1e-13)
    assert abs(sol.kappa - solr.kappa) < 1e-11 * sol.kappa
    # and the anisotropy matters: the same mask with the gradient along y differs
    w2 = _swap_xy(wl)
    w2.ords = wl.ords
    _, sol2 = _solve(w2, rtol=1e-13)
    assert abs(sol2.kappa - sol.kappa) > 1e-3 * sol.kappa


def test_fourier_anisotropic_closed_form_and_transposition():
    """Fourier model with the axis-aligned bulk tensor: exact linear profile
    without pores (kappa_fourier = kappa_xx), and x <-> y transposition
    symmetry with a pore."""
    L = 100e-9
    pf = I.anisotropic(I.make_2d("pf", 10, L, [], 2, I.circle_quadrature(8)), 0.4, 0.6)
    pr = bte.Problem.from_workload(pf)
    k = pr.ords.kappa_axes
    r = fourier.solve_fourier(pr.mesh, k)
    assert abs(r["kappa"] - k[0]) < 1e-10 * k[0]
    wl = I.anisotropic(I.make_2d("asym", 10, L, [I.square_pore(L, L, 0.1, x=0.3 * L, y=0.6 * L)],
                                 2, I.circle_quadrature(8)), 0.4, 0.6)
    p1 = bte.Problem.from_workload(wl)
    p2 = bte.Problem.from_workload(_swap_xy(wl))
    assert abs(p1.ords.kappa_axes[0] - p2.ords.kappa_axes[1]) < 1e-12 * p1.ords.kappa_axes[0]
    k1 = fourier.solve_fourier(p1.mesh, p1.ords.kappa_axes)["kappa"]
    k2 = fourier.solve_fourier(p2.mesh, p2.ords.kappa_axes)["kappa"]
    assert abs(k1 - k2) < 1e-10 * k1
    # an isotropic stencil at kappa_xx gives a different value: the tensor is used
    k_iso = fourier.solve_fourier(p1.mesh, p1.ords.kappa_axes[0])["kappa"]
    assert abs(k_iso - k1) > 1e-3 * k1


def test_adjoint_gradient_anisotropic():
    """d kappa / d s by the adjoint equals central differences (h = 1e-5)."""
    wl = I.anisotropic(I.small_2d(n=6, porosity=0.15, n_bins=2, n_phi=8, s_seed=7), 0.3, 0.5)
    pr = bte.Problem.from_workload(wl)
    g, _ = adjoint.kappa_grad_s(pr, rtol=1e-13)
    h = 1e-5
    rng = np.random.default_rng(5)
    for i in rng.choice(pr.mesh.nc, size=4, replace=False):
        sp_, sm_ = pr.s.copy(), pr.s.copy()
        sp_[i] += h
        sm_[i] -= h
        kp = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, sp_), rtol=1e-14).kappa
        km = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, sm_), rtol=1e-14).kappa
        assert abs((kp - km) / (2 * h) - g[i]) < 1e-5 * np.abs(g).max()
