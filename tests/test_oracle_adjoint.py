"""Pins of the oracle's adjoint and d kappa_eff / d s(x) (CPU)."""
import numpy as np

from paper_2106_02764_gb300 import inputs as I
from oracle import adjoint, bte, dense


def _wl():
    return I.small_2d(n=6, porosity=0.15, n_bins=2, n_phi=8, s_seed=7)


def test_gradient_matches_central_differences():
    """Central finite differences of the converged kappa (h = 1e-5)."""
    wl = _wl()
    pr = bte.Problem.from_workload(wl)
    g, _ = adjoint.kappa_grad_s(pr, rtol=1e-13)
    h = 1e-5
    rng = np.random.default_rng(5)
    for i in rng.choice(pr.mesh.nc, size=6, replace=False):
        sp_, sm_ = pr.s.copy(), pr.s.copy()
        sp_[i] += h
        sm_[i] -= h
        kp = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, sp_), rtol=1e-14).kappa
        km = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, sm_), rtol=1e-14).kappa
        fd = (kp - km) / (2 * h)
        assert abs(fd - g[i]) < 1e-5 * np.abs(g).max()


def test_adjoint_matches_dense_transpose():
    """lambda from the transposed sparse solves + GMRES equals the E1 block of
    the dense transposed system A^T Lambda = q (4x4 mesh with a 2x2 pore)."""
    wl = I.small_2d(n=4, porosity=0, n_bins=2, n_phi=8, s_seed=11)
    wl.mask = np.ones((1, 4, 4), np.uint8)
    wl.mask[0, 1:3, 1:3] = 0
    pr = bte.Problem.from_workload(wl)
    g, info = adjoint.kappa_grad_s(pr, rtol=1e-14)
    d = dense.dense_from_workload(wl, transpose_rhs=lambda out: out["q"])
    O, nc = pr.ords.n, pr.mesh.nc
    lam_d = d["adjoint"][:O * nc].reshape(O, nc)
    lams = info["adjoint"].lams
    # adjoint fields are defined up to the left null vector of A; compare the
    # gauge-free gradient and the fields after removing a common shift
    gd = np.zeros(nc)
    for o in range(O):
        gd -= lam_d[o] * (info["forward"]["T"][o] - info["solution"].T_L)
    assert np.abs(g - gd).max() < 1e-9 * np.abs(g).max()


def test_reciprocity_identity():
    """The adjoint field of ordinate o, divided by its energy weight a_o, is the
    forward field of the reversed ordinate for an applied jump
    -(L/(dT N_sec)) d_ang h_x sum kappa_m / Lambda_m^2, up to a constant
    (the transposed upwind operator is the upwind operator of -p)."""
    wl = _wl()
    pr = bte.Problem.from_workload(wl)
    g, info = adjoint.kappa_grad_s(pr, rtol=1e-13)
    rev = adjoint.reversed_ordinate(pr.ords)
    J = adjoint.adjoint_jump(pr) / pr.mesh.delta_T
    lams, T = info["adjoint"].lams, info["forward"]["T"]
    for o in range(pr.ords.n):
        d = lams[o] / pr.ords.a[o] - J * T[rev[o]]
        assert d.max() - d.min() < 1e-8 * np.abs(lams[o] / pr.ords.a[o]).max()
    # hence the gradient from forward fields alone
    g2 = np.zeros(pr.mesh.nc)
    for o in range(pr.ords.n):
        g2 -= pr.ords.a[o] * J * T[rev[o]] * (T[o] - info["solution"].T_L)
    assert np.abs(g - g2).max() < 1e-8 * np.abs(g).max()


def test_gradient_gauge_and_sign():
    """Uniformly stronger scattering lowers kappa: sum_i dkappa/ds_i < 0, and
    equals the derivative of kappa along s -> s (1 + t)."""
    wl = _wl()
    pr = bte.Problem.from_workload(wl)
    g, info = adjoint.kappa_grad_s(pr, rtol=1e-13)
    assert g.sum() < 0
    t = 1e-6
    kp = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, pr.s * (1 + t)), rtol=1e-14).kappa
    km = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, pr.s * (1 - t)), rtol=1e-14).kappa
    assert abs((kp - km) / (2 * t) - np.dot(g, pr.s)) < 1e-5 * abs(np.dot(g, pr.s))
