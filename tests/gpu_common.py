"""Helpers shared by the GPU test modules (oracle references and solver runs)."""
import json
import os

import numpy as np

from paper_2106_02764_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))

# tolerances of the parity bar
KAPPA_RTOL = {"fp64": 1e-6, "mixed": 1e-4}
TL_ATOL = 1e-5


def oracle(wl, rtol=1e-13):
    from oracle import bte
    pr = bte.Problem.from_workload(wl)
    return pr, bte.solve_mode_B(pr, rtol=rtol)


def gpu(wl, precision="fp64", **kw):
    """Solve to a tight fixed point.  FP64: relative kappa change <= 1e-12 and
    max |dT_L| <= 1e-13 K.  Mixed: a fixed 4000 iterations (float rounding
    noise sits above any tight change test).  Long-MFP ordinates converge
    through the lagged periodic cut, so a test on T_L alone is not enough."""
    from paper_2106_02764_gb300.binding import Solver
    s = Solver.from_workload(wl)
    if precision == "fp64":
        opts = dict(tol=1e-12, tol_TL=1e-13, max_iter=200000, check_every=32)
    else:
        opts = dict(tol=0.0, tol_TL=0.0, max_iter=4000, check_every=50)
    opts.update(kw)
    st = s.solve(precision=precision, allow_not_converged=True, **opts)
    return s, st


def solid_vector(pr, grid):
    c = pr.mesh.coords
    return grid[c[:, 2], c[:, 1], c[:, 0]]


def golden(name):
    p = os.path.join(HERE, "golden", f"kappa_star_cfg{name}.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        return json.load(f)


SMALL = {
    "2d_circle_8": lambda: I.small_2d(n=8, porosity=0.2, n_bins=3, n_phi=8),
    "2d_circle_12_ragged": lambda: I.small_2d(n=12, porosity=0.25, n_bins=2, n_phi=12),
    "2d_square_16": lambda: I.small_2d(n=16, porosity=0.15, n_bins=3, n_phi=8, pore="square"),
    "2d_projected": lambda: I.make_2d("proj", 8, 100e-9, [I.circle_pore(100e-9, 100e-9, 0.2)], 3,
                                      I.projected_quadrature(8, 4)),
    "2d_porefree": lambda: I.small_2d(n=8, porosity=0.0, n_bins=3, n_phi=8),
    "3d_film": lambda: I.small_film(n=8, nz=4, porosity=0.15, n_bins=2, n_phi=8, n_mu=4),
    "3d_film_porefree": lambda: I.small_film(n=8, nz=4, porosity=0.0, n_bins=2, n_phi=4, n_mu=4),
    "2d_scatter": lambda: I.small_2d(n=8, porosity=0.2, n_bins=3, n_phi=8, s_seed=3),
}


def rect_2d():
    """nx = 8, ny = 16 (ny a multiple of nx), off-centre square pore."""
    L = 100e-9
    wl = I.make_2d("rect", 8, L, [], 3, I.circle_quadrature(8))
    mask = I.pores_mask(8, 16, L, 2 * L, [I.square_pore(L, 2 * L, 0.1, x=0.3 * L, y=0.7 * L)])
    wl.mask = mask
    wl.shape = (8, 16, 1)
    wl.lengths = (L, 2 * L, 0.0)
    return wl


def transposed(wl):
    """Same problem with the gradient along y (mask transposed)."""
    import copy
    w = copy.deepcopy(wl)
    w.mask = np.ascontiguousarray(np.transpose(wl.mask, (0, 2, 1)))
    w.shape = (wl.shape[1], wl.shape[0], wl.shape[2])
    w.lengths = (wl.lengths[1], wl.lengths[0], wl.lengths[2])
    w.grad_axis = 1
    if wl.s is not None:
        w.s = np.ascontiguousarray(np.transpose(wl.s, (0, 2, 1)))
    return w
