"""FP64 oracle: heat-conduction first guess and kappa_fourier (App. B).

TEST INFRASTRUCTURE ONLY (see the package docstring).

On a Cartesian grid every face is orthogonal to the line joining the two cell
centres, so the secondary ("non-orthogonal") flux of App. B vanishes and the
iteration Eq. fourier_iter reduces to one linear solve of the primary-flux
system: for every solid cell i,

    sum_{solid neighbours j} kappa_bulk / h_a^2 * (T_j - T_i - R^P_ij) = 0,

where R^P_ij is the jump of App. B (-dT when i is on the hot side of the
periodic plane and j the cold image; read here as: the image across the low
side of the gradient axis is hotter by dT).  Walls are adiabatic (no term).
The solution is fixed to solid-cell mean 0 by a bordered system.

kappa_fourier = -(L / (dT A)) sum_{hot-contact faces} g . S (App. B, last
equation), i.e. the conductive flux through the solid faces of the plane
x = 0 divided by the full cross-section.  An anisotropic material enters as
the diagonal of its bulk tensor (axis-aligned: kappa_a / h_a^2 per axis).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _axes(kappa_bulk):
    """kappa along each axis: a scalar (isotropic) or three diagonal entries
    (input handling only)."""
    return np.broadcast_to(np.asarray(kappa_bulk, float), (3,))


def assemble(mesh, kappa_bulk):
    """Primary-flux stiffness of App. B's finite-volume heat equation
    (negative semidefinite; the secondary flux vanishes on Cartesian cells)
    and the right-hand side of the periodic jump.
    kappa_bulk: scalar or the diagonal of an axis-aligned bulk tensor."""
    kap = _axes(kappa_bulk)
    rows, cols, vals = [], [], []
    rhs = np.zeros(mesh.nc)
    diag = np.zeros(mesh.nc)
    for a in mesh.axes:
        G = kap[a] / mesh.h[a] ** 2
        for side in (0, 1):
            j = mesh.nbr[:, a, side]
            ok = j >= 0
            c = np.nonzero(ok)[0]
            rows.append(c)
            cols.append(j[ok])
            vals.append(np.full(len(c), G))
            diag[c] -= G
            # G (T_j + jump - T_i): the jump goes to the right-hand side
            rhs[c] -= G * mesh.jump[c, a, side]
    rows.append(np.arange(mesh.nc))
    cols.append(np.arange(mesh.nc))
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.nc, mesh.nc))
    return A, rhs


def solve_fourier(mesh, kappa_bulk):
    """Solve App. B's Fourier system with the solid-cell mean of T fixed at 0
    (the gauge of E4); the first guess of Algorithm 1."""
    A, rhs = assemble(mesh, kappa_bulk)
    n = mesh.nc
    one = sp.csr_matrix(np.ones((1, n)))
    Bm = sp.bmat([[A, one.T], [one, None]], format="csc")
    x = spla.spsolve(Bm, np.concatenate([rhs, [0.0]]))
    T = x[:n]
    return {"T": T, "kappa": kappa_fourier(mesh, kappa_bulk, T)}


def kappa_fourier(mesh, kappa_bulk, T):
    """kappa_fourier: the conductive flux through the solid faces of the plane
    x_g = 0 times L / (dT A_sec) (App. B, last equation)."""
    g = mesh.grad_axis
    cells, img = mesh.hot_faces()
    jump = mesh.jump[cells, g, 0]
    flux = _axes(kappa_bulk)[g] * (T[img] + jump - T[cells]) / mesh.h[g]
    return mesh.lengths[g] / (mesh.delta_T * mesh.n_sec) * flux.sum()
