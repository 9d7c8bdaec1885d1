"""Brute-force dense solve of the whole discrete aMFP-BTE system (tiny meshes).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every unknown of App. A is written out -- the ordinate temperatures T_oi, the
lattice temperature T_Li and one wall temperature per wall face -- and every
equation (E1 transport rows, E2 energy conservation, E3 thermalising walls, E4
gauge) becomes one row of a dense matrix solved by least squares.  Neighbours,
jumps and walls are found here by walking the voxel grid directly, so this
module shares no indexing code with ``bte``: it checks that module's sparse
assembly, periodic wrap, wall bookkeeping and GMRES fixed point.
"""
from __future__ import annotations

import numpy as np


def dense_solve(mask, lengths, periodic, delta_T, dim, kappa_m, lambda_m, dirs,
                weights, angular_dim, s=None, grad_axis=0, transpose_rhs=None, ordinates=None):
    """``ordinates``: a general per-ordinate material {lambda, dirs, weight}
    (Sec. 5) replacing the bin x direction one; a_o = W_o / sum W and
    K_o = W_o Lambda_o s_o."""
    mask = np.asarray(mask).astype(bool)
    if mask.ndim == 2:
        mask = mask[None]
    nz, ny, nx = mask.shape
    n = (nx, ny, nz)
    h = (lengths[0] / nx, lengths[1] / ny, lengths[2] / nz if dim == 3 else 1.0)
    axes = list(range(dim))
    cells = [(x, y, z) for z in range(nz) for y in range(ny) for x in range(nx) if mask[z, y, x]]
    cid = {c: i for i, c in enumerate(cells)}
    nc = len(cells)
    sc = np.ones(nc) if s is None else np.array(
        [np.asarray(s).reshape(mask.shape)[z, y, x] for (x, y, z) in cells])

    lam, pv, aw, Kv = [], [], [], []
    if ordinates is None:
        # ordinate data, o = m * S + s
        M, S = len(kappa_m), len(weights)
        tot = sum(kappa_m[m] / lambda_m[m] ** 2 for m in range(M))
        for m in range(M):
            for q in range(S):
                p = [dirs[q][a] if a < dim else 0.0 for a in range(3)]
                lam.append(lambda_m[m])
                pv.append(p)
                aw.append(kappa_m[m] / lambda_m[m] ** 2 / tot * weights[q])
                Kv.append([angular_dim * kappa_m[m] * weights[q] * p[a] / lambda_m[m] for a in range(3)])
    else:
        Wtot = float(sum(ordinates["weight"]))
        for lo, do, wo in zip(ordinates["lambda"], ordinates["dirs"], ordinates["weight"]):
            p = [float(do[a]) if a < dim else 0.0 for a in range(3)]
            lam.append(float(lo))
            pv.append(p)
            aw.append(float(wo) / Wtot)
            Kv.append([float(wo) * float(lo) * p[a] for a in range(3)])
    O = len(lam)

    def neighbour(c, a, sgn):
        """(solid neighbour or None, jump, is_wall): the face kinds of App. A
        (R_ij between cells, R^P_ij across the period with the jump, g_si at a
        wall), found by walking the grid."""
        q = list(c)
        q[a] += sgn
        jump = 0.0
        if q[a] < 0 or q[a] >= n[a]:
            if not periodic[a]:
                return None, 0.0, True
            q[a] %= n[a]
            if a == grad_axis:
                jump = delta_T if sgn < 0 else -delta_T
        q = tuple(q)
        if not mask[q[2], q[1], q[0]]:
            return None, 0.0, True
        return q, jump, False

    walls = {}
    for c in cells:
        for a in axes:
            for sgn in (-1, 1):
                _, _, is_wall = neighbour(c, a, sgn)
                if is_wall:
                    walls[(c, a, sgn)] = len(walls)
    nw = len(walls)

    iT = lambda o, i: o * nc + i
    iL = lambda i: O * nc + i
    iW = lambda f: O * nc + nc + f
    nu = O * nc + nc + nw
    A = np.zeros((nu + 1, nu))
    b = np.zeros(nu + 1)
    row = 0
    # E1
    for o in range(O):
        for i, c in enumerate(cells):
            beta = [lam[o] * abs(pv[o][a]) / h[a] for a in range(3)]
            A[row, iT(o, i)] += sc[i] + sum(beta[a] for a in axes)
            A[row, iL(i)] -= sc[i]
            for a in axes:
                if pv[o][a] == 0.0:
                    continue
                sgn = -1 if pv[o][a] > 0 else 1          # inflow side
                q, jump, is_wall = neighbour(c, a, sgn)
                if is_wall:
                    A[row, iW(walls[(c, a, sgn)])] -= beta[a]
                else:
                    A[row, iT(o, cid[q])] -= beta[a]
                    b[row] += beta[a] * jump
            row += 1
    # E2
    for i in range(nc):
        A[row, iL(i)] = 1.0
        for o in range(O):
            A[row, iT(o, i)] -= aw[o]
        row += 1
    # E3
    for (c, a, sgn), f in walls.items():
        i = cid[c]
        num = [max(Kv[o][a] * sgn, 0.0) for o in range(O)]
        den = sum(num)
        A[row, iW(f)] = 1.0
        for o in range(O):
            if num[o] > 0:
                A[row, iT(o, i)] -= num[o] / den
        row += 1
    # E4
    for i in range(nc):
        A[row, iL(i)] = 1.0
    row += 1
    assert row == nu + 1

    # kappa functional: flux through the solid faces of the plane x_g = 0
    n_sec = int(np.prod([n[a] for a in axes if a != grad_axis]))
    scale = lengths[grad_axis] / (delta_T * n_sec)
    qv = np.zeros(nu)
    q0 = 0.0
    for i, c in enumerate(cells):
        if c[grad_axis] != 0:
            continue
        img, jump, is_wall = neighbour(c, grad_axis, -1)
        if is_wall:
            continue
        for o in range(O):
            kx = Kv[o][grad_axis]
            if kx > 0:
                qv[iT(o, cid[img])] += scale * kx
                q0 += scale * kx * jump
            elif kx < 0:
                qv[iT(o, i)] += scale * kx

    X = np.linalg.lstsq(A, b, rcond=None)[0]
    out = {
        "T": X[:O * nc].reshape(O, nc),
        "T_L": X[O * nc:O * nc + nc],
        "T_w": X[O * nc + nc:],
        "kappa": float(qv @ X + q0),
        "cells": cells,
        "walls": walls,
        "A": A[:nu],
        "q": qv,
        "residual": float(np.linalg.norm(A @ X - b)),
    }
    if transpose_rhs is not None:
        out["adjoint"] = np.linalg.lstsq(A[:nu].T, transpose_rhs(out), rcond=None)[0]
    return out


def dense_from_workload(wl, s=None, **kw):
    """dense_solve on a synthetic workload's inputs (input marshalling only)."""
    q = wl.quad
    return dense_solve(wl.mask, wl.lengths, wl.periodic, wl.delta_T, wl.dim,
                       list(wl.kappa_m), list(wl.lambda_m), [list(d) for d in q.dirs],
                       list(q.weights), q.angular_dim, s=s if s is not None else wl.s,
                       grad_axis=wl.grad_axis, ordinates=getattr(wl, "ords", None), **kw)
