"""FP64 oracle: adjoint of the discrete aMFP-BTE and d kappa_eff / d s(x).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper lists differentiability as future work (Sec. 9); the sensitivity
computed here is that of the discrete system written out in ``bte`` (E1-E4)
to a per-cell scattering scale s_i, which multiplies the collision term of E1
only:  Lambda_m p . grad T + s_i (T - T_L) = 0.

Write the full system as A(s) X = b with X = (T_o, T_L, T_w) and
kappa = q . X + q0 (the upwinded hot-contact flux).  Then
    d kappa / d s_i = - Lambda^T (dA/ds_i) X,   A^T Lambda = q.
Only the E1 rows of cell i depend on s_i (coefficient +1 on T_oi, -1 on T_Li),
so with lambda_o the part of Lambda on the E1 rows,
    d kappa / d s_i = - sum_o lambda_oi (T_oi - T_Li).
Splitting Lambda = (lambda_o, mu, nu) by block rows gives
    A_o^T lambda_o = q_o + a_o mu + C_o^T nu         (transposed transport)
    mu_i = s_i sum_o lambda_oi                         (column of T_L)
    nu_f = sum_{o entering from wall f} beta_o lambda_o,i(f)   (column of T_w)
where C_o holds the E3 weights.  The transposed per-ordinate systems are
solved with the same sparse LU factors (``trans='T'``) and the reduced
adjoint unknowns (mu, nu) by GMRES, mirroring mode B of the forward oracle.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from . import bte


def kappa_functional(prob: bte.Problem):
    """q_o: coefficients of kappa on T_o (one vector per ordinate, dict): the
    hot-contact flux of Eq. keff (App. A) as a linear functional."""
    me, od = prob.mesh, prob.ords
    g = me.grad_axis
    scale = me.lengths[g] / (me.delta_T * me.n_sec)
    cells0, img = me.hot_faces()
    q = {}
    for o in range(od.n):
        v = np.zeros(me.nc)
        kx = od.K[o, g]
        if kx > 0:
            np.add.at(v, img, scale * kx)
        elif kx < 0:
            np.add.at(v, cells0, scale * kx)
        q[o] = v
    return q


class Adjoint:
    """Adjoint of the discrete system E1-E3 (module docstring): transposed
    per-ordinate solves and GMRES on the reduced unknowns (mu, nu)."""
    def __init__(self, prob: bte.Problem, tr: bte.Transport = None):
        self.prob = prob
        self.tr = tr or bte.Transport(prob)
        self.q = kappa_functional(prob)
        me = prob.mesh
        self.wc = me.walls[:, 0]
        self.wa = me.walls[:, 1]
        self.ws = me.walls[:, 2]

    def lam_o(self, o, mu, nu, with_q=True):
        """Solve A_o^T lambda_o = q_o + a_o mu + C_o^T nu."""
        tr, od = self.tr, self.prob.ords
        r = od.a[o] * mu
        if with_q:
            r = r + self.q[o]
        cw = tr.w_out[o] / tr.w_den                      # E3 weights c_{f,o}
        np.add.at(r, self.wc, cw * nu)
        return tr.lu(o).solve(r, trans="T")

    def reduced(self, mu, nu, with_q=True, keep=False):
        """(mu, nu) -> (s sum_o lambda_o, sum_o B_o^T lambda_o)."""
        me, od = self.prob.mesh, self.prob.ords
        mu_new = np.zeros(me.nc)
        nu_new = np.zeros(me.nw)
        lams = {} if keep else None
        for o in range(od.n):
            lam = self.lam_o(o, mu, nu, with_q)
            mu_new += lam
            # walls this ordinate enters from: side sgn with sgn * p_a < 0
            pa = od.p[o, self.wa]
            enter = self.ws * pa < 0
            beta = od.lam[o] * np.abs(pa) / np.array(me.h)[self.wa]
            nu_new += np.where(enter, beta * lam[self.wc], 0.0)
            if keep:
                lams[o] = lam
        mu_new *= self.prob.s
        return mu_new, nu_new, lams

    def solve(self, rtol=1e-12, restart=60, maxiter=400):
        """GMRES on (mu, nu), the adjoint counterpart of the forward mode B
        (Algorithm 1's fixed point solved by a Krylov method)."""
        me = self.prob.mesh
        n1, n2 = me.nc, me.nw
        b_mu, b_nu, _ = self.reduced(np.zeros(n1), np.zeros(n2), with_q=True)
        b = np.concatenate([b_mu, b_nu])

        def matvec(y):
            m, n, _ = self.reduced(y[:n1], y[n1:], with_q=False)
            return y - np.concatenate([m, n])

        op = spla.LinearOperator((n1 + n2, n1 + n2), matvec=matvec, dtype=float)
        y, info = spla.gmres(op, b, rtol=rtol, atol=0.0, restart=restart, maxiter=maxiter)
        self.mu, self.nu = y[:n1], y[n1:]
        _, _, self.lams = self.reduced(self.mu, self.nu, with_q=True, keep=True)
        return self.lams


def kappa_grad_s(prob: bte.Problem, sol: bte.Solution = None, tr=None, rtol=1e-12):
    """d kappa_eff / d s_i for every solid cell i (adjoint method)."""
    tr = tr or bte.Transport(prob)
    if sol is None:
        sol = bte.solve_mode_B(prob, tr=tr, rtol=rtol)
    fw = tr.sweep(sol.T_L, sol.T_w, keep_T=True)
    adj = Adjoint(prob, tr)
    lams = adj.solve(rtol=rtol)
    g = np.zeros(prob.mesh.nc)
    for o, T in fw["T"].items():
        g -= lams[o] * (T - sol.T_L)
    return g, {"forward": fw, "adjoint": adj, "solution": sol}


def reversed_ordinate(ords: bte.Ordinates):
    """Index of the ordinate with the same MFP bin and MFP and the opposite
    direction."""
    rev = np.empty(ords.n, dtype=np.int64)
    for o in range(ords.n):
        cand = np.nonzero((ords.m_of == ords.m_of[o]) &
                          (np.abs(ords.lam - ords.lam[o]) <= 1e-12 * ords.lam[o]) &
                          np.all(np.abs(ords.p + ords.p[o]) < 1e-12, axis=1))[0]
        if len(cand) != 1:
            raise ValueError("quadrature is not symmetric under p -> -p")
        rev[o] = cand[0]
    return rev


def adjoint_jump(prob: bte.Problem):
    """Temperature jump whose forward solution, with directions reversed,
    reproduces lambda_o / a_o: -(L_x / (dT N_sec)) d_ang h_x sum_m kappa_m / Lambda_m^2.
    (q_o / a_o at a hot-contact cell equals beta_ox times this jump.)"""
    me, od = prob.mesh, prob.ords
    g = me.grad_axis
    scale = me.lengths[g] / (me.delta_T * me.n_sec)
    # recover the total weight from the ordinate table: K_o / (a_o Lambda_o p_o)
    # = sum_o W_o for every o (d_ang sum_m kappa_m / Lambda_m^2 for the
    # bin x direction material)
    o = int(np.argmax(np.abs(od.p[:, g])))
    ratio = od.K[o, g] / (od.a[o] * od.lam[o] * od.p[o, g])
    return -scale * ratio * me.h[g]
