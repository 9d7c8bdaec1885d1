"""A model of the mixed-precision mode's rounding, built on the FP64 oracle
(test helper, CPU).

A float sweep stores App. A's upwind coefficients of E1, divided by its
diagonal: A_a = fl(fl(beta_a) A0) with A0 = 1 / (1 + D).  Written as
T_i = A0 s_i T_L,i + sum_a A_a u_a with A0 = fl(1 / (1 + D)) (the first
mixed sweeps), the weight of T_L is a rounded number of its own; written in
delta form T_i = T_L,i + sum_a A_a (u_a - T_L,i) (the current sweeps, which
carry psi = T - T_L), it is 1 - sum_a A_a exactly.  ``RoundedCoefficients`` is the oracle's transport
with such rounded coefficients and everything else exact, so its FP64 fixed
point shows what the rounding of the coefficients alone does;
``DeltaCoefficients`` the same for the delta form, optionally with the E2
weights a_o rounded to float as well.  ``FloatTransport`` instead solves each
ordinate in float32 (sparse LU) with the moments in FP64.  ``quantised_iteration``
runs Algorithm 1 with exact solves but float-rounded carried values, either
T_o itself (and the source s T_L) or the deviation psi_o = T_o - T_L: the
first stalls where the slow diffusive mode's step falls below the float
quantum, the second does not.
"""
import copy

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import bte

f32 = np.float32


class RoundedCoefficients(bte.Transport):
    """E1 with float-rounded coefficients.  ``which`` picks what is rounded:
    "A0", "Aa" (A_x, A_y, A_z) or both; ``bins`` limits the rounding to
    those MFP bins (None: all)."""

    def __init__(self, prob, which=("A0", "Aa"), bins=None):
        super().__init__(prob)
        self.which = which
        self.bins = bins

    def _coef(self, o):
        b = self.beta(o)
        me = self.prob.mesh
        a0 = 1.0 / (1.0 + sum(b[a] for a in me.axes))
        rounded = self.bins is None or self.prob.ords.m_of[o] in self.bins
        if rounded and "Aa" in self.which:
            A = [float(f32(float(f32(b[a])) * float(f32(a0)))) for a in range(3)]
        else:
            A = [b[a] * a0 for a in range(3)]
        if rounded and "A0" in self.which:
            a0 = float(f32(a0))
        return a0, A

    def matrix(self, o):
        me, od = self.prob.mesh, self.prob.ords
        _, A = self._coef(o)
        rows, cols, vals = [np.arange(me.nc)], [np.arange(me.nc)], [np.ones(me.nc)]
        for a in me.axes:
            if od.p[o, a] == 0.0:
                continue
            j = me.nbr[:, a, 0 if od.p[o, a] > 0 else 1]
            ok = j >= 0
            rows.append(np.nonzero(ok)[0])
            cols.append(j[ok])
            vals.append(np.full(ok.sum(), -A[a]))
        return sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(me.nc, me.nc))

    def rhs(self, o, T_L, T_w, with_jump=True):
        me, od = self.prob.mesh, self.prob.ords
        a0, A = self._coef(o)
        r = a0 * self.prob.s * T_L
        for a in me.axes:
            if od.p[o, a] == 0.0:
                continue
            side = 0 if od.p[o, a] > 0 else 1
            if with_jump:
                r = r + A[a] * me.jump[:, a, side]
            wid = me.wall[:, a, side]
            ok = wid >= 0
            if ok.any():
                r[ok] += A[a] * T_w[wid[ok]]
        return r


class DeltaCoefficients(RoundedCoefficients):
    """E1 as the delta-form float sweep has it: A_a rounded as above, the
    weight of s_i T_L exactly 1 - sum_a A_a."""

    def __init__(self, prob):
        super().__init__(prob, which=("Aa",))

    def _coef(self, o):
        _a0, A = super()._coef(o)
        return 1.0 - sum(A[a] for a in self.prob.mesh.axes), A


def delta_form_floor(pr, ref, float_weights=True):
    """max |T_L - T_L*| for the delta-form coefficients (and, with
    ``float_weights``, the E2 weights a_o rounded to float as the sweep holds
    them)."""
    p2 = copy.deepcopy(pr)
    if float_weights:
        p2.ords.a = p2.ords.a.astype(f32).astype(np.float64)
    sol = bte.solve_mode_B(p2, rtol=1e-13, tr=DeltaCoefficients(p2))
    return float(np.abs(sol.T_L - ref.T_L).max())


class FloatTransport(bte.Transport):
    """Each ordinate's E1 solved in float32 (sparse LU of the float matrix,
    float right-hand side); the moments stay FP64."""

    def lu(self, o):
        f = self._lu.get(o)
        if f is None:
            f = spla.splu(self.matrix(o).astype(np.float32))
            self._lu[o] = f
        return f

    def solve_ordinate(self, o, T_L, T_w, with_jump=True):
        r = self.rhs(o, T_L, T_w, with_jump).astype(np.float32)
        return self.lu(o).solve(r).astype(np.float64)


def float_coefficient_floor(pr, ref, which=("A0", "Aa"), bins=None):
    """max |T_L - T_L*| between the exact fixed point ``ref`` and the FP64
    fixed point of E1-E4 with the float-rounded coefficients."""
    sol = bte.solve_mode_B(pr, rtol=1e-13, tr=RoundedCoefficients(pr, which, bins))
    return float(np.abs(sol.T_L - ref.T_L).max())


def tall_cell(ny, nx=16, length=100e-9):
    """The tall test cell of the fixed-rows warp variants: nx x ny cells,
    L x (L ny / nx), one square pore of porosity 0.1, two MFP bins (1 nm and
    10 um), 16 in-plane directions."""
    from paper_2106_02764_gb300 import inputs as I
    Ly = length * ny / nx
    wl = I.make_2d(f"tall{ny}", nx, length, [], 2, I.circle_quadrature(16))
    wl.mask = I.pores_mask(nx, ny, length, Ly, [I.square_pore(length, Ly, 0.1, x=0.35 * length,
                                                              y=0.6 * Ly)])
    wl.shape = (nx, ny, 1)
    wl.lengths = (length, Ly, 0.0)
    return wl


def quantised_iteration(pr, n_iter, form, run=32):
    """Algorithm 1 from the Fourier first guess with the per-ordinate solves
    exact and the values a float sweep would carry rounded to float: form
    "T" rounds the source T_L and every T_o; form "psi" rounds only
    psi_o = T_o - T_L (T_L and the moments stay FP64); form "psi_sums" also
    forms the moment partial sum_o a_o psi_o of each run of ``run``
    consecutive ordinates in float (sequential float32 adds, float a_o), as
    the sweep's per-lane and block-combined partials are, before the FP64
    accumulation.  Returns max |T_L - T_L*| against the exact fixed point
    after n_iter iterations (gauged)."""
    ref = bte.solve_mode_B(pr, rtol=1e-13)
    tr = bte.Transport(pr)
    me, od = pr.mesh, pr.ords
    wc = me.walls[:, 0]
    T_L, T_w = bte.initial_guess(tr)
    for _ in range(n_iter):
        src = T_L.astype(f32).astype(np.float64) if form == "T" else T_L
        TL_new, wn = np.zeros(me.nc), np.zeros(me.nw)
        part = np.zeros(me.nc, dtype=f32)
        for o in range(od.n):
            T = tr.lu(o).solve(tr.rhs(o, src, T_w))
            if form == "psi_sums":
                psi = (T - T_L).astype(f32)
                part = part + f32(od.a[o]) * psi          # float32 multiply-add
                if (o + 1) % run == 0 or o + 1 == od.n:
                    TL_new += part.astype(np.float64)
                    part = np.zeros(me.nc, dtype=f32)
                T = T_L + psi.astype(np.float64)
            else:
                T = T.astype(f32).astype(np.float64) if form == "T" else \
                    T_L + (T - T_L).astype(f32).astype(np.float64)
                TL_new += od.a[o] * T
            wn += tr.w_out[o] * T[wc]
        if form == "psi_sums":
            TL_new += T_L      # sum_o a_o = 1: T_L added back in FP64
        T_L, T_w = TL_new, wn / tr.w_den
    return float(np.abs(bte.gauge(T_L, T_w)[0] - ref.T_L).max())
