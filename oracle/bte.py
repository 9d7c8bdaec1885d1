"""FP64 oracle: upwind finite-volume aMFP-BTE on a periodic Cartesian voxel mesh.

TEST INFRASTRUCTURE ONLY (see the package docstring): never imported by the
product path.

What is computed (the discrete system, App. A of the paper):

  (E1)  for every ordinate o = (m, s) and solid cell i
          (s_i + sum_a Lambda_m |p_a| / h_a) T_oi
              - sum_{inflow faces f} (Lambda_m |p_a| / h_a) u_of  =  s_i T_Li
        The outgoing flux of every face sits on the diagonal (App. A, first
        sentence; Eq. iter2 with A_l).  u_of is the upwind value across face f:
          * T_o of the solid neighbour (periodic images included), plus the
            jump of the applied gradient: +dT when the neighbour is the image
            across the low side of the gradient axis, -dT across the high side
            (R^P and P_il of App. A);
          * the wall temperature T_wf when the neighbour is a pore or a
            non-periodic boundary (diffuse wall, B term of Eq. iter2).
  (E2)  T_Li = sum_o a_o T_oi with a_o = abar_m w_s,
        abar_m = (kappa_m / Lambda_m^2) / sum_m' (kappa_m' / Lambda_m'^2)
        (lattice temperature from energy conservation, Sec. 2; C/tau per bin
        is proportional to kappa_m / Lambda_m^2 for a gray bin).  A general
        per-ordinate material (Ordinates.from_ordinates) gives each ordinate
        its own Lambda_o and weight W_o: a_o = W_o / sum W, K_o = W_o F_o.
  (E3)  T_wf = sum_{o: K_o.n_f > 0} (K_o.n_f) T_o,i(f) / sum_{o: K_o.n_f > 0} K_o.n_f
        with K_o = d_ang kappa_m w_s p_s / Lambda_m the flux weight
        (thermalising wall, R_mu_nu of Sec. 2; S_ml of App. A).
  (E4)  gauge: sum over solid cells of T_L = 0 (the system is singular up to a
        common shift of all temperatures; the paper does not say how it fixes
        it).
  kappa_eff: upwinded heat flux through the solid faces of the plane x = 0
        (Eq. keff and its hot-contact form in App. A):
          kappa = L_x / (dT * N_sec) * sum_faces [ sum_{p_x>0} K_ox (T_o,img + dT)
                                                 + sum_{p_x<0} K_ox T_o,cell ]
        with N_sec the number of cells in a full cross-section (pores included).
        The dT term is the kappa_bal / 2 of App. A; the rest is K^T T.

How it is computed: per ordinate, the sparse matrix of E1 with the periodic
neighbours kept implicit is factorised by SciPy's sparse LU (Sec. 3: LU
factorisations reused across iterations; A_ml = I + Lambda_m A_l assembled on
the fly).  Walls and T_L are lagged as in Eq. iter2.

  mode A  -- Algorithm 1: T_L, T_w from iteration n-1, solve all ordinates,
             update T_L, T_w and kappa, stop when |d kappa| / kappa < tol.
  mode B  -- the same fixed point solved by GMRES on the reduced unknowns
             x = (T_L, T_w): x - M_lin(x) = M(0), where one application of M is
             one pass of mode A.  Used as the parity reference.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


# ---------------------------------------------------------------------------
# mesh: solid cells, neighbours, jumps and wall faces
# ---------------------------------------------------------------------------
class Mesh:
    """Cartesian voxel mesh; cells numbered over solid voxels in (z, y, x)
    order with x fastest.  Faces follow App. A: R_ij between neighbours,
    R^P_ij between periodic images, g_si at walls."""

    def __init__(self, mask, lengths, periodic, delta_T, dim, grad_axis=0):
        mask = np.asarray(mask).astype(bool)
        if mask.ndim == 2:
            mask = mask[None]
        nz, ny, nx = mask.shape
        if dim == 2 and nz != 1:
            raise ValueError("2D mesh needs nz = 1")
        if not periodic[grad_axis]:
            raise ValueError("the gradient axis must be periodic")
        self.mask = mask
        self.dim = dim
        self.n = (nx, ny, nz)
        self.lengths = tuple(float(v) for v in lengths)
        self.h = (lengths[0] / nx, lengths[1] / ny, (lengths[2] / nz) if dim == 3 else 1.0)
        self.periodic = tuple(int(v) for v in periodic)
        self.delta_T = float(delta_T)
        self.grad_axis = grad_axis
        self.axes = (0, 1) if dim == 2 else (0, 1, 2)

        zz, yy, xx = np.nonzero(mask)             # C order: x fastest
        self.coords = np.stack([xx, yy, zz], axis=1)
        self.nc = len(xx)
        index = -np.ones(mask.shape, dtype=np.int64)
        index[zz, yy, xx] = np.arange(self.nc)
        self.index = index

        # nbr[c, a, side]: side 0 = minus face, 1 = plus face
        self.nbr = -np.ones((self.nc, 3, 2), dtype=np.int64)
        self.jump = np.zeros((self.nc, 3, 2))
        self.wall = -np.ones((self.nc, 3, 2), dtype=np.int64)
        walls = []
        for a in self.axes:
            for side, sgn in ((0, -1), (1, +1)):
                q = self.coords.copy()
                q[:, a] += sgn
                outside = (q[:, a] < 0) | (q[:, a] >= self.n[a])
                jump = np.zeros(self.nc)
                if self.periodic[a]:
                    q[:, a] %= self.n[a]
                    if a == grad_axis:
                        # image across the low side is hotter by dT (P_il, R^P)
                        jump[outside] = self.delta_T if sgn < 0 else -self.delta_T
                    inside = np.ones(self.nc, dtype=bool)
                else:
                    inside = ~outside
                j = -np.ones(self.nc, dtype=np.int64)
                qi = q[inside]
                j[inside] = index[qi[:, 2], qi[:, 1], qi[:, 0]]
                solid_nbr = j >= 0
                self.nbr[solid_nbr, a, side] = j[solid_nbr]
                self.jump[solid_nbr, a, side] = jump[solid_nbr]
                for c in np.nonzero(~solid_nbr)[0]:
                    self.wall[c, a, side] = len(walls)
                    walls.append((c, a, sgn))
        self.walls = np.array(walls, dtype=np.int64).reshape(-1, 3)
        self.nw = len(walls)
        # number of cells in a full cross-section normal to the gradient axis
        self.n_sec = int(np.prod([self.n[a] for a in self.axes if a != grad_axis]))

    def hot_faces(self):
        """Solid-solid faces on the periodic plane x_g = 0 of Eq. keff (App. A):
        (cell at x_g = 0,
        its periodic image neighbour)."""
        g = self.grad_axis
        at0 = self.coords[:, g] == 0
        cells = np.nonzero(at0 & (self.nbr[:, g, 0] >= 0))[0]
        return cells, self.nbr[cells, g, 0]

    def section_faces(self, i):
        """Solid-solid faces on the plane between columns i-1 and i of the
        gradient axis: (cell at column i, its minus-side neighbour, jump)."""
        g = self.grad_axis
        cells = np.nonzero((self.coords[:, g] == i) & (self.nbr[:, g, 0] >= 0))[0]
        return cells, self.nbr[cells, g, 0], self.jump[cells, g, 0]


# ---------------------------------------------------------------------------
# ordinates: (m, s) pairs with their transport and moment weights
# ---------------------------------------------------------------------------
class Ordinates:
    """o = m * S + s.  F_ml = Lambda_m s_l (App. A); D_ml and S_ml become the
    E2 weights a_o and the flux weights K_o."""

    def __init__(self, kappa_m, lambda_m, dirs, weights, angular_dim, dim):
        kappa_m = np.asarray(kappa_m, float)
        lambda_m = np.asarray(lambda_m, float)
        dirs = np.asarray(dirs, float)
        weights = np.asarray(weights, float)
        M, S = len(kappa_m), len(weights)
        self.M, self.S, self.n = M, S, M * S
        p = np.zeros((S, 3))
        p[:, :dim] = dirs[:, :dim]          # in 2D the z component drops out
        self.lam = np.repeat(lambda_m, S)
        self.p = np.tile(p, (M, 1))
        self.w = np.tile(weights, M)
        km = np.repeat(kappa_m, S)
        abar = (kappa_m / lambda_m ** 2) / np.sum(kappa_m / lambda_m ** 2)
        self.a = np.repeat(abar, S) * self.w
        self.K = angular_dim * (km * self.w / self.lam)[:, None] * self.p
        self.kappa_bulk = float(kappa_m.sum())
        # bulk conductivity along each axis (isotropic for these sets)
        self.kappa_axes = np.full(3, self.kappa_bulk)
        self.m_of = np.repeat(np.arange(M), S)
        self.s_of = np.tile(np.arange(S), M)

    @classmethod
    def from_ordinates(cls, lam, dirs, weight, bins, dim):
        """General aMFP material (Sec. 5, App. A): ordinate o carries its own
        vectorial MFP F_o = Lambda_o s_o and a weight W_o >= 0 standing for the
        C/tau of the modes interpolated onto it (D_ml of App. A before
        normalisation).  Then a_o = W_o / sum W (E2) and K_o = W_o Lambda_o s_o
        (S_ml of App. A, in the form for which sum_o K_o . grad T_o =
        -sum_o W_o (T_o - T_L) = 0 holds for the transport of every ordinate,
        i.e. energy is conserved).  The bin-separable set above is the case
        W_o = d_ang (kappa_m / Lambda_m^2) w_s."""
        self = cls.__new__(cls)
        lam = np.asarray(lam, float)
        W = np.asarray(weight, float)
        bins = np.asarray(bins, np.int64)
        n = len(lam)
        p = np.zeros((n, 3))
        p[:, :dim] = np.asarray(dirs, float).reshape(n, 3)[:, :dim]
        self.n, self.M, self.S = n, int(bins.max()) + 1, None
        self.lam, self.p = lam, p
        self.w = W / W.sum()
        self.a = W / W.sum()
        self.K = (W * lam)[:, None] * p
        # kappa_aa = sum_o K_oa Lambda_o p_oa: the response of the flux to a
        # uniform gradient along a (diagonal of the bulk tensor)
        self.kappa_axes = np.array([float((self.K[:, a] * lam * p[:, a]).sum()) for a in range(3)])
        self.kappa_bulk = float(self.kappa_axes[0])
        self.m_of = bins
        self.s_of = np.arange(n)
        return self


@dataclasses.dataclass
class Problem:
    """Inputs of E1-E4: the voxel mesh (Sec. 6, faces of App. A), the
    ordinates (Sec. 2 and App. A, F_ml = Lambda_m s_l) and the per-cell
    scattering scale s_i of E1 (1 unless a sensitivity is asked for)."""
    mesh: Mesh
    ords: Ordinates
    s: np.ndarray            # scattering scale per solid cell (E1), default 1

    @classmethod
    def from_workload(cls, wl, s=None):
        """Build E1-E4's inputs from a synthetic workload (mask, lengths,
        bins and quadrature, or a general per-ordinate material of Sec. 5)."""
        mesh = Mesh(wl.mask, wl.lengths, wl.periodic, wl.delta_T, wl.dim, wl.grad_axis)
        if getattr(wl, "ords", None) is not None:
            o = wl.ords
            ords = Ordinates.from_ordinates(o["lambda"], o["dirs"], o["weight"], o["bin"], wl.dim)
        else:
            ords = Ordinates(wl.kappa_m, wl.lambda_m, wl.quad.dirs, wl.quad.weights,
                             wl.quad.angular_dim, wl.dim)
        field = s if s is not None else wl.s
        if field is None:
            sv = np.ones(mesh.nc)
        else:
            field = np.asarray(field, float).reshape(wl.mask.shape)
            c = mesh.coords
            sv = field[c[:, 2], c[:, 1], c[:, 0]].copy()
        return cls(mesh, ords, sv)


# ---------------------------------------------------------------------------
# per-ordinate system (E1) and one pass of the source iteration
# ---------------------------------------------------------------------------
class Transport:
    """Per-ordinate sparse matrices of E1 with their LU factors (Sec. 3)."""

    def __init__(self, prob: Problem, cache: bool = True, cache_max: int = None):
        """E3 weights of the thermalising walls (Sec. 2): a wall face takes the
        flux-weighted mean sum_{K.n>0} (K_o.n) T_o / sum_{K.n>0} K_o.n of the
        ordinates leaving its cell into it.  ``cache_max`` bounds the number
        of LU factors kept (the rest are refactorised on every pass)."""
        self.prob = prob
        self.cache = cache
        self.cache_max = cache_max
        self._lu = {}
        me, od = prob.mesh, prob.ords
        # wall-face weights of E3: numerator weights per (wall, ordinate)
        wa = me.walls[:, 1]
        wsg = me.walls[:, 2]
        kn = od.K[:, wa] * wsg[None, :]                   # K_o . n_f, shape [O, Nw]
        self.w_out = np.maximum(kn, 0.0)                  # ordinates leaving into the wall
        den = self.w_out.sum(axis=0)
        self.w_den = np.where(den > 0, den, 1.0)

    def beta(self, o):
        """Upwind face coefficients Lambda_m |p_a| A_f / V_i = Lambda_m |p_a| / h_a
        of E1 (App. A, Eq. iter2 on a Cartesian cell)."""
        me, od = self.prob.mesh, self.prob.ords
        return np.array([od.lam[o] * abs(od.p[o, a]) / me.h[a] for a in range(3)])

    def matrix(self, o):
        """E1 left-hand side for ordinate o (CSC), periodic neighbours implicit."""
        me, od = self.prob.mesh, self.prob.ords
        b = self.beta(o)
        diag = self.prob.s + sum(b[a] for a in me.axes)
        rows, cols, vals = [np.arange(me.nc)], [np.arange(me.nc)], [diag]
        for a in me.axes:
            if od.p[o, a] == 0.0:
                continue
            side = 0 if od.p[o, a] > 0 else 1          # inflow face
            j = me.nbr[:, a, side]
            ok = j >= 0
            rows.append(np.nonzero(ok)[0])
            cols.append(j[ok])
            vals.append(np.full(ok.sum(), -b[a]))
        A = sp.csc_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(me.nc, me.nc))
        return A

    def lu(self, o):
        """Sparse LU of ordinate o's E1 matrix, kept across iterations when
        memory allows (Sec. 3: the factorisations are reused)."""
        f = self._lu.get(o)
        if f is None:
            f = spla.splu(self.matrix(o))
            if self.cache and (self.cache_max is None or len(self._lu) < self.cache_max):
                self._lu[o] = f
        return f

    def rhs(self, o, T_L, T_w, with_jump=True):
        """E1 right-hand side: s_i T_L + inflow jumps + inflow wall temperatures."""
        me, od = self.prob.mesh, self.prob.ords
        b = self.beta(o)
        r = self.prob.s * T_L
        for a in me.axes:
            if od.p[o, a] == 0.0:
                continue
            side = 0 if od.p[o, a] > 0 else 1
            if with_jump:
                r = r + b[a] * me.jump[:, a, side]
            wid = me.wall[:, a, side]
            ok = wid >= 0
            if ok.any():
                r[ok] += b[a] * T_w[wid[ok]]
        return r

    def solve_ordinate(self, o, T_L, T_w, with_jump=True):
        """One ordinate's transport solve of E1 (App. A, Eq. iter2) with T_L
        and the wall temperatures lagged (Algorithm 1)."""
        return self.lu(o).solve(self.rhs(o, T_L, T_w, with_jump))

    def flux_section(self, o, T, i=0, with_jump=True):
        """Upwinded x-flux of ordinate o through the solid faces of plane i
        (the flux of App. A's Eq. keff; equal on every plane by E2)."""
        me, od = self.prob.mesh, self.prob.ords
        g = me.grad_axis
        cells, img, jmp = me.section_faces(i)
        Kx = od.K[o, g]
        if Kx > 0:
            up = T[img] + (jmp if with_jump else 0.0)
        else:
            up = T[cells]
        return Kx * up.sum()

    def sweep(self, T_L, T_w, ords=None, with_jump=True, keep_T=False, sections=False,
              flux=False):
        """One pass of Algorithm 1's loop over ordinates (Sec. 3): solves E1 for
        each and returns partial moments
        (sum a_o T_o, wall numerators, x=0 face flux and its split by MFP bin
        [, per-section fluxes][, cell heat flux J = sum_o K_o T_o][, T])."""
        me, od = self.prob.mesh, self.prob.ords
        if ords is None:
            ords = range(od.n)
        TL_new = np.zeros(me.nc)
        wall_num = np.zeros(me.nw)
        phi = 0.0
        phi_bins = np.zeros(int(od.m_of.max()) + 1)
        phis = np.zeros(me.n[me.grad_axis]) if sections else None
        J = np.zeros((me.nc, 3)) if flux else None
        Ts = {} if keep_T else None
        wc = me.walls[:, 0]
        for o in ords:
            T = self.solve_ordinate(o, T_L, T_w, with_jump)
            TL_new += od.a[o] * T
            wall_num += self.w_out[o] * T[wc]
            f0 = self.flux_section(o, T, 0, with_jump)
            phi += f0
            phi_bins[od.m_of[o]] += f0
            if sections:
                for i in range(len(phis)):
                    phis[i] += self.flux_section(o, T, i, with_jump)
            if flux:
                J += T[:, None] * od.K[o][None, :]
            if keep_T:
                Ts[o] = T
        out = {"TL": TL_new, "wall_num": wall_num, "phi": phi, "phi_bins": phi_bins}
        if sections:
            out["phis"] = phis
        if flux:
            out["J"] = J[:, :me.dim]
        if keep_T:
            out["T"] = Ts
        return out

    def kappa_from_phi(self, phi, with_jump=True):
        """kappa_eff = L_x / (dT A_sec) times the upwinded flux through the plane
        x = 0 (App. A, Eq. keff in its hot-contact form); A_sec counts the
        cells of a full cross-section, pores included."""
        me = self.prob.mesh
        return me.lengths[me.grad_axis] / (me.delta_T * me.n_sec) * phi


# ---------------------------------------------------------------------------
# the fixed-point map M and the two solution modes
# ---------------------------------------------------------------------------
def apply_M(tr: Transport, T_L, T_w, with_jump=True, parts=None):
    """One pass of Algorithm 1: (T_L, T_w) of iteration n-1 -> iteration n,
    plus kappa of the ordinate fields just solved."""
    r = tr.sweep(T_L, T_w, with_jump=with_jump) if parts is None else parts
    TL = r["TL"]
    Tw = r["wall_num"] / tr.w_den
    kappa = tr.kappa_from_phi(r["phi"])
    return TL, Tw, kappa


def initial_guess(tr: Transport, T_F=None):
    """Algorithm 1, first line: T from Fourier's law; walls take the
    temperature of their cell."""
    from .fourier import solve_fourier
    me = tr.prob.mesh
    if T_F is None:
        T_F = solve_fourier(me, tr.prob.ords.kappa_axes)["T"]
    T_w = T_F[me.walls[:, 0]] if me.nw else np.zeros(0)
    return T_F.copy(), T_w.copy()


def gauge(T_L, T_w):
    """E4: shift every temperature so that the solid-cell mean of T_L is 0."""
    c = T_L.mean()
    return T_L - c, T_w - c, c


@dataclasses.dataclass
class Solution:
    """Fixed point of Algorithm 1 (Sec. 3): gauged T_L and T_w (E4), kappa_eff,
    the iterations or GMRES matrix products taken, the kappa history."""
    T_L: np.ndarray
    T_w: np.ndarray
    kappa: float
    iterations: int
    history: list
    residual: float = float("nan")


def solve_mode_A(prob: Problem, tol=1e-6, max_iter=100000, x0=None, tr=None,
                 apply=None, callback=None):
    """Algorithm 1 of the paper: source iteration with lagged T_L and walls,
    stopped when the relative change of kappa falls below ``tol``."""
    tr = tr or Transport(prob)
    T_L, T_w = initial_guess(tr) if x0 is None else (x0[0].copy(), x0[1].copy())
    apply = apply or (lambda a, b: apply_M(tr, a, b))
    hist = []
    kappa_old = None
    it = 0
    for it in range(1, max_iter + 1):
        T_L, T_w, kappa = apply(T_L, T_w)
        hist.append(kappa)
        if callback is not None:
            callback(it, T_L, T_w, kappa)
        if kappa_old is not None and abs(kappa - kappa_old) <= tol * abs(kappa):
            break
        kappa_old = kappa
    T_L, T_w, _ = gauge(T_L, T_w)
    return Solution(T_L, T_w, hist[-1], it, hist)


def solve_mode_B(prob: Problem, rtol=1e-12, restart=60, maxiter=400, tr=None, x0=None):
    """Parity reference: GMRES on the reduced unknowns (T_L, T_w) of the
    fixed point of Algorithm 1; then one more pass gives T_o and kappa."""
    tr = tr or Transport(prob)
    me = prob.mesh
    n1, n2 = me.nc, me.nw
    zL, zw = np.zeros(n1), np.zeros(n2)
    b_L, b_w, _ = apply_M(tr, zL, zw)                 # M(0): carries the dT source
    b = np.concatenate([b_L, b_w])

    def matvec(x):
        TL, Tw = x[:n1], x[n1:]
        r = tr.sweep(TL, Tw, with_jump=False)
        return x - np.concatenate([r["TL"], r["wall_num"] / tr.w_den])

    op = spla.LinearOperator((n1 + n2, n1 + n2), matvec=matvec, dtype=float)
    if x0 is None:
        T0, w0 = initial_guess(tr)
        x0 = np.concatenate([T0, w0])
    count = [0]

    def cb(_):
        count[0] += 1

    x, info = spla.gmres(op, b, x0=x0, rtol=rtol, atol=0.0, restart=restart,
                         maxiter=maxiter, callback=cb, callback_type="pr_norm")
    res = np.linalg.norm(op.matvec(x) - b) / max(np.linalg.norm(b), 1e-300)
    T_L, T_w, _ = gauge(x[:n1], x[n1:])
    TL2, Tw2, kappa = apply_M(tr, T_L, T_w)
    return Solution(T_L, T_w, kappa, count[0], [kappa], residual=res)


def fields(prob: Problem, sol: Solution, tr=None):
    """Ordinate fields T_o at the solution: one more pass of E1 (App. A)
    from its T_L and T_w, with the E2 / E3 numerators and section fluxes."""
    tr = tr or Transport(prob)
    return tr.sweep(sol.T_L, sol.T_w, keep_T=True, sections=True)


def heat_flux(prob: Problem, Ts: dict):
    """Cell heat flux J_i = sum_o K_o T_oi (Sec. 2, J = sum S_mu dT_mu)."""
    od = prob.ords
    J = np.zeros((prob.mesh.nc, 3))
    for o, T in Ts.items():
        J += T[:, None] * od.K[o][None, :]
    return J[:, :prob.mesh.dim]


def kappa_bins(prob: Problem, sol: Solution, tr=None):
    """Per-MFP-bin contributions to kappa_eff (the aMFP counterpart of the
    mode-resolved conductivity, Sec. 2 and App. A): the upwinded flux of Eq.
    keff through the plane x = 0 summed over the ordinates of each bin, times
    L_x / (dT A_sec).  They add up to kappa_eff."""
    tr = tr or Transport(prob)
    od = prob.ords
    Ts = tr.sweep(sol.T_L, sol.T_w, keep_T=True)["T"]
    out = np.zeros(int(od.m_of.max()) + 1)
    for o, T in Ts.items():
        out[od.m_of[o]] += tr.flux_section(o, T, 0)
    return tr.kappa_from_phi(out)


def kappa_bulk_discrete(prob: Problem):
    """Pore-free closed form of the upwind scheme: the exact discrete solution
    is T_o = T_L - Lambda_m p_x a (linear T_L of slope a = -dT/L_x), whose
    upwinded face flux gives kappa_bulk + (h_x / 2) sum_o |K_ox| (kappa_bulk:
    the bulk tensor's entry along the gradient axis)."""
    me, od = prob.mesh, prob.ords
    g = me.grad_axis
    return od.kappa_axes[g] + 0.5 * me.h[g] * np.abs(od.K[:, g]).sum()


def to_grid(prob: Problem, v, fill=np.nan):
    """Scatter a per-solid-cell vector onto the (nz, ny, nx) grid (layout only;
    no arithmetic of the method)."""
    me = prob.mesh
    out = np.full(me.mask.shape, fill, dtype=float)
    c = me.coords
    out[c[:, 2], c[:, 1], c[:, 0]] = v
    return out
