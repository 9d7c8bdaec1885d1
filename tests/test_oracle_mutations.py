"""Planted mistakes in the FP64 oracle must fail its pins (CPU).

Each test plants one plausible mistake for the duration of the test
(monkeypatch): in ``oracle.bte`` (a flipped jump sign, a term dropped from the E1
diagonal, wrong E2 or E3 weights, upwinding from the downwind side, a lost
scattering scale on the right-hand side, a wrong angular dimension in the
flux weights), in ``oracle.fourier`` (jump sign, conducting pore walls, the
hot-face flux read from the wrong side) or in ``oracle.adjoint`` (an
untransposed solve, a lost s_i in the T_L column, wall couplings taken from
the leaving side).  It then checks that the pin that guards that part of the
method fails.  A control test runs the same pins on the unmodified
oracle.  The pins here recompute what they need (flux weights from the
workload, the dense brute-force system from ``oracle.dense``) instead of
reading it back from the oracle under test.
"""
import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I
from oracle import bte, dense

L = 100e-9


def _solve(wl):
    pr = bte.Problem.from_workload(wl)
    return pr, bte.solve_mode_B(pr, rtol=1e-12, maxiter=20)


def _flux_weights(wl):
    """K_o = d_ang kappa_m w_s p_s / Lambda_m (Sec. 2), from the workload."""
    q = wl.quad
    K = []
    for k, lam in zip(wl.kappa_m, wl.lambda_m):
        for p, w in zip(q.dirs, q.weights):
            K.append(q.angular_dim * k * w * np.asarray(p[:3], float) / lam)
    K = np.array(K)
    if wl.dim == 2:
        K[:, 2] = 0.0
    return K


def pin_porefree(quad):
    """Pore-free closed form: kappa = kappa_bulk + (h/2) sum_o |K_ox| and T_L
    linear with slope -dT/L."""
    wl = I.make_2d("pf", 8, L, [], 3, quad)
    pr, sol = _solve(wl)
    K = _flux_weights(wl)
    h = L / 8
    expect = float(np.sum(wl.kappa_m)) + 0.5 * h * np.abs(K[:, 0]).sum()
    x = (pr.mesh.coords[:, 0] + 0.5) * h
    lin = -(x - x.mean()) / L
    return abs(sol.kappa - expect) < 1e-10 * expect and np.abs(sol.T_L - lin).max() < 1e-10


def _porous_4x4(s_seed=None):
    wl = I.small_2d(n=4, porosity=0, n_bins=2, n_phi=8, s_seed=s_seed)
    wl.mask = np.ones((1, 4, 4), np.uint8)
    wl.mask[0, 1:3, 1:3] = 0
    return wl


def pin_dense(s_seed=None):
    """The oracle's kappa and T_L equal the dense brute-force solve."""
    wl = _porous_4x4(s_seed)
    pr, sol = _solve(wl)
    d = dense.dense_from_workload(wl)
    return abs(sol.kappa - d["kappa"]) < 1e-9 * abs(d["kappa"]) and np.abs(sol.T_L - d["T_L"]).max() < 1e-9


def pin_conservation():
    """Every cell's upwinded face fluxes balance and every wall face carries
    zero net flux (E2, E3), with K recomputed from the workload."""
    wl = I.small_2d(n=8, porosity=0.2, n_bins=2, n_phi=8)
    pr, sol = _solve(wl)
    me = pr.mesh
    K = _flux_weights(wl)
    Ts = bte.fields(pr, sol)["T"]
    div = np.zeros(me.nc)
    wall_net = np.zeros(me.nw)
    for o, T in Ts.items():
        for a in me.axes:
            k = K[o, a] / me.h[a]
            for side, sgn in ((0, -1), (1, 1)):
                kn = k * sgn
                j = me.nbr[:, a, side]
                f = me.wall[:, a, side]
                if kn > 0:
                    up = T
                else:
                    up = np.where(j >= 0, T[np.maximum(j, 0)] + me.jump[:, a, side],
                                  sol.T_w[np.maximum(f, 0)])
                div += kn * up
                wf = f >= 0
                np.add.at(wall_net, f[wf], (kn * up)[wf])
    scale = np.abs(K).sum() / me.h[0]
    return np.abs(div).max() < 1e-9 * scale and np.abs(wall_net).max() < 1e-9 * scale


def all_pins():
    return {
        "porefree_circle": pin_porefree(I.circle_quadrature(8)),
        "porefree_projected": pin_porefree(I.projected_quadrature(8, 4)),
        "dense": pin_dense(),
        "dense_s": pin_dense(s_seed=3),
        "conservation": pin_conservation(),
    }


def test_control_all_pins_pass():
    r = all_pins()
    assert all(r.values()), r


# ----------------------------------------------------------------- mutations
def _jump_flipped(monkeypatch):
    orig = bte.Mesh.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        self.jump = -self.jump
    monkeypatch.setattr(bte.Mesh, "__init__", init)


def _upwind_from_downwind_side(monkeypatch):
    orig = bte.Mesh.__init__

    def init(self, *a, **k):
        orig(self, *a, **k)
        self.nbr = self.nbr[:, :, ::-1].copy()
        self.jump = self.jump[:, :, ::-1].copy()
        self.wall = self.wall[:, :, ::-1].copy()
    monkeypatch.setattr(bte.Mesh, "__init__", init)


def _wall_outflow_off_diagonal(monkeypatch):
    """Outgoing flux into a wall face left off the E1 diagonal."""
    orig = bte.Transport.matrix

    def matrix(self, o):
        A = orig(self, o).tolil()
        me, od = self.prob.mesh, self.prob.ords
        b = self.beta(o)
        for a in me.axes:
            if od.p[o, a] == 0.0:
                continue
            out = 1 if od.p[o, a] > 0 else 0
            for c in np.nonzero(me.wall[:, a, out] >= 0)[0]:
                A[c, c] -= b[a]
        return A.tocsc()
    monkeypatch.setattr(bte.Transport, "matrix", matrix)


def _TL_weights_without_inverse_lambda_squared(monkeypatch):
    orig = bte.Ordinates.__init__

    def init(self, kappa_m, lambda_m, dirs, weights, angular_dim, dim):
        orig(self, kappa_m, lambda_m, dirs, weights, angular_dim, dim)
        km = np.asarray(kappa_m, float)
        self.a = np.repeat(km / km.sum(), self.S) * self.w
    monkeypatch.setattr(bte.Ordinates, "__init__", init)


def _wall_temperature_from_every_ordinate(monkeypatch):
    orig = bte.Transport.__init__

    def init(self, prob, cache=True):
        orig(self, prob, cache)
        me, od = prob.mesh, prob.ords
        kn = od.K[:, me.walls[:, 1]] * me.walls[:, 2][None, :]
        self.w_out = np.abs(kn)
        den = self.w_out.sum(axis=0)
        self.w_den = np.where(den > 0, den, 1.0)
    monkeypatch.setattr(bte.Transport, "__init__", init)


def _scattering_scale_dropped_from_rhs(monkeypatch):
    orig = bte.Transport.rhs

    def rhs(self, o, T_L, T_w, with_jump=True):
        return orig(self, o, T_L, T_w, with_jump) - (self.prob.s - 1.0) * T_L
    monkeypatch.setattr(bte.Transport, "rhs", rhs)


def _flux_weights_with_planar_angular_dim(monkeypatch):
    orig = bte.Ordinates.__init__

    def init(self, kappa_m, lambda_m, dirs, weights, angular_dim, dim):
        orig(self, kappa_m, lambda_m, dirs, weights, angular_dim, dim)
        if angular_dim == 3:
            self.K = self.K * (2.0 / 3.0)
    monkeypatch.setattr(bte.Ordinates, "__init__", init)


@pytest.mark.parametrize("plant,caught_by", [
    (_jump_flipped, "porefree_circle"),
    (_upwind_from_downwind_side, "porefree_circle"),
    (_wall_outflow_off_diagonal, "conservation"),
    (_TL_weights_without_inverse_lambda_squared, "conservation"),
    (_wall_temperature_from_every_ordinate, "conservation"),
    (_scattering_scale_dropped_from_rhs, "dense_s"),
    (_flux_weights_with_planar_angular_dim, "porefree_projected"),
])
def test_planted_mistake_fails_a_pin(monkeypatch, plant, caught_by):
    plant(monkeypatch)
    r = all_pins()
    assert not r[caught_by], r


# ----------------------------------------------------------------- Fourier model (App. B)
from oracle import adjoint, fourier  # noqa: E402


def fourier_pins():
    """Pore-free: kappa_fourier = kappa_bulk and T linear.  Circular pore
    (phi = 0.1, 128^2): Eucken-Maxwell (1 - phi)/(1 + phi) within 1 %."""
    wl = I.make_2d("pf", 16, L, [], 1, I.circle_quadrature(4))
    me = bte.Mesh(wl.mask, wl.lengths, wl.periodic, 1.0, 2)
    r = fourier.solve_fourier(me, 150.0)
    x = (me.coords[:, 0] + 0.5) / 16
    porefree = abs(r["kappa"] - 150.0) < 1e-10 and np.abs(r["T"] + (x - x.mean())).max() < 1e-12
    wl = I.make_2d("em", 128, L, [I.circle_pore(L, L, 0.1)], 1, I.circle_quadrature(4))
    me = bte.Mesh(wl.mask, wl.lengths, wl.periodic, 1.0, 2)
    k = fourier.solve_fourier(me, 150.0)["kappa"] / 150.0
    ph = wl.porosity
    em = abs(k / ((1 - ph) / (1 + ph)) - 1) < 0.01
    return {"fourier_porefree": porefree, "eucken_maxwell": em}


def test_control_fourier_pins_pass():
    r = fourier_pins()
    assert all(r.values()), r


def _fourier_jump_sign(monkeypatch):
    orig = fourier.assemble

    def assemble(mesh, kappa_bulk):
        A, rhs = orig(mesh, kappa_bulk)
        return A, -rhs
    monkeypatch.setattr(fourier, "assemble", assemble)


def _fourier_walls_conducting(monkeypatch):
    """Pore faces held at T = 0 instead of adiabatic."""
    orig = fourier.assemble

    def assemble(mesh, kappa_bulk):
        A, rhs = orig(mesh, kappa_bulk)
        A = A.tolil()
        for a in mesh.axes:
            G = 150.0 / mesh.h[a] ** 2
            for side in (0, 1):
                for c in np.nonzero(mesh.wall[:, a, side] >= 0)[0]:
                    A[c, c] -= G
        return A.tocsr(), rhs
    monkeypatch.setattr(fourier, "assemble", assemble)


def _fourier_flux_wrong_side(monkeypatch):
    """Hot-face flux with the jump on the cell's side instead of the image's."""
    def kappa_fourier(mesh, kappa_bulk, T):
        g = mesh.grad_axis
        cells, img = mesh.hot_faces()
        jump = mesh.jump[cells, g, 0]
        flux = fourier._axes(kappa_bulk)[g] * (T[img] - jump - T[cells]) / mesh.h[g]
        return mesh.lengths[g] / (mesh.delta_T * mesh.n_sec) * flux.sum()
    monkeypatch.setattr(fourier, "kappa_fourier", kappa_fourier)


@pytest.mark.parametrize("plant,caught_by", [
    (_fourier_jump_sign, "fourier_porefree"),
    (_fourier_walls_conducting, "eucken_maxwell"),
    (_fourier_flux_wrong_side, "fourier_porefree"),
])
def test_planted_fourier_mistake_fails_a_pin(monkeypatch, plant, caught_by):
    plant(monkeypatch)
    r = fourier_pins()
    assert not r[caught_by], r


# ----------------------------------------------------------------- adjoint gradient
def adjoint_pin():
    """d kappa / d s_i against central differences of the converged kappa on
    three seeded cells (6 x 6 cell, circular pore, s ~ U[0.5, 2])."""
    wl = I.small_2d(n=6, porosity=0.15, n_bins=2, n_phi=8, s_seed=7)
    pr = bte.Problem.from_workload(wl)
    g, _ = adjoint.kappa_grad_s(pr, rtol=1e-13)
    h = 1e-5
    ok = True
    for i in np.random.default_rng(5).choice(pr.mesh.nc, size=3, replace=False):
        sp_, sm_ = pr.s.copy(), pr.s.copy()
        sp_[i] += h
        sm_[i] -= h
        kp = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, sp_), rtol=1e-14).kappa
        km = bte.solve_mode_B(bte.Problem(pr.mesh, pr.ords, sm_), rtol=1e-14).kappa
        ok = ok and abs((kp - km) / (2 * h) - g[i]) < 1e-5 * np.abs(g).max()
    return ok


def test_control_adjoint_pin_passes():
    assert adjoint_pin()


def _adjoint_not_transposed(monkeypatch):
    def lam_o(self, o, mu, nu, with_q=True):
        tr, od = self.tr, self.prob.ords
        r = od.a[o] * mu
        if with_q:
            r = r + self.q[o]
        np.add.at(r, self.wc, tr.w_out[o] / tr.w_den * nu)
        return tr.lu(o).solve(r)
    monkeypatch.setattr(adjoint.Adjoint, "lam_o", lam_o)


def _adjoint_TL_column_without_s(monkeypatch):
    orig = adjoint.Adjoint.reduced

    def reduced(self, mu, nu, with_q=True, keep=False):
        m, n, lams = orig(self, mu, nu, with_q, keep)
        return m / self.prob.s, n, lams
    monkeypatch.setattr(adjoint.Adjoint, "reduced", reduced)


def _adjoint_wall_column_from_leaving_side(monkeypatch):
    def reduced(self, mu, nu, with_q=True, keep=False):
        me, od = self.prob.mesh, self.prob.ords
        mu_new, nu_new = np.zeros(me.nc), np.zeros(me.nw)
        lams = {} if keep else None
        for o in range(od.n):
            lam = self.lam_o(o, mu, nu, with_q)
            mu_new += lam
            pa = od.p[o, self.wa]
            leave = self.ws * pa > 0
            beta = od.lam[o] * np.abs(pa) / np.array(me.h)[self.wa]
            nu_new += np.where(leave, beta * lam[self.wc], 0.0)
            if keep:
                lams[o] = lam
        return mu_new * self.prob.s, nu_new, lams
    monkeypatch.setattr(adjoint.Adjoint, "reduced", reduced)


@pytest.mark.parametrize("plant", [_adjoint_not_transposed, _adjoint_TL_column_without_s,
                                   _adjoint_wall_column_from_leaving_side])
def test_planted_adjoint_mistake_fails_the_pin(monkeypatch, plant):
    plant(monkeypatch)
    assert not adjoint_pin()


# ----------------------------------------------------------------- cell heat flux J (Sec. 2)
def flux_pins():
    """Pore-free: J = (kappa_bulk dT / L_x, 0) in every cell.  With a pore:
    the section identity of sum_i J_x,i (test_oracle_pins) and the y mirror
    symmetry of a centred pore."""
    from test_oracle_pins import _flux_section_identity
    wl = I.make_2d("pf", 8, L, [], 3, I.circle_quadrature(8))
    pr, sol = _solve(wl)
    J = bte.heat_flux(pr, bte.fields(pr, sol)["T"])
    expect = float(np.sum(wl.kappa_m)) / L
    porefree = np.abs(J[:, 0] - expect).max() < 1e-9 * expect and np.abs(J[:, 1]).max() < 1e-9 * expect
    lhs, rhs, pr, J = _flux_section_identity(I.small_2d(n=12, porosity=0.2, n_bins=3, n_phi=8))
    grid = np.full((12, 12), np.nan)
    c = pr.mesh.coords
    grid[c[:, 1], c[:, 0]] = J[:, 1]
    mirror = np.nanmax(np.abs(grid + grid[::-1])) < 1e-9 * np.abs(J[:, 0]).max()
    return {"flux_porefree": porefree, "flux_sections": abs(lhs - rhs) < 1e-10 * abs(lhs),
            "flux_mirror": bool(mirror)}


def test_control_flux_pins_pass():
    r = flux_pins()
    assert all(r.values()), r


def _flux_with_unsigned_weights(monkeypatch):
    def heat_flux(prob, Ts):
        J = np.zeros((prob.mesh.nc, 3))
        for o, T in Ts.items():
            J += T[:, None] * np.abs(prob.ords.K[o])[None, :]
        return J[:, :prob.mesh.dim]
    monkeypatch.setattr(bte, "heat_flux", heat_flux)


def _flux_components_swapped(monkeypatch):
    orig = bte.heat_flux

    def heat_flux(prob, Ts):
        return orig(prob, Ts)[:, ::-1].copy()
    monkeypatch.setattr(bte, "heat_flux", heat_flux)


def _flux_from_reversed_ordinate(monkeypatch):
    """Each field weighted by the flux weight of the opposite direction."""
    def heat_flux(prob, Ts):
        J = np.zeros((prob.mesh.nc, 3))
        for o, T in Ts.items():
            J -= T[:, None] * prob.ords.K[o][None, :]
        return J[:, :prob.mesh.dim]
    monkeypatch.setattr(bte, "heat_flux", heat_flux)


@pytest.mark.parametrize("plant,caught_by", [
    (_flux_with_unsigned_weights, "flux_porefree"),
    (_flux_components_swapped, "flux_porefree"),
    (_flux_from_reversed_ordinate, "flux_sections"),
])
def test_planted_flux_mistake_fails_a_pin(monkeypatch, plant, caught_by):
    plant(monkeypatch)
    r = flux_pins()
    assert not r[caught_by], r
