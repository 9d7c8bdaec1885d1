"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU).

Each test names what it pins.  None compares the oracle with itself: closed
forms, a brute-force dense solve written separately, conservation laws,
symmetries and limits that reduce to textbook results.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2106_02764_gb300 import inputs as I
from oracle import bte, dense, fourier


def _solve(wl, **kw):
    pr = bte.Problem.from_workload(wl)
    return pr, bte.solve_mode_B(pr, **kw)


# ---------------------------------------------------------------- p1 pore-free
@pytest.mark.parametrize("quad", [I.circle_quadrature(8), I.projected_quadrature(8, 4),
                                  I.sphere_quadrature(8, 4)])
def test_porefree_closed_form(quad):
    """Pore-free periodic cell: the exact discrete solution is T_L linear with
    slope -dT/L and T_o = T_L - Lambda_m p_x a (upwind differencing is exact on
    linear fields); its upwinded face flux is kappa_bulk + (h/2) sum |K_ox|.
    Pins E1 (diagonal and jump), E2 weights and K weights (c1, c2, c8)."""
    L = 100e-9
    wl = I.make_2d("pf", 8, L, [], 3, quad)
    pr, sol = _solve(wl)
    od = pr.ords
    h = L / 8
    expect = 150.0 + 0.5 * h * np.sum(np.abs(od.K[:, 0]))
    assert abs(sol.kappa - expect) < 1e-12 * expect
    x = (pr.mesh.coords[:, 0] + 0.5) * h
    lin = -(x - x.mean()) / L
    assert np.abs(sol.T_L - lin).max() < 1e-12
    # the Fourier first guess is exact, so Algorithm 1 converges in one pass
    solA = bte.solve_mode_A(pr, tol=1e-14, max_iter=3)
    assert abs(solA.history[0] - expect) < 1e-12 * expect
    # kappa_bulk recovered by the discrete flux weights (c2)
    assert abs(np.sum(od.K[:, 0] * od.lam * od.p[:, 0]) - 150.0) < 1e-11


def test_porefree_3d_periodic():
    L = 60e-9
    mask = np.ones((4, 4, 4), np.uint8)
    k, lam = I.mfp_bins(2)
    wl = I.Workload("pf3", 3, (4, 4, 4), (L, L, L), mask, (1, 1, 1), 1.0, k, lam,
                    I.sphere_quadrature(4, 2))
    pr, sol = _solve(wl)
    expect = 150.0 + 0.5 * (L / 4) * np.sum(np.abs(pr.ords.K[:, 0]))
    assert abs(sol.kappa - expect) < 1e-12 * expect


def test_discrete_bulk_tends_to_kappa_bulk():
    """As h -> 0 the upwind numerical-diffusion term vanishes."""
    vals = []
    for n in (8, 16, 32):
        wl = I.make_2d("pf", n, 100e-9, [], 4, I.circle_quadrature(8))
        pr = bte.Problem.from_workload(wl)
        vals.append(bte.kappa_bulk_discrete(pr) - 150.0)
    assert vals[0] > 0 and abs(vals[1] / vals[0] - 0.5) < 1e-12 and abs(vals[2] / vals[1] - 0.5) < 1e-12


# ---------------------------------------------------------------- p2 dense brute force
def _wall_map(pr, d):
    m = {}
    for f, (c, a, sgn) in enumerate(pr.mesh.walls):
        xyz = tuple(int(v) for v in pr.mesh.coords[c])
        m[f] = d["walls"][(xyz, int(a), int(sgn))]
    return m


@pytest.mark.parametrize("case", ["2d", "3d", "2d_s"])
def test_dense_brute_force(case):
    if case.startswith("2d"):
        wl = I.small_2d(n=4, porosity=0, n_bins=2, n_phi=8, s_seed=3 if case == "2d_s" else None)
        wl.mask = np.ones((1, 4, 4), np.uint8)
        wl.mask[0, 1:3, 1:3] = 0
    else:
        wl = I.small_film(n=4, nz=2, porosity=0, n_bins=2, n_phi=4, n_mu=2)
        wl.mask[:, 1:3, 1:3] = 0
    pr, sol = _solve(wl, rtol=1e-13)
    d = dense.dense_from_workload(wl)
    assert d["residual"] < 1e-10
    wm = _wall_map(pr, d)
    fw = bte.fields(pr, sol)
    inv = {v: k for k, v in wm.items()}
    X = np.concatenate([np.concatenate([fw["T"][o] for o in range(pr.ords.n)]), sol.T_L,
                        np.array([sol.T_w[inv[k]] for k in range(pr.mesh.nw)])])
    Xd = np.concatenate([d["T"].ravel(), d["T_L"], d["T_w"]])
    b = d["A"] @ Xd
    # the oracle's full solution satisfies every row of the dense system
    assert np.linalg.norm(d["A"] @ X - b) < 1e-10 * np.linalg.norm(b)
    # values agree to the conditioning of the dense least-squares solve
    assert abs(sol.kappa - d["kappa"]) < 1e-9 * abs(d["kappa"])
    assert np.abs(sol.T_L - d["T_L"]).max() < 1e-9
    for f in range(pr.mesh.nw):
        assert abs(sol.T_w[f] - d["T_w"][wm[f]]) < 1e-9
    for o in range(pr.ords.n):
        assert np.abs(fw["T"][o] - d["T"][o]).max() < 1e-9


# ---------------------------------------------------------------- p3 conservation
def test_conservation_config1():
    """Net heat flux through every x-section is the same at the fixed point,
    every cell's upwinded face fluxes balance (div J = 0, the condition that
    defines T_L in Sec. 2) and every wall face carries zero net flux."""
    wl = I.config1()
    pr, sol = _solve(wl)
    fw = bte.fields(pr, sol)
    phis = fw["phis"]
    assert np.abs(phis - phis[0]).max() < 1e-9 * abs(phis[0])
    me, od = pr.mesh, pr.ords
    tr = bte.Transport(pr)
    div = np.zeros(me.nc)
    wall_net = np.zeros(me.nw)
    for o, T in fw["T"].items():
        for a in me.axes:
            k = od.K[o, a] / me.h[a]
            for side, sgn in ((0, -1), (1, 1)):
                kn = k * sgn                     # outward normal component
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
    scale = np.abs(od.K).sum() / me.h[0]
    assert np.abs(div).max() < 1e-9 * scale
    assert np.abs(wall_net).max() < 1e-9 * scale


# ---------------------------------------------------------------- p4 thin film
def _film(nz, n_mu, lam, t, lx=1e-15):
    mask = np.ones((nz, 2, 2), np.uint8)
    wl = I.Workload("film", 3, (2, 2, nz), (lx, lx, t), mask, (1, 1, 0), 1.0,
                    np.array([150.0]), np.array([lam]), I.sphere_quadrature(4, n_mu))
    return wl


def test_film_discrete_recurrence():
    """Gray film, diffuse walls at z = 0, t: T_o = a x + c_k with the discrete
    recurrence c_k = (beta_z c_{k-1} - Lambda p_x a) / (1 + beta_z), c_{-1} = 0,
    solved in closed form (geometric series).  Pins walls (E3), 3D, c14."""
    lam, t, nz = 40e-9, 30e-9, 12
    wl = _film(nz, 6, lam, t, lx=20e-9)
    pr, sol = _solve(wl, rtol=1e-13)
    od = pr.ords
    hz = t / nz
    bz = od.lam * np.abs(od.p[:, 2]) / hz
    r = bz / (1 + bz)
    geo = r * (1 - r ** nz) / (1 - r)
    kx_lp = od.K[:, 0] * od.lam * od.p[:, 0]
    hx = wl.lengths[0] / 2
    expect = 0.5 * hx * np.abs(od.K[:, 0]).sum() + kx_lp.sum() - (kx_lp * geo).sum() / nz
    assert abs(sol.kappa - expect) < 1e-11 * expect


def test_film_fuchs_sondheimer_limit():
    """Fine z grid and polar quadrature approach the Fuchs-Sondheimer result
    kappa / kappa_b = 1 - 3/(2 delta) int_0^1 mu (1 - mu^2)(1 - exp(-delta/mu)) dmu
    once the x-direction numerical-diffusion term (h_x/2) sum |K_ox| of the
    pore-free closed form is taken off."""
    lam, t = 50e-9, 25e-9
    delta = t / lam
    fs = 1 - 1.5 / delta * integrate.quad(lambda m: m * (1 - m * m) * (1 - math.exp(-delta / m)),
                                          0, 1, limit=200)[0]
    errs = []
    for nz, n_mu in ((32, 8), (128, 16)):
        wl = _film(nz, n_mu, lam, t, lx=1e-10)
        pr, sol = _solve(wl, rtol=1e-10, maxiter=20)
        offset = 0.5 * (wl.lengths[0] / 2) * np.abs(pr.ords.K[:, 0]).sum()
        errs.append(abs((sol.kappa - offset) / 150.0 - fs))
    assert errs[1] < 0.5 * errs[0] and errs[1] < 5e-3


# ---------------------------------------------------------------- p5 small-MFP limit
def test_small_mfp_tends_to_fourier():
    """Single bin with Lambda << L and h = Lambda / 2: kappa_eff relative to the
    discrete bulk value approaches kappa_fourier / kappa_bulk of the same mask,
    with a gap that shrinks as Lambda / L does (Knudsen layers)."""
    L = 100e-9
    gaps = []
    for ratio, n in ((10, 20), (20, 40)):
        wl = I.make_2d("x", n, L, [I.circle_pore(L, L, 0.2)], 1, I.circle_quadrature(16))
        wl.lambda_m = np.array([L / ratio])
        wl.kappa_m = np.array([150.0])
        pr, sol = _solve(wl, rtol=1e-10, restart=100, maxiter=50)
        kF = fourier.solve_fourier(pr.mesh, 150.0)["kappa"] / 150.0
        gaps.append(abs(sol.kappa / bte.kappa_bulk_discrete(pr) - kF))
    assert gaps[1] < 0.6 * gaps[0] and gaps[1] < 0.05


# ---------------------------------------------------------------- p6 Fourier
def test_fourier_porefree_exact():
    wl = I.make_2d("pf", 16, 100e-9, [], 1, I.circle_quadrature(4))
    me = bte.Mesh(wl.mask, wl.lengths, wl.periodic, 1.0, 2)
    r = fourier.solve_fourier(me, 150.0)
    assert abs(r["kappa"] - 150.0) < 1e-10
    x = (me.coords[:, 0] + 0.5) / 16
    assert np.abs(r["T"] + (x - x.mean())).max() < 1e-12


@pytest.mark.parametrize("phi", [0.05, 0.1, 0.2, 0.25])
def test_fourier_eucken_maxwell(phi):
    """Circular pores: kappa_fourier / kappa_bulk -> (1 - phi)/(1 + phi)
    (Sec. 8 reports < 1 % agreement); the voxel staircase error shrinks with N."""
    L = 100e-9
    devs = []
    for n in (64, 128):
        wl = I.make_2d("em", n, L, [I.circle_pore(L, L, phi)], 1, I.circle_quadrature(4))
        me = bte.Mesh(wl.mask, wl.lengths, wl.periodic, 1.0, 2)
        k = fourier.solve_fourier(me, 150.0)["kappa"] / 150.0
        ph = wl.porosity
        devs.append(abs(k / ((1 - ph) / (1 + ph)) - 1))
    assert devs[1] < devs[0] and devs[1] < 0.01


# ---------------------------------------------------------------- p7 symmetries
def _asym_wl(n=8):
    L = 100e-9
    return I.make_2d("asym", n, L, [I.square_pore(L, L, 0.1, x=0.3 * L, y=0.6 * L)], 2,
                     I.circle_quadrature(8))


def test_rotation_symmetry():
    wl = _asym_wl()
    pr, sol = _solve(wl)
    wr = _asym_wl()
    wr.mask = np.ascontiguousarray(np.transpose(wl.mask, (0, 2, 1)))
    wr.grad_axis = 1
    prr, solr = _solve(wr)
    assert abs(sol.kappa - solr.kappa) < 1e-11 * sol.kappa


def test_roll_and_mirror_symmetry():
    wl = _asym_wl()
    pr, sol = _solve(wl)
    for sh in ((2, 0), (0, 3), (5, 1)):
        w2 = _asym_wl()
        w2.mask = np.roll(wl.mask, sh, axis=(2, 1))
        _, s2 = _solve(w2)
        assert abs(sol.kappa - s2.kappa) < 1e-11 * sol.kappa
    w3 = _asym_wl()
    w3.mask = np.ascontiguousarray(wl.mask[:, :, ::-1])
    p3, s3 = _solve(w3)
    assert abs(sol.kappa - s3.kappa) < 1e-11 * sol.kappa
    g = bte.to_grid(pr, sol.T_L)
    g3 = bte.to_grid(p3, s3.T_L)
    ok = ~np.isnan(g)
    assert np.abs(g3[:, :, ::-1][ok] + g[ok]).max() < 1e-11


# ---------------------------------------------------------------- p11 reciprocity
def _cross_flux(wl, plane=0):
    """kappa of the in-plane axis normal to the gradient: the upwinded heat
    rate through the solid faces of the plane y' = plane (y' the other axis;
    no jump along it), divided by dT.  With the gradient along x this is
    kappa_yx (Q_y = kappa_yx dT / L_x over the length L_x of the plane)."""
    pr = bte.Problem.from_workload(wl)
    sol = bte.solve_mode_B(pr, rtol=1e-13)
    me, od = pr.mesh, pr.ords
    g = me.grad_axis
    a = 1 - g
    cells = np.nonzero((me.coords[:, a] == plane) & (me.nbr[:, a, 0] >= 0))[0]
    img = me.nbr[cells, a, 0]
    q = 0.0
    for o, T in bte.fields(pr, sol)["T"].items():
        K = od.K[o, a]
        q += K * (T[img].sum() if K > 0 else T[cells].sum())
    return me.h[g] * q / me.delta_T


def _random_mask_wl(quad, with_s):
    """8 x 8 cell with seven seeded single-cell pores: no mirror or transposition
    symmetry, so the off-diagonal conductivities are not zero by symmetry."""
    L = 100e-9
    wl = I.make_2d("rand", 8, L, [], 2, quad)
    rng = np.random.default_rng(7)
    m = np.ones((1, 8, 8), np.uint8)
    for _ in range(7):
        x, y = rng.integers(1, 7, size=2)
        m[0, y, x] = 0
    wl.mask = m
    if with_s:
        wl.s = I.scattering_field(m.shape, seed=11)
    return wl


@pytest.mark.parametrize("with_s", [False, True])
@pytest.mark.parametrize("quad", [I.circle_quadrature(8), I.projected_quadrature(8, 4)])
def test_onsager_reciprocity(quad, with_s):
    """kappa_xy = kappa_yx for an asymmetric mask and a quadrature symmetric
    under s -> -s: the upwind transport of p is the transpose of that of -p and
    the diffuse-wall and T_L couplings are symmetric (Sec. 2 with App. A's
    discretisation), so the discrete conductivity tensor is symmetric.  The
    cross flux is also the same through every section (conservation)."""
    import copy
    wl = _random_mask_wl(quad, with_s)
    k_yx = _cross_flux(wl)
    assert abs(k_yx) > 1e-3          # a real off-diagonal term (~1 % of kappa_xx)
    assert abs(_cross_flux(wl, plane=5) - k_yx) < 1e-10 * abs(k_yx)
    wt = copy.deepcopy(wl)
    wt.grad_axis = 1
    k_xy = _cross_flux(wt)
    assert abs(k_xy - k_yx) < 1e-10 * abs(k_yx), (k_xy, k_yx)


# ---------------------------------------------------------------- p8 folding
def test_projected_folding():
    L = 100e-9
    pores = [I.circle_pore(L, L, 0.2)]
    a = I.make_2d("f", 8, L, pores, 3, I.projected_quadrature(8, 4, fold=True))
    b = I.make_2d("u", 8, L, pores, 3, I.projected_quadrature(8, 4, fold=False))
    pa, sa = _solve(a, rtol=1e-13)
    pb, sb = _solve(b, rtol=1e-13)
    assert abs(sa.kappa - sb.kappa) < 1e-12 * sa.kappa
    assert np.abs(sa.T_L - sb.T_L).max() < 1e-12


# ---------------------------------------------------------------- p9 schemes
def test_mode_a_equals_mode_b():
    wl = I.small_2d(n=12, porosity=0.2, n_bins=3, n_phi=8)
    pr = bte.Problem.from_workload(wl)
    sb = bte.solve_mode_B(pr, rtol=1e-13)
    sa = bte.solve_mode_A(pr, tol=1e-15, max_iter=2000)
    assert abs(sa.kappa - sb.kappa) < 1e-11 * sb.kappa
    assert np.abs(sa.T_L - sb.T_L).max() < 1e-10


# ---------------------------------------------------------------- f1 per-bin spectrum
def test_kappa_bins_porefree_closed_form_and_sum():
    """Pore-free cell: bin m carries kappa_m + (h/2) sum_{o in m} |K_ox| (the
    closed form of p1 split by bin, K recomputed from the inputs); on a porous
    cell the bins add up to kappa_eff and agree with the same split of the
    dense brute-force solve."""
    L = 100e-9
    wl = I.make_2d("pf", 8, L, [], 3, I.circle_quadrature(8))
    pr, sol = _solve(wl)
    kb = bte.kappa_bins(pr, sol)
    q = wl.quad
    h = L / 8
    for m, (k, lam) in enumerate(zip(wl.kappa_m, wl.lambda_m)):
        Kx = q.angular_dim * k * q.weights * q.dirs[:, 0] / lam
        assert abs(kb[m] - (k + 0.5 * h * np.abs(Kx).sum())) < 1e-11 * kb.sum()
    wl = I.small_2d(n=4, porosity=0, n_bins=2, n_phi=8)
    wl.mask = np.ones((1, 4, 4), np.uint8)
    wl.mask[0, 1:3, 1:3] = 0
    pr, sol = _solve(wl, rtol=1e-13)
    kb = bte.kappa_bins(pr, sol)
    assert abs(kb.sum() - sol.kappa) < 1e-12 * sol.kappa
    d = dense.dense_from_workload(wl)
    me = pr.mesh
    cells, img = me.hot_faces()
    jmp = me.jump[cells, 0, 0]
    S = len(wl.quad.weights)
    for m in range(2):
        phi = 0.0
        for o in range(m * S, (m + 1) * S):
            Kx = pr.ords.K[o, 0]
            T = d["T"][o]
            phi += Kx * ((T[img] + jmp).sum() if Kx > 0 else T[cells].sum())
        km = L / (1.0 * me.n_sec) * phi
        assert abs(kb[m] - km) < 1e-9 * abs(sol.kappa)


# ---------------------------------------------------------------- heat flux J (Sec. 2)
def _flux_weights(wl):
    """K_o = d_ang kappa_m w_s p_s / Lambda_m (Sec. 2), from the workload."""
    q = wl.quad
    K = np.array([q.angular_dim * k * w * np.asarray(p[:3], float) / lam
                  for k, lam in zip(wl.kappa_m, wl.lambda_m) for p, w in zip(q.dirs, q.weights)])
    if wl.dim == 2:
        K[:, 2] = 0.0
    return K


@pytest.mark.parametrize("quad", [I.circle_quadrature(8), I.projected_quadrature(8, 4)])
@pytest.mark.parametrize("axis", [0, 1])
def test_heat_flux_porefree_closed_form(quad, axis):
    """Pore-free periodic cell: T_o = T_L - Lambda_m p_g a exactly (a the slope
    -dT/L_g of T_L along the gradient axis g), so the cell flux
    J_i = sum_o K_o T_o,i = -a sum_o K_o Lambda_m p_og is kappa_bulk dT / L_g
    along g and 0 across it, in every cell: the cell-centred flux carries no
    upwind term.  Pins heat_flux's weights, sign and component order."""
    L = 100e-9
    wl = I.make_2d("pf", 8, L, [], 3, quad)
    wl.grad_axis = axis
    pr, sol = _solve(wl, rtol=1e-13)
    J = bte.heat_flux(pr, bte.fields(pr, sol)["T"])
    expect = float(np.sum(wl.kappa_m)) * wl.delta_T / L
    assert np.abs(J[:, axis] - expect).max() < 1e-11 * expect
    assert np.abs(J[:, 1 - axis]).max() < 1e-11 * expect


def _flux_section_identity(wl):
    """Sum over cells of J_x against the face fluxes: every cell's x flux
    K_ox T_o,i leaves through its downwind x face, a solid face of one of the
    nx sections or a wall face, so
      sum_i J_x,i = nx Phi - dT N_hot sum_{p_x>0} K_ox
                    + sum_{+x walls} num_f - sum_{-x walls} num_f,
    Phi the section flux (kappa_eff dT N_sec / L_x, the same through every
    section), N_hot the solid faces of the plane x = 0 (their upwind values
    carry +dT) and num_f the E3 numerator of wall face f, den_f T_w,f at the
    fixed point (den_f from K recomputed here).  Returns (lhs, rhs)."""
    pr, sol = _solve(wl, rtol=1e-13)
    me = pr.mesh
    J = bte.heat_flux(pr, bte.fields(pr, sol)["T"])
    K = _flux_weights(wl)
    nx = me.n[0]
    phi = sol.kappa * wl.delta_T * me.n_sec / me.lengths[0]
    n_hot = len(me.hot_faces()[0])
    kpos = K[K[:, 0] > 0, 0].sum()
    den = np.array([np.maximum(K[:, a] * sg, 0.0).sum() for (_c, a, sg) in me.walls])
    num = den * sol.T_w
    xw = me.walls[:, 1] == 0
    plus, minus = xw & (me.walls[:, 2] > 0), xw & (me.walls[:, 2] < 0)
    rhs = nx * phi - wl.delta_T * n_hot * kpos + num[plus].sum() - num[minus].sum()
    return J[:, 0].sum(), rhs, pr, J


def test_heat_flux_sections_and_mirror():
    """Cell flux with pores: the section identity above ties sum J_x to the
    pinned kappa and wall temperatures, and for a pore centred in the cell J
    is mirror-symmetric in y (J_x even, J_y odd).  Pins J's x weights and
    the sign of its y component."""
    wl = I.small_2d(n=12, porosity=0.2, n_bins=3, n_phi=8)
    lhs, rhs, pr, J = _flux_section_identity(wl)
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    grid = np.full((2, 12, 12), np.nan)
    c = pr.mesh.coords
    grid[:, c[:, 1], c[:, 0]] = J.T
    assert np.nanmax(np.abs(grid[0] - grid[0][::-1])) < 1e-9 * np.nanmax(np.abs(grid[0]))
    assert np.nanmax(np.abs(grid[1] + grid[1][::-1])) < 1e-9 * np.nanmax(np.abs(grid[0]))
    assert np.nanmax(np.abs(grid[1])) > 1e-3 * np.nanmax(np.abs(grid[0]))  # J_y is not trivially 0
