"""CUDA path vs the FP64 oracle, element by element, through the C ABI (GPU).

Small seeded cases span several sweep tiles, ragged ordinate groups (octant
sizes not multiples of the group size), 2D and 3D, pores and film walls, a
permuted gradient axis and a per-cell scattering scale.  Both precisions are
checked at a tight fixed point against the bar: kappa_eff within 1e-6
relative (FP64) / 1e-4 (mixed), T_L within 1e-5 K.
"""
import numpy as np
import pytest

from gpu_common import KAPPA_RTOL, SMALL, TL_ATOL, gpu, oracle, rect_2d, solid_vector, transposed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


_REF = {}


def _ref(name, factory):
    if name not in _REF:
        wl = factory()
        _REF[name] = (wl,) + oracle(wl)
    return _REF[name]


def _check(wl, pr, ref, s, precision):
    k = s.kappa_eff
    assert abs(k - ref.kappa) <= KAPPA_RTOL[precision] * abs(ref.kappa), (k, ref.kappa)
    TL = solid_vector(pr, s.T_L())
    assert np.abs(TL - ref.T_L).max() <= TL_ATOL
    return abs(k - ref.kappa) / abs(ref.kappa), np.abs(TL - ref.T_L).max()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", sorted(SMALL))
def test_small_cases(name, precision):
    """kappa_eff, T_L and kappa per MFP bin (the per-bin split of Eq. keff,
    App. A) against the oracle, bin by bin: within the kappa bar times
    kappa_eff; FP64 within 1e-9."""
    from oracle import bte
    wl, pr, ref = _ref(name, SMALL[name])
    s, st = gpu(wl, precision)
    rk, rt = _check(wl, pr, ref, s, precision)
    kb_ref = bte.kappa_bins(pr, ref)
    kb = s.kappa_bins()
    assert kb.shape == kb_ref.shape
    rb = np.abs(kb - kb_ref).max() / abs(ref.kappa)
    assert rb <= KAPPA_RTOL[precision], rb
    if precision == "fp64":
        # a tight FP64 fixed point agrees far below the bar
        assert rk < 1e-9 and rt < 1e-9 and rb < 1e-9, (rk, rt, rb)
    # pores are NaN in the returned field
    TL = s.T_L()
    assert np.all(np.isnan(TL[wl.mask == 0])) and np.all(np.isfinite(TL[wl.mask == 1]))


def test_porefree_closed_form_gpu():
    from oracle import bte
    wl = SMALL["2d_porefree"]()
    pr = bte.Problem.from_workload(wl)
    s, _ = gpu(wl, "fp64", tol=1e-14, tol_TL=1e-15)
    # long-MFP ordinates converge through the lagged periodic cut at a rate
    # close to 1 in a pore-free cell: the fixed point is reached to ~1e-10
    assert abs(s.kappa_eff - bte.kappa_bulk_discrete(pr)) < 1e-9 * bte.kappa_bulk_discrete(pr)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_rectangular_and_transposed(precision):
    wl = rect_2d()
    pr, ref = oracle(wl)
    s, _ = gpu(wl, precision)
    _check(wl, pr, ref, s, precision)
    wt = transposed(SMALL["2d_square_16"]())
    prt, reft = oracle(wt)
    st, _ = gpu(wt, precision)
    _check(wt, prt, reft, st, precision)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_every_compiled_variant(precision):
    """All (group size, rows per thread) variants that fit a 16x16 mesh."""
    from paper_2106_02764_gb300.binding import ObteError
    wl, pr, ref = _ref("2d_square_16", SMALL["2d_square_16"])
    tried = 0
    for G in (4, 8, 16):
        for R in (1, 2, 4, 8):
            try:
                s, st = gpu(wl, precision, group_size=G, rows_per_thread=R)
            except ObteError as e:
                assert "variant" in str(e)
                continue
            assert st["group_size"] == G and st["rows_per_thread"] == R
            _check(wl, pr, ref, s, precision)
            tried += 1
    assert tried >= 4


def test_graph_and_direct_launch_agree():
    wl, pr, ref = _ref("2d_circle_8", SMALL["2d_circle_8"])
    a, sa = gpu(wl, "fp64", use_graph=True, tol_TL=0.0, tol=0.0, max_iter=37, check_every=5)
    b, sb = gpu(wl, "fp64", use_graph=False, tol_TL=0.0, tol=0.0, max_iter=37, check_every=3)
    assert sa["iterations"] == sb["iterations"] == 37
    assert np.array_equal(np.array(sa["kappa_history"]), np.array(sb["kappa_history"])) or \
        np.allclose(sa["kappa_history"], sb["kappa_history"], rtol=1e-13, atol=0)


def test_algorithm1_stopping_rule():
    """tol on the relative change of kappa stops the iteration (Algorithm 1)."""
    wl, pr, ref = _ref("2d_circle_8", SMALL["2d_circle_8"])
    from paper_2106_02764_gb300.binding import Solver
    s = Solver.from_workload(wl)
    st = s.solve(precision="fp64", tol=1e-6, max_iter=5000, check_every=1)
    h = st["kappa_history"]
    assert st["converged"] == 1 and st["iterations"] == len(h)
    assert abs(h[-1] - h[-2]) <= 1e-6 * abs(h[-1])
    assert all(abs(h[i] - h[i - 1]) > 1e-6 * abs(h[i]) for i in range(1, len(h) - 1))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_flux_outputs(precision):
    """J = sum_o K_o T_o per cell, section fluxes equal kappa_eff (conservation)
    and the per-bin contributions add up to kappa_eff."""
    from oracle import bte
    wl, pr, ref = _ref("2d_square_16", SMALL["2d_square_16"])
    s, _ = gpu(wl, precision)
    J = s.flux()
    fw = bte.fields(pr, ref)
    Jo = bte.heat_flux(pr, fw["T"])
    Jg = np.stack([solid_vector(pr, J[..., a]) for a in range(2)], axis=1)
    scale = np.abs(Jo).max()
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert np.abs(Jg - Jo).max() <= tol * scale
    sec = s.section_flux(wl.shape[0])
    assert np.abs(sec - s.kappa_eff).max() <= (1e-9 if precision == "fp64" else 2e-4) * s.kappa_eff
    kb = s.kappa_bins()
    assert abs(kb.sum() - s.kappa_eff) <= (1e-10 if precision == "fp64" else 1e-5) * s.kappa_eff


def test_nonfinite_and_state_errors():
    from paper_2106_02764_gb300.binding import ObteError, Solver, OBTE_ESTATE, OBTE_ENONFINITE, OBTE_EINVAL
    s = Solver()
    with pytest.raises(ObteError) as e:
        s.solve()
    assert e.value.code == OBTE_ESTATE
    wl = SMALL["2d_circle_8"]()
    s.create_mesh(wl.mask, wl.lengths, wl.periodic, 0, 1.0)
    k = wl.kappa_m.copy()
    k[0] = np.nan
    with pytest.raises(ObteError) as e:
        s.set_material(k, wl.lambda_m, wl.quad.dirs, wl.quad.weights, 2)
    assert e.value.code == OBTE_ENONFINITE
    with pytest.raises(ObteError) as e:
        s.set_material(wl.kappa_m, wl.lambda_m, wl.quad.dirs, wl.quad.weights * 2, 2)
    assert e.value.code == OBTE_EINVAL
    bad = np.ones((1, 8, 8), np.uint8)
    with pytest.raises(ObteError):
        s.create_mesh(bad, wl.lengths, (0, 1, 1), 0, 1.0)  # gradient axis not periodic
    with pytest.raises(ObteError):
        s.create_mesh(np.ones((1, 12, 8), np.uint8), (1e-7, 1.5e-7, 0), (1, 1, 1), 0, 1.0)


def test_iteration_cap_reports_not_converged():
    from paper_2106_02764_gb300.binding import ObteError, OBTE_NOT_CONVERGED, Solver
    wl = SMALL["2d_circle_8"]()
    s = Solver.from_workload(wl)
    with pytest.raises(ObteError) as e:
        s.solve(precision="fp64", tol=1e-14, max_iter=3, check_every=1)
    assert e.value.code == OBTE_NOT_CONVERGED
    assert s.stats["iterations"] == 3 and np.isfinite(s.kappa_eff)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name", ["2d_circle_8", "2d_square_16", "3d_film", "2d_scatter", "2d_porefree"])
def test_anderson_same_fixed_point(name, precision):
    """Anderson mixing of (T_L, T_w, carried row values) reaches the oracle's
    fixed point, in fewer iterations than the plain source iteration."""
    wl, pr, ref = _ref(name, SMALL[name])
    s, st = gpu(wl, precision, accel=5)
    _check(wl, pr, ref, s, precision)
    if precision == "fp64":
        _, st0 = gpu(wl, precision)
        assert st["iterations"] < st0["iterations"], (st["iterations"], st0["iterations"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kernel", ["block", "block3d"])
def test_3d_kernels(precision, kernel):
    """Both 3D kernels (plain block kernel, block kernel with skewed records)
    against the oracle on the small film, with and without pores."""
    for name in ("3d_film", "3d_film_porefree"):
        wl, pr, ref = _ref(name, SMALL[name])
        s, st = gpu(wl, precision, kernel=kernel)
        assert st["kernel"] == (3 if kernel == "block3d" else 1)
        _check(wl, pr, ref, s, precision)


def test_3d_periodic_cube_porefree():
    """3D periodic cube (nz = nx): the z wrap through the skewed exchange."""
    import numpy as np
    from paper_2106_02764_gb300 import inputs as I
    from oracle import bte
    L = 60e-9
    k, lam = I.mfp_bins(2)
    mask = np.ones((8, 8, 8), np.uint8)
    mask[:, 3:5, 2:6] = 0
    wl = I.Workload("cube", 3, (8, 8, 8), (L, L, L), mask, (1, 1, 1), 1.0, k, lam,
                    I.sphere_quadrature(4, 2))
    pr, ref = oracle(wl)
    for precision in ("fp64", "mixed"):
        s, st = gpu(wl, precision)
        _check(wl, pr, ref, s, precision)


def test_fma_rate_measurement():
    """The measured FMA throughput is positive and below the unit-count peak
    (152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s, with a
    margin for a box with more SMs or a higher boost clock); FP64 is far
    slower than FP32 on this part."""
    from paper_2106_02764_gb300.binding import measure_fma_rate
    f32 = measure_fma_rate("mixed") / 1e12
    f64 = measure_fma_rate("fp64") / 1e12
    assert 1.0 < f32 < 1.3 * 80.5
    assert 0.0 < f64 < f32


@pytest.mark.parametrize("ny,G,R", [(32, 8, 1), (32, 16, 1), (64, 8, 2), (64, 16, 2), (96, 8, 3),
                                    (160, 8, 5), (192, 8, 6), (256, 8, 4)])
def test_full_lane_variants_block_combine(ny, G, R):
    """Fixed-rows variants whose rows fill the 32 lanes (N_y = 32 R), or the 64
    lanes of a two-warp group (N_y = 64 R), add the four groups' moments of a
    block in shared memory before the atomics; every row range must be added
    once, also with fewer than four or a number of rows per lane that is not a
    power of two (plain record-slot order).

    The row-combining logic is checked against the 8 x 8 variant on the same
    mesh, whose rows fill at most 24 lanes, so that each warp issues its own
    atomics (no block combine): both sum the same float products in another
    order, while a row range dropped or added twice moves T_L by ~0.1 K.
    Against the FP64 oracle, kappa is held to the mixed bar and T_L to
    1e-5 K.  These tall cells are the most sensitive to the float transport
    coefficients (through the 1 nm bin, which carries almost all of the T_L
    weight); the delta form of the sweep keeps the weight of T_L at exactly
    1 - A_x - A_y, which brings the coefficient floor from 1.08e-5 K (A0
    rounded on its own) to below 1e-6 K (tests/test_mixed_precision_model)."""
    from paper_2106_02764_gb300 import inputs as I
    L, nx = 100e-9, 16
    Ly = L * ny / nx
    wl = I.make_2d(f"full{ny}", nx, L, [], 2, I.circle_quadrature(16))
    wl.mask = I.pores_mask(nx, ny, L, Ly, [I.square_pore(L, Ly, 0.1, x=0.35 * L, y=0.6 * Ly)])
    wl.shape = (nx, ny, 1)
    wl.lengths = (L, Ly, 0.0)
    pr, ref = oracle(wl)
    s, st = gpu(wl, "mixed", group_size=G, rows_per_thread=R)
    assert st["group_size"] == G and st["rows_per_thread"] == R and st["kernel"] == 2
    if ny == 64 * R:  # two-warp groups: eight warps per block
        assert st["threads_per_block"] == 256
    b, sb = gpu(wl, "mixed", group_size=8, rows_per_thread=8)
    assert sb["rows_per_thread"] == 8 and sb["kernel"] == 2
    TL, TLb = solid_vector(pr, s.T_L()), solid_vector(pr, b.T_L())
    assert np.abs(TL - TLb).max() <= TL_ATOL
    assert abs(s.kappa_eff - b.kappa_eff) <= 1e-5 * abs(b.kappa_eff)
    assert abs(s.kappa_eff - ref.kappa) <= KAPPA_RTOL["mixed"] * abs(ref.kappa)
    assert np.abs(TL - ref.T_L).max() <= TL_ATOL


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_single_solve_autotune(precision):
    """group_size = -1 times every compiled variant that fits the mesh for a few
    sweeps, solves with the fastest and caches it for the mesh shape; a later
    solve with the default options takes the cached variant."""
    wl, pr, ref = _ref("2d_square_16", SMALL["2d_square_16"])
    s, st = gpu(wl, precision, group_size=-1)
    _check(wl, pr, ref, s, precision)
    assert st["group_size"] > 0 and st["rows_per_thread"] > 0 and st["kernel"] in (1, 2)
    s2, st2 = gpu(wl, precision)
    assert (st2["kernel"], st2["group_size"], st2["rows_per_thread"]) == \
        (st["kernel"], st["group_size"], st["rows_per_thread"])
    _check(wl, pr, ref, s2, precision)


def test_fast_step_loop_8x8_tall_cell():
    """The 8 x 8 FP32 form's compile-time step loop (two steps per trip) runs
    when the rows fill the 32 lanes (N_y = 256), the block combines four
    groups of one quadrant and nx is a multiple of 8: a 16 x 256 cell with a
    square pore, 2 bins x 16 directions, against the FP64 oracle at the
    mixed bars, and against the same mesh on the general loop (8 x 4 rows,
    two warps per group) within the T_L bar."""
    from paper_2106_02764_gb300 import inputs as I
    L, nx, ny = 100e-9, 16, 256
    Ly = L * ny / nx
    wl = I.make_2d("fast256", nx, L, [], 2, I.circle_quadrature(16))
    wl.mask = I.pores_mask(nx, ny, L, Ly, [I.square_pore(L, Ly, 0.1, x=0.35 * L, y=0.6 * Ly)])
    wl.shape = (nx, ny, 1)
    wl.lengths = (L, Ly, 0.0)
    pr, ref = oracle(wl)
    s, st = gpu(wl, "mixed", group_size=8, rows_per_thread=8)
    assert st["group_size"] == 8 and st["rows_per_thread"] == 8 and st["kernel"] == 2
    assert st["threads_per_block"] == 128  # four one-warp groups per block: the block combine
    b, sb = gpu(wl, "mixed", group_size=8, rows_per_thread=4)
    assert sb["rows_per_thread"] == 4
    TL, TLb = solid_vector(pr, s.T_L()), solid_vector(pr, b.T_L())
    assert abs(s.kappa_eff - ref.kappa) <= KAPPA_RTOL["mixed"] * abs(ref.kappa)
    assert np.abs(TL - ref.T_L).max() <= TL_ATOL
    assert np.abs(TL - TLb).max() <= TL_ATOL
