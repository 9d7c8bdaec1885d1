"""Batched solve: several geometries of uneven size in one persistent launch
per iteration (GPU)."""
import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I
from gpu_common import KAPPA_RTOL, TL_ATOL, oracle, solid_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


def _geoms():
    L = 100e-9
    q = I.circle_quadrature(8)
    return [
        I.make_2d("b0", 8, L, [I.circle_pore(L, L, 0.2)], 3, q),
        I.make_2d("b1", 16, L, [I.square_pore(L, L, 0.1, x=0.3 * L, y=0.6 * L)], 3, q),
        I.make_2d("b2", 16, L, [I.circle_pore(L, L, 0.05, x=0.2 * L, y=0.2 * L),
                                I.square_pore(L, L, 0.05, x=0.7 * L, y=0.7 * L)], 3, q),
        I.make_2d("b3", 12, L, [], 3, q),
    ]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_matches_oracle(precision):
    from paper_2106_02764_gb300.binding import Solver, solve_batch
    geoms = _geoms()
    solvers = [Solver.from_workload(w) for w in geoms]
    if precision == "fp64":
        opts = dict(tol=1e-12, tol_TL=1e-13, max_iter=200000, check_every=32)
    else:
        opts = dict(tol=0.0, tol_TL=0.0, max_iter=4000, check_every=50)
    stats = solve_batch(solvers, precision=precision, allow_not_converged=True, **opts)
    for w, s, st in zip(geoms, solvers, stats):
        pr, ref = oracle(w)
        assert abs(s.kappa_eff - ref.kappa) <= KAPPA_RTOL[precision] * ref.kappa
        assert np.abs(solid_vector(pr, s.T_L()) - ref.T_L).max() <= TL_ATOL
    if precision == "fp64":
        # per-geometry stopping: iteration counts differ between geometries
        its = [st["iterations"] for st in stats]
        assert len(set(its)) > 1


def test_batch_equals_single():
    from paper_2106_02764_gb300.binding import Solver, solve_batch
    geoms = _geoms()
    solvers = [Solver.from_workload(w) for w in geoms]
    solve_batch(solvers, precision="fp64", tol=1e-12, tol_TL=1e-13, max_iter=200000,
                allow_not_converged=True)
    for w, s in zip(geoms, solvers):
        one = Solver.from_workload(w)
        one.solve(precision="fp64", tol=1e-12, tol_TL=1e-13, max_iter=200000, allow_not_converged=True)
        assert abs(one.kappa_eff - s.kappa_eff) < 1e-10 * one.kappa_eff


def test_batch_anderson():
    from paper_2106_02764_gb300.binding import Solver, solve_batch
    geoms = _geoms()
    solvers = [Solver.from_workload(w) for w in geoms]
    solve_batch(solvers, precision="fp64", tol=1e-12, tol_TL=1e-13, max_iter=200000, accel=5,
                allow_not_converged=True)
    for w, s in zip(geoms, solvers):
        pr, ref = oracle(w)
        assert abs(s.kappa_eff - ref.kappa) <= KAPPA_RTOL["fp64"] * ref.kappa
        assert np.abs(solid_vector(pr, s.T_L()) - ref.T_L).max() <= TL_ATOL


def _class_geoms():
    """Sizes that make the mixed batch run several fixed-rows classes at once:
    32 (1 row per lane, 32 lanes: moments combined per block of four warps),
    64 (2 rows, 32 lanes: combined), 48 (2 rows, 24 lanes), 96 (3 rows,
    32 lanes: combined), 80 (4 rows, 20 lanes)."""
    L = 100e-9
    q = I.circle_quadrature(16)
    return [
        I.make_2d("c32", 32, L, [I.circle_pore(L, L, 0.2)], 3, q),
        I.make_2d("c64", 64, L, [I.square_pore(L, L, 0.12, x=0.3 * L, y=0.6 * L)], 3, q),
        I.make_2d("c48", 48, L, [I.circle_pore(L, L, 0.15, x=0.4 * L, y=0.45 * L)], 3, q),
        I.make_2d("c96", 96, L, [I.circle_pore(L, L, 0.1)], 3, q),
        I.make_2d("c80", 80, L, [], 3, q),
    ]


def test_mixed_batch_fixed_row_classes():
    """Mixed precision: every geometry of a batch that runs several fixed-rows
    classes side by side (forked streams, block-combined moments where rows
    fill the lanes) agrees with the oracle and with its own single solve."""
    from paper_2106_02764_gb300.binding import Solver, solve_batch
    geoms = _class_geoms()
    solvers = [Solver.from_workload(w) for w in geoms]
    opts = dict(tol=0.0, tol_TL=0.0, max_iter=3000, check_every=50)
    stats = solve_batch(solvers, precision="mixed", allow_not_converged=True, **opts)
    assert sorted({st["rows_per_thread"] for st in stats}) == [1, 2, 3, 4]
    for w, s in zip(geoms, solvers):
        pr, ref = oracle(w)
        assert abs(s.kappa_eff - ref.kappa) <= KAPPA_RTOL["mixed"] * ref.kappa
        assert np.abs(solid_vector(pr, s.T_L()) - ref.T_L).max() <= TL_ATOL
        one = Solver.from_workload(w)
        one.solve(precision="mixed", allow_not_converged=True, **opts)
        assert abs(one.kappa_eff - s.kappa_eff) <= 1e-5 * one.kappa_eff


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_autotune(precision):
    """group_size = -1 times the batch forms the compiled variants allow
    (fixed-rows class launches, persistent warp queue, persistent block
    kernel) for a few iterations and solves with the fastest: every geometry
    reaches the kappa_eff of the default form, geometries 1 and 2 the oracle's
    stored value, and a second call takes the cached choice."""
    from paper_2106_02764_gb300.binding import Solver, solve_batch
    from gpu_common import golden
    geoms = I.config4(n_geom=4)  # N = 96, 64, 48, 96
    solvers = [Solver.from_workload(w) for w in geoms]
    opts = dict(precision=precision, tol=1e-9 if precision == "fp64" else 1e-8, max_iter=3000, check_every=16)
    solve_batch(solvers, **opts)
    k_default = [s.kappa_eff for s in solvers]
    st = solve_batch(solvers, group_size=-1, **opts)
    assert all(x["converged"] == 1 for x in st)
    assert st[0]["kernel"] in (1, 2)
    for s, k in zip(solvers, k_default):
        assert abs(s.kappa_eff - k) <= 1e-5 * k, (s.kappa_eff, k)
    for gi in (1, 2):
        g = golden(f"4_{gi}")
        if g is not None:
            assert abs(solvers[gi].kappa_eff - g["kappa_eff"]) <= KAPPA_RTOL[precision] * g["kappa_eff"]
    st2 = solve_batch(solvers, group_size=-1, **opts)
    assert [(x["kernel"], x["group_size"], x["rows_per_thread"]) for x in st2] == \
        [(x["kernel"], x["group_size"], x["rows_per_thread"]) for x in st]
    print(f"batch autotune ({precision}): kernel {st[0]['kernel']}, G {st[0]['group_size']}, "
          f"rows per lane {[x['rows_per_thread'] for x in st]}")
