"""Full-size workloads on the GPU (GPU).

Where the oracle finishes (configs 1 and 5, two small geometries of the batch,
config 2 when its stored value exists), kappa_eff and T_L at seeded sample
cells are compared with the oracle's stored values (tests/golden, written by
tests/golden/make_golden.py, which calls only the oracle).  Where it cannot
(the 3D film), properties that hold at any size are checked: equal heat flux
through every x-section, per-bin contributions that add up to kappa_eff, and
agreement of the two precisions.
"""
import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I
from gpu_common import KAPPA_RTOL, TL_ATOL, golden, gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


def _samples(g, TL):
    xyz = np.array(g["samples_xyz"])
    return TL[xyz[:, 2], xyz[:, 1], xyz[:, 0]]


def _check_golden(name, wl, precision, **kw):
    g = golden(name)
    if g is None:
        pytest.skip(f"no stored oracle value for {name}")
    s, st = gpu(wl, precision, **kw)
    k = s.kappa_eff
    assert abs(k - g["kappa_eff"]) <= KAPPA_RTOL[precision] * g["kappa_eff"], (k, g["kappa_eff"])
    t = _samples(g, s.T_L())
    assert np.abs(t - np.array(g["T_L_samples"])).max() <= TL_ATOL
    return s, st


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config1_vs_oracle(precision):
    _check_golden("1", I.config1(), precision)


def test_config1_algorithm1_stop():
    """The workload's own stopping rule (relative change of kappa 1e-6)."""
    g = golden("1")
    from paper_2106_02764_gb300.binding import Solver
    s = Solver.from_workload(I.config1())
    st = s.solve(precision="fp64", tol=1e-6, max_iter=5000)
    assert st["converged"] == 1
    assert abs(s.kappa_eff - g["kappa_eff"]) <= 1e-4 * g["kappa_eff"]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_config5_vs_oracle(precision):
    _check_golden("5", I.config5(), precision)


def test_config2_bench_launch():
    """The bench's launch configuration: mixed precision, Anderson(5), Algorithm-1
    stop 1e-6 tested every 8 iterations (bench.py's solve options)."""
    from paper_2106_02764_gb300.binding import Solver
    wl = I.config2()
    s = Solver.from_workload(wl)
    st = s.solve(precision="mixed", tol=1e-6, max_iter=3000, check_every=8, accel=5)
    assert st["converged"] == 1
    g = golden("2")
    if g is not None:
        assert abs(s.kappa_eff - g["kappa_eff"]) <= KAPPA_RTOL["mixed"] * g["kappa_eff"]
        assert np.abs(_samples(g, s.T_L()) - np.array(g["T_L_samples"])).max() <= 1e-4
    sec = s.section_flux(wl.shape[0])
    assert np.abs(sec - s.kappa_eff).max() <= 2e-4 * s.kappa_eff
    assert abs(s.kappa_bins().sum() - s.kappa_eff) <= 1e-5 * s.kappa_eff


def test_config3_film_properties():
    """3D film: conservation across every x-section, bins add up, and the
    mixed-precision fixed point agrees with the FP64 one."""
    wl = I.config3()
    sm, _ = gpu(wl, "mixed", tol=1e-8, max_iter=3000, check_every=16)
    sec = sm.section_flux(wl.shape[0])
    assert np.abs(sec - sm.kappa_eff).max() <= 1e-3 * sm.kappa_eff
    assert abs(sm.kappa_bins().sum() - sm.kappa_eff) <= 1e-5 * sm.kappa_eff
    sd, _ = gpu(wl, "fp64", tol=1e-10, tol_TL=0.0, max_iter=3000, check_every=16)
    assert abs(sm.kappa_eff - sd.kappa_eff) <= 1e-4 * sd.kappa_eff
    assert np.nanmax(np.abs(sm.T_L() - sd.T_L())) <= 1e-4
    # thinner than wide and porous: well below the bulk value
    assert 0 < sd.kappa_eff < 150.0


def test_config4_batch():
    """64 uneven geometries in one persistent launch per iteration; geometries
    with stored oracle values are compared with them, all converge, and the
    batch agrees with single solves."""
    from paper_2106_02764_gb300.binding import Solver, solve_batch
    geoms = I.config4()
    solvers = [Solver.from_workload(w) for w in geoms]
    stats = solve_batch(solvers, precision="mixed", tol=1e-8, max_iter=3000, check_every=16)
    assert all(st["converged"] == 1 for st in stats)
    checked = 0
    for gi in range(len(geoms)):
        g = golden(f"4_{gi}")
        if g is None:
            continue
        k = solvers[gi].kappa_eff
        assert abs(k - g["kappa_eff"]) <= KAPPA_RTOL["mixed"] * g["kappa_eff"], (gi, k, g["kappa_eff"])
        assert np.abs(_samples(g, solvers[gi].T_L()) - np.array(g["T_L_samples"])).max() <= 1e-4
        checked += 1
    for gi in (0, 7, 33):
        one = Solver.from_workload(geoms[gi])
        one.solve(precision="mixed", tol=1e-8, max_iter=3000, check_every=16)
        assert abs(one.kappa_eff - solvers[gi].kappa_eff) <= 1e-5 * one.kappa_eff
