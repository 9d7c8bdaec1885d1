"""Ordinate sharding of one solve (GPU).

The paper spreads the phonon directions over MPI processes (Sec. 3); within
an iteration the ordinates are independent and the only exchange is a sum of
the FP64 moment partials.  Here two or three contexts on one GPU each sweep
their share of the ordinate groups, their partials are summed on the device
between sweep and finalisation (what an all-reduce does across devices), and
every context finalises from the sum.  The sharded iteration must follow the
one-context iteration (same variant, plain source iteration) to rounding, and
the per-rank flux outputs must add up to the one-context outputs.
"""
import numpy as np
import pytest

from paper_2106_02764_gb300 import inputs as I
from gpu_common import SMALL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2106_02764_gb300 import build
    build.build()


def _sharded(wl, n_ranks, precision, iters, **kw):
    import torch
    from paper_2106_02764_gb300.binding import Solver
    ranks = [Solver.from_workload(wl).set_shard(r, n_ranks) for r in range(n_ranks)]
    for s in ranks:
        s.shard_begin(precision=precision, tol=0.0, max_iter=iters, **kw)
    n = ranks[0].shard_partials_count()
    bufs = [torch.empty(n, dtype=torch.float64, device="cuda") for _ in ranks]
    total = torch.empty(n, dtype=torch.float64, device="cuda")
    done = 0
    for _ in range(iters):
        for s, b in zip(ranks, bufs):
            s.shard_sweep(b)
        torch.cuda.synchronize()
        total.copy_(bufs[0])
        for b in bufs[1:]:
            total += b
        torch.cuda.synchronize()
        codes = [s.shard_finalize(total) for s in ranks]
        assert len(set(codes)) == 1
        done = codes[0]
        if done:
            break
    return ranks, done


def _whole(wl, precision, iters, **kw):
    from paper_2106_02764_gb300.binding import Solver
    s = Solver.from_workload(wl)
    s.solve(precision=precision, tol=0.0, max_iter=iters, check_every=1, accel=0,
            allow_not_converged=True, **kw)
    return s


@pytest.mark.parametrize("n_ranks", [2, 3])
@pytest.mark.parametrize("case,kw", [
    ("2d_square_16", {}),
    ("2d_circle_12_ragged", {"kernel": "block"}),
    ("3d_film", {}),
])
def test_sharded_fp64_equals_one_context(case, kw, n_ranks):
    wl = SMALL[case]()
    iters = 60
    ranks, done = _sharded(wl, n_ranks, "fp64", iters, **kw)
    one = _whole(wl, "fp64", iters, **kw)
    assert done == 2 and one.stats["iterations"] == iters
    k1 = one.kappa_eff
    for s in ranks:
        assert abs(s.kappa_eff - k1) <= 1e-12 * abs(k1)
        assert np.nanmax(np.abs(s.T_L() - one.T_L())) <= 1e-12
    J = sum(s.flux() for s in ranks)
    assert np.nanmax(np.abs(J - one.flux())) <= 1e-11 * np.nanmax(np.abs(one.flux()))
    kb = sum(s.kappa_bins() for s in ranks)
    assert np.abs(kb - one.kappa_bins()).max() <= 1e-11 * abs(k1)


def test_sharded_mixed_config1_to_the_oracle():
    """Config 1 in mixed precision, two ranks, to the stored oracle value."""
    from gpu_common import golden
    g = golden("1")
    wl = I.config1()
    ranks, done = _sharded(wl, 2, "mixed", 4000)
    for s in ranks:
        assert abs(s.kappa_eff - g["kappa_eff"]) <= 1e-4 * g["kappa_eff"]


def test_sharded_context_refuses_whole_solve_and_gradient():
    from paper_2106_02764_gb300.binding import ObteError, OBTE_ESTATE, OBTE_EINVAL, Solver
    wl = SMALL["2d_circle_8"]()
    s = Solver.from_workload(wl).set_shard(1, 2)
    with pytest.raises(ObteError) as e:
        s.solve(precision="fp64")
    assert e.value.code == OBTE_ESTATE
    with pytest.raises(ObteError) as e:
        s.shard_begin(precision="fp64", accel=5)
    assert e.value.code == OBTE_EINVAL
    with pytest.raises(ObteError):
        s.set_shard(2, 2)
    s.shard_begin(precision="fp64", max_iter=3)
    import torch
    b = torch.zeros(s.shard_partials_count(), dtype=torch.float64, device="cuda")
    s.shard_sweep(b)
    s.shard_finalize(b)
    with pytest.raises(ObteError) as e:
        s.kappa_grad_s()
    assert e.value.code == OBTE_ESTATE
