"""Short solves of the seeded workloads, for profiler captures and variant timing.

    python -m paper_2106_02764_gb300.profile_case --config 2 --precision mixed \
        [--iters 4] [--accel 5] [--kernel auto|warp|block|block3d] \
        [--group-size G] [--rows-per-thread R] [--time] [--grad]

Without --time: one solve of ``--iters`` source iterations launched one by
one (no CUDA graph), so that a profiler sees every launch; a capture of the
n-th sweep launch then picks a steady-state sweep.  With --time: a full solve
with per-launch CUDA events and one JSON line of per-launch sweep and
finalisation times (the figures used to order the compiled variants).
Config 4 (the batch of 64 geometries) is solved through ``solve_batch``.
With --grad the solve is followed by one d kappa / d s (record passes and
contractions; config 5 has s(x)).
"""
from __future__ import annotations

import argparse
import json
import time

from . import build, inputs
from .binding import Solver, solve_batch


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", type=int, default=2, choices=sorted(inputs.CONFIGS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--iters", type=int, default=4)
    ap.add_argument("--accel", type=int, default=5)
    ap.add_argument("--kernel", default="auto", choices=["auto", "warp", "block", "block3d"])
    ap.add_argument("--group-size", type=int, default=0)
    ap.add_argument("--rows-per-thread", type=int, default=0)
    ap.add_argument("--fourier-tol", type=float, default=0.0)
    ap.add_argument("--fourier-max-iter", type=int, default=0)
    ap.add_argument("--time", action="store_true")
    ap.add_argument("--grad", action="store_true")
    a = ap.parse_args(argv)
    build.build()
    wl = inputs.CONFIGS[a.config]()
    kw = dict(precision=a.precision, accel=a.accel, kernel=a.kernel, group_size=a.group_size,
              rows_per_thread=a.rows_per_thread)
    if a.time:
        kw.update(tol=1e-6, max_iter=3000, check_every=8, profile=True, fourier_tol=a.fourier_tol,
                  fourier_max_iter=a.fourier_max_iter)
    else:
        kw.update(tol=0.0, max_iter=a.iters, check_every=1, use_graph=False, fourier_max_iter=5)
    t0 = time.perf_counter()
    if isinstance(wl, list):
        solvers = [Solver.from_workload(w) for w in wl]
        stats = solve_batch(solvers, allow_not_converged=True, **kw)
        st = stats[0]
    else:
        s = Solver.from_workload(wl)
        st = s.solve(allow_not_converged=True, **kw)
        if a.grad:
            s.kappa_grad_s()
    wall = time.perf_counter() - t0
    out = {"config": a.config, "precision": a.precision, "iterations": st["iterations"],
           "kappa_eff": st["kappa_eff"], "group_size": st["group_size"],
           "rows_per_thread": st["rows_per_thread"], "kernel": st["kernel"], "wall_s": round(wall, 3)}
    if a.time:
        n = max(1, st["n_sweeps"])
        out.update(sweep_ms_per_launch=st["time_sweep_ms"] / n,
                   finalize_ms_per_launch=st["time_finalize_ms"] / n,
                   iter_ms=st["time_iter_ms"], fourier_ms=st["time_fourier_ms"],
                   fourier_iterations=st["fourier_iterations"])
    print(json.dumps(out))


if __name__ == "__main__":
    main()
