"""Write the oracle's converged reference values for the named workloads.

Calls only ``oracle/`` (and the seeded input generators).  For each workload it
runs the oracle's mode B (GMRES on the reduced unknowns T_L, T_w of the
Algorithm-1 fixed point, per-ordinate sparse LU solves in worker processes)
and stores kappa_eff, the GMRES residual and the gauged lattice temperature at
seeded sample cells in ``kappa_star_<name>.json`` beside this script.

    python tests/golden/make_golden.py 1 5 2 [--workers 6] [--rtol 1e-10]
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from paper_2106_02764_gb300 import inputs as I  # noqa: E402
from oracle import bte, fourier, pool  # noqa: E402


def golden(cfg: str, workers: int, rtol: float, n_samples: int = 64):
    if cfg.startswith("4:"):
        g = int(cfg.split(":")[1])
        wl = I.config4()[g]
    else:
        wl = I.CONFIGS[int(cfg)]()
    t0 = time.time()
    with pool.PoolTransport(wl, workers=workers) as tr:
        sol = bte.solve_mode_B(tr.prob, rtol=rtol, tr=tr)
    dt = time.time() - t0
    prob = tr.prob
    rng = np.random.default_rng(I.seed_for(9, 0))
    pick = np.sort(rng.choice(prob.mesh.nc, size=min(n_samples, prob.mesh.nc), replace=False))
    c = prob.mesh.coords[pick]
    kF = fourier.solve_fourier(prob.mesh, prob.ords.kappa_bulk)["kappa"]
    out = {
        "workload": wl.name,
        "config": cfg,
        "kappa_eff": sol.kappa,
        "kappa_fourier": kF,
        "gmres_matvecs": sol.iterations,
        "relative_residual": sol.residual,
        "n_solid": prob.mesh.nc,
        "n_ordinates": prob.ords.n,
        "samples_xyz": c.tolist(),
        "T_L_samples": sol.T_L[pick].tolist(),
        "T_L_mean_abs": float(np.abs(sol.T_L).mean()),
        "oracle_seconds": dt,
        "workers": workers,
        "made_by": "tests/golden/make_golden.py (oracle mode B)",
    }
    name = cfg.replace(":", "_")
    path = os.path.join(HERE, f"kappa_star_cfg{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(cfg, wl.name, "kappa", sol.kappa, "res", sol.residual, "matvecs", sol.iterations,
          f"{dt:.1f}s", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("configs", nargs="+")
    ap.add_argument("--workers", type=int, default=pool.usable_cores())
    ap.add_argument("--rtol", type=float, default=1e-10)
    a = ap.parse_args()
    for cfg in a.configs:
        golden(cfg, a.workers, a.rtol)


if __name__ == "__main__":
    main()
