"""Write the oracle's converged reference values for the named workloads.

Calls only ``oracle/`` (and the seeded input generators).  For each workload it
runs the oracle's mode B (GMRES on the reduced unknowns T_L, T_w of the
Algorithm-1 fixed point, per-ordinate sparse LU solves in worker processes),
then one more pass at the solution for the per-bin split of kappa (App. A,
Eq. keff summed per MFP bin) and the cell heat flux J = sum_o K_o T_o
(Sec. 2).  It stores

  kappa_star_<name>.json  kappa_eff, the GMRES residual, kappa per bin, the
                          gauged T_L and J at seeded sample cells, timings;
  kappa_star_<name>.npz   the full gauged T_L and T_w (oracle cell / wall
                          order) and J per solid cell.

``grad5`` writes ``grad_cfg5.npz`` / ``.json``: d kappa_eff / d s(x) of the
sensitivity workload by the oracle adjoint (transposed solves, GMRES on the
adjoint unknowns), full vector over solid cells.

    python tests/golden/make_golden.py 1 5 2 3r 4:7 grad5 [--workers 6] [--rtol 1e-12]

Names: 1, 2, 3r (the config-3 film mesh with 3 bins x 8 x 4 directions),
4:<g> (geometry g of the batch), 5, grad5.
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


def workload(cfg: str):
    if cfg.startswith("4:"):
        return I.config4()[int(cfg.split(":")[1])]
    if cfg == "3r":
        return I.config3_reduced()
    return I.CONFIGS[int(cfg)]()


def _samples(prob, n_samples=64):
    rng = np.random.default_rng(I.seed_for(9, 0))
    return np.sort(rng.choice(prob.mesh.nc, size=min(n_samples, prob.mesh.nc), replace=False))


def golden(cfg: str, workers: int, rtol: float, cache_gb: float):
    wl = workload(cfg)
    # pinned workers keep as many LU factors as the memory budget allows
    # (factor size measured on the first ordinate)
    from oracle.bte import Problem, Transport
    probe = Transport(Problem.from_workload(wl), cache=False)
    lu0 = probe.lu(0)
    # SciPy's SuperLU object holds about 32 bytes per stored entry (0.94 GB for
    # the 3D film's 30 M entries)
    lu_bytes = 40 * (lu0.L.nnz + lu0.U.nnz) + 4096
    per_worker = int(cache_gb * 1e9 / lu_bytes / workers)
    del probe, lu0
    t0 = time.time()
    with pool.PoolTransport(wl, workers=workers, pinned=True, cache=per_worker > 0,
                            cache_max=per_worker) as tr:
        sol = bte.solve_mode_B(tr.prob, rtol=rtol, tr=tr)
        t1 = time.time()
        r = tr.sweep(sol.T_L, sol.T_w, flux=True)
    dt = t1 - t0
    prob = tr.prob
    pick = _samples(prob)
    c = prob.mesh.coords[pick]
    kF = fourier.solve_fourier(prob.mesh, prob.ords.kappa_axes)["kappa"]
    kb = tr.kappa_from_phi(r["phi_bins"])
    out = {
        "workload": wl.name,
        "config": cfg,
        "kappa_eff": sol.kappa,
        "kappa_fourier": kF,
        "kappa_bins": [float(v) for v in kb],
        "gmres_matvecs": sol.iterations,
        "relative_residual": sol.residual,
        "n_solid": prob.mesh.nc,
        "n_walls": prob.mesh.nw,
        "n_ordinates": prob.ords.n,
        "samples_xyz": c.tolist(),
        "T_L_samples": sol.T_L[pick].tolist(),
        "J_samples": r["J"][pick].tolist(),
        "T_L_mean_abs": float(np.abs(sol.T_L).mean()),
        "oracle_seconds": dt,
        "workers": workers,
        "lu_factors_cached_per_worker": per_worker,
        "made_by": "tests/golden/make_golden.py (oracle mode B)",
    }
    name = cfg.replace(":", "_")
    path = os.path.join(HERE, f"kappa_star_cfg{name}.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    np.savez_compressed(os.path.join(HERE, f"kappa_star_cfg{name}.npz"),
                        T_L=sol.T_L, T_w=sol.T_w, J=r["J"], coords=prob.mesh.coords.astype(np.int32))
    print(cfg, wl.name, "kappa", sol.kappa, "res", sol.residual, "matvecs", sol.iterations,
          f"{dt:.1f}s", flush=True)


def golden_grad5(rtol: float):
    from oracle import adjoint
    wl = I.config5()
    prob = bte.Problem.from_workload(wl)
    t0 = time.time()
    g, info = adjoint.kappa_grad_s(prob, rtol=rtol)
    dt = time.time() - t0
    sol = info["solution"]
    rng = np.random.default_rng(I.seed_for(5, 64))
    fd_cells = np.sort(rng.choice(prob.mesh.nc, size=64, replace=False))
    out = {
        "workload": wl.name,
        "kappa_eff": sol.kappa,
        "relative_residual": sol.residual,
        "grad_max_abs": float(np.abs(g).max()),
        "grad_sum_s_weighted": float((prob.s * g).sum()),
        "fd_cells_xyz": prob.mesh.coords[fd_cells].tolist(),
        "grad_fd_cells": g[fd_cells].tolist(),
        "oracle_seconds": dt,
        "made_by": "tests/golden/make_golden.py grad5 (oracle adjoint)",
    }
    with open(os.path.join(HERE, "grad_cfg5.json"), "w") as f:
        json.dump(out, f, indent=1)
    np.savez_compressed(os.path.join(HERE, "grad_cfg5.npz"), grad=g,
                        coords=prob.mesh.coords.astype(np.int32))
    print("grad5 kappa", sol.kappa, "max|g|", out["grad_max_abs"], f"{dt:.1f}s", flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("configs", nargs="+")
    ap.add_argument("--workers", type=int, default=pool.usable_cores())
    ap.add_argument("--rtol", type=float, default=1e-12)
    ap.add_argument("--cache-gb", type=float, default=30.0,
                    help="host memory for cached LU factors, all workers together")
    a = ap.parse_args()
    for cfg in a.configs:
        if cfg == "grad5":
            golden_grad5(a.rtol)
        else:
            golden(cfg, a.workers, a.rtol, a.cache_gb)


if __name__ == "__main__":
    main()
