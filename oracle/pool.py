"""Worker processes over ordinate chunks for the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper parallelises Eq. iter over phonon directions (Sec. 3: a set of
directions per core, MFPs serial, MPI4Py).  Here a ``spawn`` process pool
plays the cores: every worker rebuilds the problem from the workload, owns a
fixed chunk of ordinates (its own LU factors, optionally cached), and returns
partial moments that the parent sums.  BLAS threads are pinned to 1 per
worker.  ``PoolTransport`` exposes the interface of ``bte.Transport`` used by
``solve_mode_A`` / ``solve_mode_B``.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_STATE = {}


def _init(workload, s, cache):
    """Worker set-up: the problem and its per-ordinate LU cache (Sec. 3)."""
    from . import bte
    prob = bte.Problem.from_workload(workload, s=s)
    _STATE["tr"] = bte.Transport(prob, cache=cache)


def _work(args):
    """One worker's share of Algorithm 1's loop over ordinates (Sec. 3)."""
    ords, T_L, T_w, with_jump = args
    tr = _STATE["tr"]
    return tr.sweep(T_L, T_w, ords=ords, with_jump=with_jump)


def usable_cores():
    """Cores this process may run on (the core count the baseline reports)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class PoolTransport:
    def __init__(self, workload, s=None, workers=None, cache=False, chunks_per_worker=4,
                 ordinates=None):
        from . import bte
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.prob = bte.Problem.from_workload(workload, s=s)
        self._local = bte.Transport(self.prob, cache=False)   # wall weights, kappa scale
        self.w_den = self._local.w_den
        self.workers = workers or usable_cores()
        all_o = np.arange(self.prob.ords.n) if ordinates is None else np.asarray(ordinates)
        n_chunks = min(len(all_o), self.workers * chunks_per_worker)
        self.chunks = [c for c in np.array_split(all_o, n_chunks) if len(c)]
        ctx = mp.get_context("spawn")
        self.pool = ctx.Pool(self.workers, initializer=_init, initargs=(workload, s, cache))

    def sweep(self, T_L, T_w, with_jump=True, **_kw):
        parts = self.pool.map(_work, [(c, T_L, T_w, with_jump) for c in self.chunks])
        out = {"TL": sum(p["TL"] for p in parts),
               "wall_num": sum(p["wall_num"] for p in parts),
               "phi": float(sum(p["phi"] for p in parts))}
        return out

    def kappa_from_phi(self, phi, with_jump=True):
        return self._local.kappa_from_phi(phi, with_jump)

    def close(self):
        self.pool.close()
        self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
