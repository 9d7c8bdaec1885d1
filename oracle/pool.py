"""Worker processes over ordinate chunks for the FP64 oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper parallelises Eq. iter over phonon directions (Sec. 3: a set of
directions per core, MFPs serial, MPI4Py).  Here ``spawn`` processes play the
cores: every worker rebuilds the problem from the workload, solves its share
of the ordinates and returns partial moments that the parent sums.  BLAS
threads are pinned to 1 per worker.  ``PoolTransport`` exposes the interface
of ``bte.Transport`` used by ``solve_mode_A`` / ``solve_mode_B``.

Two ways to hand out the ordinates:
  * a process pool over ``workers x chunks_per_worker`` chunks (load balance;
    factors are recomputed on every pass);
  * ``pinned=True``: worker k owns chunk k for the pool's lifetime, like an
    MPI rank owning its directions, so with ``cache=True`` each LU factor is
    computed once and reused on every pass (Sec. 3: factorisations reused
    across iterations); ``cache_max`` caps the factors a worker keeps.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

_STATE = {}


def _init(workload, s, cache, cache_max=None):
    """Worker set-up: the problem and its per-ordinate LU cache (Sec. 3)."""
    from . import bte
    prob = bte.Problem.from_workload(workload, s=s)
    _STATE["tr"] = bte.Transport(prob, cache=cache, cache_max=cache_max)


def _work(args):
    """One worker's share of Algorithm 1's loop over ordinates (Sec. 3)."""
    ords, T_L, T_w, with_jump, flux = args
    tr = _STATE["tr"]
    return tr.sweep(T_L, T_w, ords=ords, with_jump=with_jump, flux=flux)


def _pinned_main(conn, workload, s, cache, ords, cache_max):
    """A worker that owns a fixed set of ordinates until told to stop."""
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[k] = "1"
    _init(workload, s, cache, cache_max)
    while True:
        msg = conn.recv()
        if msg is None:
            break
        T_L, T_w, with_jump, flux = msg
        conn.send(_work((ords, T_L, T_w, with_jump, flux)))
    conn.close()


def usable_cores():
    """Cores this process may run on (the core count the baseline reports)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class PoolTransport:
    def __init__(self, workload, s=None, workers=None, cache=False, chunks_per_worker=4,
                 ordinates=None, pinned=False, cache_max=None):
        from . import bte
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[k] = "1"
        self.prob = bte.Problem.from_workload(workload, s=s)
        self._local = bte.Transport(self.prob, cache=False)   # wall weights, kappa scale
        self.w_den = self._local.w_den
        self.workers = workers or usable_cores()
        all_o = np.arange(self.prob.ords.n) if ordinates is None else np.asarray(ordinates)
        ctx = mp.get_context("spawn")
        self.pinned = pinned
        if pinned:
            self.chunks = [c for c in np.array_split(all_o, min(len(all_o), self.workers)) if len(c)]
            self.procs, self.conns = [], []
            for c in self.chunks:
                a, b = ctx.Pipe()
                p = ctx.Process(target=_pinned_main, args=(b, workload, s, cache, c, cache_max),
                               daemon=True)
                p.start()
                self.procs.append(p)
                self.conns.append(a)
            self.pool = None
        else:
            n_chunks = min(len(all_o), self.workers * chunks_per_worker)
            self.chunks = [c for c in np.array_split(all_o, n_chunks) if len(c)]
            self.pool = ctx.Pool(self.workers, initializer=_init, initargs=(workload, s, cache))

    def sweep(self, T_L, T_w, with_jump=True, flux=False, **_kw):
        if self.pinned:
            for c in self.conns:
                c.send((T_L, T_w, with_jump, flux))
            parts = [c.recv() for c in self.conns]
        else:
            parts = self.pool.map(_work, [(c, T_L, T_w, with_jump, flux) for c in self.chunks])
        out = {"TL": sum(p["TL"] for p in parts),
               "wall_num": sum(p["wall_num"] for p in parts),
               "phi": float(sum(p["phi"] for p in parts)),
               "phi_bins": sum(p["phi_bins"] for p in parts)}
        if flux:
            out["J"] = sum(p["J"] for p in parts)
        return out

    def kappa_from_phi(self, phi, with_jump=True):
        return self._local.kappa_from_phi(phi, with_jump)

    def close(self):
        if self.pinned:
            for c in self.conns:
                c.send(None)
            for p in self.procs:
                p.join()
        else:
            self.pool.close()
            self.pool.join()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
