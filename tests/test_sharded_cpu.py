"""Ordinate sharding across ranks, on CPU with gloo (world size 2).

Within one iteration the ordinates are independent (Sec. 3: directions are
spread over cores); the only exchange is a sum of the moment partials (T_L
numerator, wall numerators, hot-face flux).  Two gloo ranks each sweep half of
the ordinates with the oracle and all-reduce their partials; the result must
equal the one-process sweep, and a few sharded iterations must equal the
unsharded ones.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2106_02764_gb300 import inputs as I
    from oracle import bte
    wl = I.small_2d(n=10, porosity=0.2, n_bins=3, n_phi=8)
    pr = bte.Problem.from_workload(wl)
    tr = bte.Transport(pr)
    mine = np.array_split(np.arange(pr.ords.n), world)[rank]
    T_L, T_w = bte.initial_guess(tr)
    hist = []
    for _ in range(5):
        r = tr.sweep(T_L, T_w, ords=mine)
        buf = torch.from_numpy(np.concatenate([r["TL"], r["wall_num"], [r["phi"]]]))
        dist.all_reduce(buf, op=dist.ReduceOp.SUM)
        v = buf.numpy()
        nc, nw = pr.mesh.nc, pr.mesh.nw
        T_L, T_w = v[:nc], v[nc:nc + nw] / tr.w_den
        hist.append(tr.kappa_from_phi(v[-1]))
    if rank == 0:
        np.savez(out_path, T_L=T_L, T_w=T_w, hist=np.array(hist))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_iteration(tmp_path):
    out = str(tmp_path / "r.npz")
    tmp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, join=True,
                        start_method="spawn")
    from paper_2106_02764_gb300 import inputs as I
    from oracle import bte
    wl = I.small_2d(n=10, porosity=0.2, n_bins=3, n_phi=8)
    pr = bte.Problem.from_workload(wl)
    tr = bte.Transport(pr)
    T_L, T_w = bte.initial_guess(tr)
    hist = []
    for _ in range(5):
        T_L, T_w, k = bte.apply_M(tr, T_L, T_w)
        hist.append(k)
    r = np.load(out)
    assert np.abs(r["T_L"] - T_L).max() < 1e-13
    assert np.abs(r["T_w"] - T_w).max() < 1e-13
    assert np.abs(r["hist"] - np.array(hist)).max() < 1e-12 * abs(hist[-1])
