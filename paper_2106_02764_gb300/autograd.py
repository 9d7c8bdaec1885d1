"""torch.autograd.Function for kappa_eff(s) with the CUDA adjoint.

``KappaEff.apply(s, workload, precision)`` solves the transport problem of
``workload`` with the per-cell scattering scale ``s`` (a float64 tensor of the
mesh's shape) on the GPU and returns kappa_eff as a 0-d tensor; ``backward``
returns d kappa_eff / d s from ``obte_kappa_grad_s`` (reversed-direction
adjoint sweeps contracted with the forward fields, group by group;
``max_field_bytes`` bounds the device memory of the recorded fields, 0 for
the library's default of 1 GiB).
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from .binding import Solver


class KappaEff(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, workload, precision="fp64", tol_TL=None, max_iter=200000,
                max_field_bytes=0):
        wl = copy.copy(workload)
        wl.s = s.detach().cpu().numpy().astype(np.float64).reshape(workload.mask.shape)
        solver = Solver.from_workload(wl)
        if precision == "fp64":
            solver.solve(precision=precision, tol=1e-12, tol_TL=1e-13 if tol_TL is None else tol_TL,
                         max_iter=max_iter, allow_not_converged=True)
        else:
            solver.solve(precision=precision, tol=0.0, tol_TL=0.0, max_iter=min(max_iter, 4000),
                         allow_not_converged=True)
        ctx.solver = solver
        ctx.shape = s.shape
        ctx.max_field_bytes = max_field_bytes
        return torch.tensor(solver.kappa_eff, dtype=torch.float64)

    @staticmethod
    def backward(ctx, grad_out):
        g = ctx.solver.kappa_grad_s(max_field_bytes=ctx.max_field_bytes)
        gt = torch.from_numpy(g).reshape(ctx.shape) * grad_out.to(torch.float64)
        ctx.solver.close()
        return gt, None, None, None, None, None
