"""torch.autograd.Function around the reverse-time adjoint of the fused step.

``channel_loss(q3, qwall, nu, workload, steps, ckpt_every, T_target)`` returns the
outlet-temperature loss L = mean_j (T(nx-1, j; steps) - T_target[j])^2 of a
D2Q9 MRT + D2Q5 MRT channel solve (FP64) as a 0-d tensor; ``backward`` hands out
dL/dq3 (per-cell heat source, W m^-3), dL/dqwall (y- and y+ wall heat flux per
node, W m^-2) and dL/dnu, all computed by the CUDA adjoint kernels in one forward
+ reverse sweep (``lbm_adjoint``).  Torch only carries the tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm

_TBC_FLUX = lbm.LBM_TBC_FLUX


def _solve_and_differentiate(q3, qwall, nu, workload, steps, ckpt_every, T_target):
    params = dict(workload["params"], nu=float(nu))
    s = lbm.Solver(params, precision=lbm.LBM_FP64)
    try:
        nx, ny = s.nx, s.ny
        for side, kind, uw, rw, tk, tw in workload["bcs"]:
            if side in (2, 3) and tk == _TBC_FLUX:
                tw = np.asarray(qwall[side - 2], dtype=np.float64)
            s.set_bc(side, kind, uw, rw, tk, tw)
        s.set_source(np.asarray(q3, dtype=np.float64), None)
        s.init(**(workload.get("init") or {}))
        return lbm.lbm_adjoint(s.h, steps, ckpt_every, T_target, nx, ny)
    finally:
        s.close()


class ChannelAdjointLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q3, qwall, nu, workload, steps, ckpt_every, T_target):
        loss, g3, gw, gnu = _solve_and_differentiate(
            q3.detach().cpu().numpy(), qwall.detach().cpu().numpy(), float(nu.detach().cpu()),
            workload, steps, ckpt_every, np.asarray(T_target, dtype=np.float64))
        ctx.save_for_backward(torch.from_numpy(g3).to(q3.device), torch.from_numpy(gw).to(qwall.device),
                              torch.tensor(gnu, dtype=torch.float64, device=nu.device))
        return torch.tensor(loss, dtype=torch.float64, device=q3.device)

    @staticmethod
    def backward(ctx, grad_out):
        g3, gw, gnu = ctx.saved_tensors
        return grad_out * g3, grad_out * gw, grad_out * gnu, None, None, None, None


def channel_loss(q3, qwall, nu, workload, steps, ckpt_every, T_target):
    return ChannelAdjointLoss.apply(q3, qwall, nu, workload, steps, ckpt_every, T_target)
