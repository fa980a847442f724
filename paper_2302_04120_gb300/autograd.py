"""torch.autograd.Function around the reverse-time adjoint of the fused step.

``channel_loss(q3, qwall, nu, workload, steps, ckpt_every, T_target)`` returns the
outlet-temperature loss L = mean_j (T(nx-1, j; steps) - T_target[j])^2 of a
D2Q9 MRT + D2Q5 MRT channel solve (FP64) as a 0-d tensor.  ``forward`` runs the
forward solve only (``lbm_step``); ``backward`` hands out dL/dq3 (per-cell heat
source, W m^-3), dL/dqwall (y- and y+ wall heat flux per node, W m^-2) and dL/dnu,
computed by the CUDA adjoint kernels in one checkpointed forward + reverse sweep
(``lbm_adjoint``).  A forward that is never differentiated therefore costs one
solve.  Torch only carries the tensors.
"""
from __future__ import annotations

import numpy as np
import torch

from . import lbm

_TBC_FLUX = lbm.LBM_TBC_FLUX


def _solver(q3, qwall, nu, workload):
    params = dict(workload["params"], nu=float(nu))
    s = lbm.Solver(params, precision=lbm.LBM_FP64)
    for side, kind, uw, rw, tk, tw in workload["bcs"]:
        if side in (2, 3) and tk == _TBC_FLUX:
            tw = np.asarray(qwall[side - 2], dtype=np.float64)
        s.set_bc(side, kind, uw, rw, tk, tw)
    s.set_source(np.asarray(q3, dtype=np.float64), None)
    s.init(**(workload.get("init") or {}))
    return s


def _forward_loss(q3, qwall, nu, workload, steps, T_target):
    s = _solver(q3, qwall, nu, workload)
    try:
        s.step(steps)
        T_out = s.moments(lbm.LBM_T)["T"][:, -1]
        return float(np.mean((T_out - T_target) ** 2))
    finally:
        s.close()


def _solve_and_differentiate(q3, qwall, nu, workload, steps, ckpt_every, T_target):
    s = _solver(q3, qwall, nu, workload)
    try:
        return lbm.lbm_adjoint(s.h, steps, ckpt_every, T_target, s.nx, s.ny)
    finally:
        s.close()


def _host(t):
    return t.detach().cpu().numpy()


class ChannelAdjointLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, q3, qwall, nu, workload, steps, ckpt_every, T_target):
        T_target = np.asarray(T_target, dtype=np.float64)
        loss = _forward_loss(_host(q3), _host(qwall), float(nu.detach().cpu()), workload, steps, T_target)
        ctx.save_for_backward(q3.detach(), qwall.detach(), nu.detach())
        ctx.args = (workload, steps, ckpt_every, T_target)
        return torch.tensor(loss, dtype=torch.float64, device=q3.device)

    @staticmethod
    def backward(ctx, grad_out):
        q3, qwall, nu = ctx.saved_tensors
        workload, steps, ckpt_every, T_target = ctx.args
        _, g3, gw, gnu = _solve_and_differentiate(_host(q3), _host(qwall), float(nu.cpu()), workload, steps,
                                                  ckpt_every, T_target)
        g3 = torch.from_numpy(g3).to(q3.device)
        gw = torch.from_numpy(gw).to(qwall.device)
        gnu = torch.tensor(gnu, dtype=torch.float64, device=nu.device)
        return grad_out * g3, grad_out * gw, grad_out * gnu, None, None, None, None


def channel_loss(q3, qwall, nu, workload, steps, ckpt_every, T_target):
    return ChannelAdjointLoss.apply(q3, qwall, nu, workload, steps, ckpt_every, T_target)
