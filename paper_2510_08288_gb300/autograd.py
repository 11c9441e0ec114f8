"""torch.autograd wrapper of the discrete-adjoint gradient (rrg_slack_gradient).

MinSlack.apply(kappa, x_t, theta, governor, v_prev, r, checkpoint, precision)
returns g = min over scenarios and steps of the slack (the robust objective
whose sign decides admissibility, Alg. 3) as a 0-d float64 tensor; its
backward pass returns dg/dkappa, dg/dx_t and dg/dtheta from the library's
adjoint kernels.  theta must hold the governor's own parameter vector (the
library folds it at rrg_create); it is an input only so that autograd can
route dg/dtheta.  All arithmetic runs in librrg; this module only moves
numbers between tensors and the C ABI.
"""
from __future__ import annotations

import numpy as np
import torch

from . import rrg as R


class MinSlack(torch.autograd.Function):
    @staticmethod
    def forward(ctx, kappa, x_t, theta, governor, v_prev, r, checkpoint=50, precision=R.FP64):
        p = theta.detach().cpu().double().numpy()
        if not np.array_equal(p, np.asarray(governor.params, dtype=np.float64)):
            raise ValueError("theta must equal the governor's parameter vector")
        g, grad, _, _ = governor.slack_gradient(x_t.detach().cpu().double().numpy(), float(v_prev), float(r),
                                                float(kappa.detach().cpu().item()), checkpoint, precision)
        ctx.save_for_backward(torch.as_tensor(grad, dtype=torch.float64))
        ctx.shapes = (kappa.shape, x_t.shape, theta.shape)
        ctx.devices = (kappa.device, x_t.device, theta.device)
        return torch.tensor(g, dtype=torch.float64, device=kappa.device)

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        s = gout.detach().cpu().double()
        gk = (s * grad[0]).reshape(ctx.shapes[0]).to(ctx.devices[0])
        gx = (s * grad[1:4]).reshape(ctx.shapes[1]).to(ctx.devices[1])
        gt = (s * grad[4:]).reshape(ctx.shapes[2]).to(ctx.devices[2])
        return gk, gx, gt, None, None, None, None, None


def min_slack(kappa, x_t, theta, governor, v_prev, r, checkpoint=50, precision=R.FP64):
    """Differentiable min slack g(kappa, x_t, theta) (see MinSlack)."""
    return MinSlack.apply(kappa, x_t, theta, governor, v_prev, r, checkpoint, precision)
