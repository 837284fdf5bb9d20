"""Differentiable Tucker solve (adjoint method) for PyTorch autograd.

For L(theta) = sum_t theta_t A_1^(t) x ... x A_d^(t), b = [G_b; U_b1, ..., U_bd] and a reference
tensor x_ref, `tucker_solve_mse` returns l = 0.5 ||x - x_ref||_F^2 with x the Tucker sGMRES
solution of L(x) = b.  Its backward pass solves the adjoint system L^T(mu) = x - x_ref with the
same solver (every mode matrix transposed) and forms

    dl/dtheta_t = -<mu, A_t x>,   dl/dG_b = mu x_k U_bk^T,   dl/dU_bk = mu_(k) (kron_{j!=k} U_bj) G_b(k)^T

in the CUDA library (tk_adjoint_grads).  These are the gradients of the exact solution map
b, theta -> L(theta)^{-1} b evaluated at the computed x and mu; they match finite differences of
the truncated solver to within its solve tolerance and truncation level.  The backward pass
needs only the forward solution (kept on the device) and the solver options, not the forward
Krylov basis.

The right-hand side of the adjoint solve, x - x_ref, is passed in its exact Tucker form: factors
concatenated per mode and the two cores placed on the block diagonal (copies and a sign change,
no rounding).
"""
from __future__ import annotations

import copy
from typing import Optional, Sequence

import torch

from .api import (DeviceOperator, DeviceTucker, Options, Report, fortran_empty, to_fortran,
                  tk_adjoint_grads, tk_solve, tk_sum_norm)


def tucker_difference(x: DeviceTucker, y: DeviceTucker) -> DeviceTucker:
    """Exact Tucker form of x - y: block-diagonal core, concatenated factors."""
    d = x.d
    rx, ry = x.r, y.r
    core = fortran_empty([a + b for a, b in zip(rx, ry)], x.core.device)
    core.zero_()
    core[tuple(slice(0, a) for a in rx)] = x.core
    core[tuple(slice(a, a + b) for a, b in zip(rx, ry))] = torch.neg(y.core)
    factors = [to_fortran(torch.cat([x.factors[k], y.factors[k]], dim=1), x.core.device) for k in range(d)]
    return DeviceTucker(to_fortran(core, x.core.device), factors)


class TuckerSolveMSE(torch.autograd.Function):
    @staticmethod
    def forward(ctx, op: DeviceOperator, opts: Options, x_ref: DeviceTucker, theta: torch.Tensor,
                b_core: torch.Tensor, *b_factors: torch.Tensor):
        op.set_theta(theta.detach().cpu().double().tolist())
        b = DeviceTucker(to_fortran(b_core.detach(), b_core.device),
                         [to_fortran(u.detach(), u.device) for u in b_factors])
        x, rep = tk_solve(op, b, opts)
        loss = 0.5 * tk_sum_norm([x, x_ref], [1.0, -1.0]) ** 2
        ctx.op, ctx.opts, ctx.x_ref, ctx.b, ctx.x = op, opts, x_ref, b, x
        ctx.theta = theta.detach().cpu().double().tolist()
        ctx.theta_dtype, ctx.theta_device = theta.dtype, theta.device
        ctx.forward_report = rep
        return torch.tensor(loss, dtype=torch.float64, device=b_core.device)

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        op, opts = ctx.op, ctx.opts
        op.set_theta(ctx.theta)
        g = tucker_difference(ctx.x, ctx.x_ref)
        adj = copy.copy(opts)
        adj.transpose = not opts.transpose
        mu, rep = tk_solve(op, g, adj)
        dth, dcore, dfac = tk_adjoint_grads(op, mu, ctx.x, ctx.b)
        go = float(grad_out)
        dtheta = torch.tensor(dth, dtype=ctx.theta_dtype, device=ctx.theta_device) * go
        return (None, None, None, dtheta, dcore * go, *[u * go for u in dfac])


def tucker_solve_mse(op: DeviceOperator, theta: torch.Tensor, b_core: torch.Tensor,
                     b_factors: Sequence[torch.Tensor], x_ref: DeviceTucker, opts: Options) -> torch.Tensor:
    """0.5 ||L(theta)^{-1} b - x_ref||^2 with gradients w.r.t. theta, b_core and b_factors."""
    return TuckerSolveMSE.apply(op, opts, x_ref, theta, b_core, *b_factors)
