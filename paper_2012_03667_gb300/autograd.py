"""torch.autograd.Function wrappers of the solver (argument marshalling only).

``gap_solve(ctx, theta)``  theta: (n_inst, 3) float64 tensor of (m, D, omega) on the CPU.
    Forward: qdse_solve from A = 1, B = 0.3 (or a warm start) -> A, B (CUDA float64).
    Backward: the implicit-function adjoint qdse_adjoint (transposed fixed point at convergence;
    no unrolled iterations are kept) -> dL/dtheta.
``condensate(ctx, A, B)``  -> -<qbar q> per instance, backward by qdse_condensate_vjp.

The chiral susceptibility dC/dm then follows from ``torch.autograd.grad`` through both.
"""
from __future__ import annotations

import numpy as np
import torch

from . import qdse as Q


def _params_rows(theta: torch.Tensor) -> np.ndarray:
    t = theta.detach().cpu().double().numpy()
    # qdse_params order is (D, omega, m, mu)
    return np.stack([t[:, 1], t[:, 2], t[:, 0], np.zeros(len(t))], axis=1)


class GapSolve(torch.autograd.Function):
    @staticmethod
    def forward(fctx, theta, context: Q.Context, A0: torch.Tensor, B0: torch.Tensor):
        rows = _params_rows(theta)
        A = A0.detach().clone().contiguous()
        B = B0.detach().clone().contiguous()
        status = torch.empty(context.n_inst, dtype=torch.int32, device=A.device)
        context.qdse_solve(rows, A, B, None, status)
        fctx.context = context
        fctx.rows = rows
        fctx.status = status
        fctx.save_for_backward(A, B)
        fctx.theta_device = theta.device
        return A, B

    @staticmethod
    def backward(fctx, gA, gB):
        A, B = fctx.saved_tensors
        c = fctx.context
        gA = torch.zeros_like(A) if gA is None else gA.contiguous().double()
        gB = torch.zeros_like(B) if gB is None else gB.contiguous().double()
        gp = torch.empty(c.n_inst * 4, dtype=torch.float64, device=A.device)
        c.qdse_adjoint(fctx.rows, A, B, gA, gB, gp)
        gp = gp.view(c.n_inst, 4)
        # (m, D, omega) <- g_params columns (m, D, omega, mu)
        g_theta = gp[:, :3].to(fctx.theta_device)
        return g_theta, None, None, None


class Condensate(torch.autograd.Function):
    @staticmethod
    def forward(fctx, A, B, context: Q.Context):
        A = A.contiguous()
        B = B.contiguous()
        out = torch.empty(context.n_inst, dtype=torch.float64, device=A.device)
        context.qdse_condensate(A, B, out)
        fctx.context = context
        fctx.save_for_backward(A, B)
        return out

    @staticmethod
    def backward(fctx, cbar):
        A, B = fctx.saved_tensors
        gA = torch.zeros_like(A)
        gB = torch.zeros_like(B)
        fctx.context.qdse_condensate_vjp(A, B, cbar.contiguous().double(), gA, gB)
        return gA, gB, None


def gap_solve(context: Q.Context, theta: torch.Tensor, A0=None, B0=None):
    dev = torch.device("cuda")
    if A0 is None:
        A0 = torch.ones(context.n_total, dtype=torch.float64, device=dev)
    if B0 is None:
        B0 = torch.full((context.n_total,), 0.3, dtype=torch.float64, device=dev)
    return GapSolve.apply(theta, context, A0, B0)


def condensate(context: Q.Context, A: torch.Tensor, B: torch.Tensor) -> torch.Tensor:
    return Condensate.apply(A, B, context)
