"""torch.autograd interface to the receiver misfits (htd_grad, htd_grad_td).

``receiver_misfit(m_cell, R_node, setup, ...)`` returns J = 1/2 sum_s
||P U_s - d_s||^2 for the model m = c^-2 per cell and damping R per node; its
backward pass returns dJ/dm and dJ/dR computed by the library's adjoint-state
gradient (forward and adjoint FGMRES solves on the GPU).

``preconditioner_misfit(...)`` is the same misfit of the time-domain
preconditioner's own approximate solution (one application of Table 1 or
S_T); its backward pass runs the reverse-time adjoint of the recurrence with
checkpoints (htd_grad_td).  The recurrence parameters (omega, dt, n_P) are the
ones chosen for the model of the call and are held fixed in the derivative.

Every call builds an htd handle for the given model (the coefficients change
with m and R).
"""
from __future__ import annotations

import numpy as np
import torch

from . import htd
from . import workloads as W


class _ReceiverMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m_cell, R_node, base, F, rec_idx, d, opts):
        c = m_cell.detach().double().cpu().numpy() ** -0.5
        R = R_node.detach().double().cpu().numpy()
        prob = W.Problem(base.name, base.ndim, base.n, base.h, c, R, base.omega, base.F,
                         base.T, base.rho)
        solver = htd.Solver(prob, **opts["solver"])
        try:
            J, gm, gR, info = solver.grad(F, rec_idx, d, tol=opts["tol"],
                                          max_iters=opts["max_iters"],
                                          want_grad=ctx.needs_input_grad[0] or
                                          ctx.needs_input_grad[1])
        finally:
            solver.close()
        ctx.save_for_backward(*(t for t in (gm, gR) if t is not None))
        ctx.has_grad = gm is not None
        ctx.devices = (m_cell.device, R_node.device)
        return torch.tensor(J, dtype=torch.float64, device=m_cell.device)

    @staticmethod
    def backward(ctx, gJ):
        if not ctx.has_grad:
            return (None,) * 7
        gm, gR = ctx.saved_tensors
        scale = gJ.to(gm.device)
        return ((scale * gm).to(ctx.devices[0]), (scale * gR).to(ctx.devices[1]),
                None, None, None, None, None)


def receiver_misfit(m_cell: torch.Tensor, R_node: torch.Tensor, base: W.Problem, F: torch.Tensor,
                    rec_idx: np.ndarray, d: torch.Tensor, tol: float = 1e-10,
                    max_iters: int = 600, **solver_opts) -> torch.Tensor:
    """J(m, R) as a differentiable scalar.  base: grid, omega, T, rho of the problem;
    F: (nsrc, *n) complex128 CUDA tensor; d: (nsrc, nrec) complex128 CUDA tensor."""
    solver_opts.setdefault("precision", "mixed")
    opts = {"solver": solver_opts, "tol": tol, "max_iters": max_iters}
    return _ReceiverMisfit.apply(m_cell, R_node, base, F, rec_idx, d, opts)


class _PreconditionerMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m_cell, R_node, base, F, rec_idx, d, opts):
        c = m_cell.detach().double().cpu().numpy() ** -0.5
        R = R_node.detach().double().cpu().numpy()
        prob = W.Problem(base.name, base.ndim, base.n, base.h, c, R, base.omega, base.F,
                         base.T, base.rho)
        solver = htd.Solver(prob, **opts["solver"])
        try:
            J, gm, gR = solver.grad_td(F, rec_idx, d, checkpoint_every=opts["checkpoint_every"],
                                       want_grad=ctx.needs_input_grad[0] or
                                       ctx.needs_input_grad[1])
        finally:
            solver.close()
        ctx.save_for_backward(*(t for t in (gm, gR) if t is not None))
        ctx.has_grad = gm is not None
        ctx.devices = (m_cell.device, R_node.device)
        return torch.tensor(J, dtype=torch.float64, device=m_cell.device)

    @staticmethod
    def backward(ctx, gJ):
        if not ctx.has_grad:
            return (None,) * 7
        gm, gR = ctx.saved_tensors
        scale = gJ.to(gm.device)
        return ((scale * gm).to(ctx.devices[0]), (scale * gR).to(ctx.devices[1]),
                None, None, None, None, None)


def preconditioner_misfit(m_cell: torch.Tensor, R_node: torch.Tensor, base: W.Problem,
                          F: torch.Tensor, rec_idx: np.ndarray, d: torch.Tensor,
                          checkpoint_every: int = 0, **solver_opts) -> torch.Tensor:
    """J(m, R) = 1/2 sum_s ||P(P F_s) - d_s||^2 with P one application of the
    preconditioner (mode "table1" or "exact"), differentiable through the
    recurrence.  Arguments as in receiver_misfit."""
    solver_opts.setdefault("precision", "mixed")
    opts = {"solver": solver_opts, "checkpoint_every": checkpoint_every}
    return _PreconditionerMisfit.apply(m_cell, R_node, base, F, rec_idx, d, opts)
