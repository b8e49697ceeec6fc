"""Differentiable corrector solves (adjoint backward).

``CorrectorSolve`` wraps one CP2 solve x = A(theta)^-1 b, with theta the
per-cell log-permeability (K = exp(theta) I).  Its backward is the adjoint
solve lambda = A^-1 dL/dx on the same assembled system (A is symmetric),
followed by the library's per-side scatter dL/dT = -(lambda_e - lambda_ep)
(x_e - x_ep) chained to dL/dtheta; dL/db = lambda.  All of it runs in
``cps_adjoint``.

``chained_solve`` runs T solves with b_t = rhs_t + c * x_{t-1} and
checkpoints every ``checkpoint_every`` steps: only the segment inputs are
kept, and the backward pass re-runs each segment's forward solves before its
adjoint solves.
"""
from __future__ import annotations

import torch
import torch.utils.checkpoint

from . import _cps
from .api import Context, System


class LogPermeabilityCorrector:
    """CP2 operator on a fixed mesh, parametrised by the cell log-permeability.

    The system is assembled on the device for the theta it is given and kept
    until theta changes (assembly and factorisation once per parameter value,
    as the scheme assembles once per time loop)."""

    def __init__(self, ctx: Context, xy, tri, dirichlet, eps, nu: float = 1.5e-5,
                 dt: float = 0.225, rtol: float = 1e-12):
        self.ctx = ctx
        self.xy = ctx.dev(xy, torch.float64)
        self.tri = ctx.dev(tri, torch.int32)
        self.dirichlet = ctx.dev(dirichlet, torch.int32)
        self.eps = ctx.dev(eps, torch.float64)
        self.nu, self.dt, self.rtol = nu, dt, rtol
        self._theta = None
        self._sys: System | None = None

    def system(self, theta: torch.Tensor) -> System:
        th = theta.detach()
        if self._sys is None or self._theta is None or not torch.equal(th, self._theta):
            if self._sys is not None:
                self._sys.free()
            self._sys = self.ctx.assemble(self.xy, self.tri, self.dirichlet, self.eps,
                                          th.contiguous(), _cps.PER_CELL_LOGK, _cps.KIND_CP2,
                                          self.nu, self.dt)
            self._theta = th.clone()
        return self._sys

    def solve(self, theta: torch.Tensor, b: torch.Tensor) -> torch.Tensor:
        return CorrectorSolve.apply(theta, b, self)

    def free(self):
        if self._sys is not None:
            self._sys.free()
            self._sys = None


class CorrectorSolve(torch.autograd.Function):
    """x = A(theta)^-1 b with an adjoint backward."""

    @staticmethod
    def forward(ctx, theta, b, model: LogPermeabilityCorrector):
        sys_ = model.system(theta)
        x, _ = sys_.solve(b.detach().contiguous(), rtol=model.rtol)
        ctx.save_for_backward(theta, x)
        ctx.model = model
        return x

    @staticmethod
    def backward(ctx, g):
        theta, x = ctx.saved_tensors
        sys_ = ctx.model.system(theta)
        dtheta = torch.zeros_like(x) if ctx.needs_input_grad[0] else None
        lam, _ = sys_.adjoint(x, g.contiguous(), dtheta=dtheta, rtol=ctx.model.rtol)
        return dtheta, (lam if ctx.needs_input_grad[1] else None), None


def chained_solve(model: LogPermeabilityCorrector, theta: torch.Tensor, rhs,
                  coupling: float = 0.1, checkpoint_every: int = 10, normalized: bool = False):
    """x_t = A(theta)^-1 (rhs[t] + coupling * f(x_{t-1})), x_0 = 0 before the
    first step; returns the list of x_t.  f(x) = x, or with normalized=True
    f(x) = x * |rhs[t]| / |x| (the previous solution rescaled to the norm of
    the new data, which keeps long chains bounded: with f(x) = x the feedback
    grows by coupling / lambda_min(A) per step).  With checkpoint_every > 0
    the autograd graph keeps only every segment's input state."""
    steps = len(rhs)
    x_prev = torch.zeros_like(rhs[0])
    xs = []

    def feed(b, xp):
        if not normalized:
            return b + coupling * xp
        nx = torch.linalg.vector_norm(xp)
        if float(nx.detach()) == 0.0:
            return b.clone()
        return b + coupling * (torch.linalg.vector_norm(b) / nx) * xp

    def segment(th, xp, *bs):
        out = []
        for b in bs:
            xp = CorrectorSolve.apply(th, feed(b, xp), model)
            out.append(xp)
        return tuple(out)

    k = checkpoint_every if checkpoint_every > 0 else steps
    for s0 in range(0, steps, k):
        bs = rhs[s0:s0 + k]
        if checkpoint_every > 0 and torch.is_grad_enabled():
            out = torch.utils.checkpoint.checkpoint(segment, theta, x_prev, *bs,
                                                    use_reentrant=False)
        else:
            out = segment(theta, x_prev, *bs)
        xs.extend(out)
        x_prev = out[-1]
    return xs
