"""Differentiation through def-CG solves of the matrix-free RBF operator.

The paper recycles Krylov subspaces across a sequence of systems, motivated by
hyperparameter search (Sec. 1), with the RBF kernel of Sec. 3. This module
makes that sequence differentiable:

* ``DefCGSolve``: ``x = A(theta)^{-1} b`` by def-CG (Algorithm 1). Its
  backward runs the adjoint solve ``A lambda = dL/dx`` (A is symmetric) with
  the same recycled W, then ``dL/dtheta = -lambda^T (dA/dtheta) x`` through the
  derivative-form kernel (``dcg_rbf_dtheta``), and ``dL/db = lambda``.
* ``LogDetProbes``: value 0; its gradient is the Hutchinson estimate of
  ``1/2 d log det A / dtheta = 1/2 tr(A^{-1} dA/dtheta)`` from Rademacher
  probes ``z_p`` solved by def-CG, ``1/2 mean_p (A^{-1} z_p)^T (dA/dtheta) z_p``.
* ``gp_objective``: ``1/2 y^T A^{-1} y`` plus the probe term, i.e. a value
  equal to the data-fit term and a gradient equal to the (probe-estimated)
  gradient of the GP negative log marginal likelihood.
* ``fit_gp``: Adam on log-hyperparameters with that gradient.

theta = (lengthscale, signal_var, noise) as a float64 tensor of shape (3,).
Every solve and every derivative form runs in the library's kernels.
"""

from __future__ import annotations

import numpy as np
import torch

from ._lib import DCG_MAX_RHS
from .solver import DefCG


def _params(theta: torch.Tensor):
    l, s2, noise = (float(v) for v in theta.detach().to(torch.float64).cpu())
    return l, s2, noise


class DefCGSolve(torch.autograd.Function):
    """x = A(theta)^{-1} b through ``solver`` (a DefCG with a matrix-free
    operator set). With ``recycle`` the harmonic-Ritz update follows the
    forward solve, so the adjoint solve and later systems deflate with W
    extracted under this A."""

    @staticmethod
    def forward(ctx, theta, b, solver: DefCG, recycle: bool = True):
        params = _params(theta)
        solver.set_rbf_params(*params)
        x, info = solver.solve(b.detach().to(torch.float32).contiguous())
        if recycle:
            solver.update_subspace()
        solver.last_forward_info = info
        ctx.solver = solver
        ctx.params = params
        ctx.theta_dtype, ctx.theta_device = theta.dtype, theta.device
        ctx.b_dtype = b.dtype
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        solver = ctx.solver
        solver.set_rbf_params(*ctx.params)
        lam, info = solver.solve(gx.detach().to(torch.float32).contiguous())
        solver.last_adjoint_info = info
        forms = solver.rbf_dtheta(lam.to(torch.float32)[None].contiguous(), x.to(torch.float32)[None].contiguous())
        gtheta = torch.tensor(-forms[0], dtype=ctx.theta_dtype, device=ctx.theta_device)
        gb = lam.to(ctx.b_dtype) if ctx.needs_input_grad[1] else None
        return gtheta, gb, None, None


class LogDetProbes(torch.autograd.Function):
    """Value 0 (log det A is not evaluated); gradient 1/2 mean_p u_p^T
    (dA/dtheta) z_p with A u_p = z_p solved by def-CG. Z: (P, n) float32
    probes on the device (rows are probes). With ``block`` the probes are
    solved in lockstep (dcg_solve_multi, up to DCG_MAX_RHS at a time), each
    operator pass serving all of them; otherwise one after another."""

    @staticmethod
    def forward(ctx, theta, solver: DefCG, Z, block: bool = True):
        params = _params(theta)
        solver.set_rbf_params(*params)
        U = torch.empty_like(Z, dtype=torch.float32)
        infos = []
        if block:
            for c0 in range(0, Z.shape[0], DCG_MAX_RHS):
                Uc, inf = solver.solve_multi(Z[c0:c0 + DCG_MAX_RHS].contiguous())
                U[c0:c0 + Uc.shape[0]] = Uc.to(torch.float32)
                infos += inf
        else:
            for p in range(Z.shape[0]):
                u, info = solver.solve(Z[p].contiguous())
                U[p] = u.to(torch.float32)
                infos.append(info)
        solver.last_probe_infos = infos
        ctx.solver = solver
        ctx.params = params
        ctx.theta_dtype, ctx.theta_device = theta.dtype, theta.device
        ctx.save_for_backward(U, Z)
        return theta.new_zeros(())

    @staticmethod
    def backward(ctx, g):
        U, Z = ctx.saved_tensors
        solver = ctx.solver
        solver.set_rbf_params(*ctx.params)
        forms = solver.rbf_dtheta(U.contiguous(), Z.to(torch.float32).contiguous())
        grad = 0.5 * forms.mean(axis=0)
        return g * torch.tensor(grad, dtype=ctx.theta_dtype, device=ctx.theta_device), None, None, None


def gp_objective(theta: torch.Tensor, y: torch.Tensor, solver: DefCG, Z: torch.Tensor | None = None,
                 recycle: bool = True, block_probes: bool = True) -> torch.Tensor:
    """1/2 y^T A(theta)^{-1} y (+ LogDetProbes when probes Z are given)."""
    x = DefCGSolve.apply(theta, y, solver, recycle)
    fit = 0.5 * torch.dot(y.detach().to(torch.float64), x)
    if Z is None:
        return fit
    return fit + LogDetProbes.apply(theta, solver, Z, block_probes).to(fit.device)


def rademacher_probes(n: int, count: int, seed: int, device="cuda") -> torch.Tensor:
    """(count, n) float32 Rademacher probes from a seeded torch generator."""
    g = torch.Generator(device="cpu")
    g.manual_seed(int(seed))
    z = torch.randint(0, 2, (count, n), generator=g, dtype=torch.int8).to(torch.float32) * 2.0 - 1.0
    return z.to(device)


def fit_gp(solver: DefCG, y: torch.Tensor, theta0, steps: int = 30, lr: float = 0.05, probes=16,
           probe_seed: int = 1000, block_probes: bool = True):
    """Adam on phi = log(theta) with the gp_objective gradient.

    ``probes`` is a probe count (Rademacher rows from ``rademacher_probes``
    with seed probe_seed + step) or a callable step -> (P, n) tensor;
    ``block_probes`` solves them in lockstep (see LogDetProbes). Returns
    (list of theta after each step, list of dL/dtheta per step).
    """
    phi = torch.tensor(np.log(np.asarray(theta0, dtype=np.float64)), dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([phi], lr=lr)
    path, grads = [np.exp(phi.detach().numpy()).copy()], []
    for step in range(steps):
        if callable(probes):
            Z = probes(step)
        elif probes:
            Z = rademacher_probes(solver.n, probes, probe_seed + step, device=y.device)
        else:
            Z = None
        opt.zero_grad()
        theta = phi.exp()
        loss = gp_objective(theta, y, solver, Z, block_probes=block_probes)
        loss.backward()
        grads.append((phi.grad.detach().numpy() / np.exp(phi.detach().numpy())).copy())
        opt.step()
        path.append(np.exp(phi.detach().numpy()).copy())
    return path, grads
