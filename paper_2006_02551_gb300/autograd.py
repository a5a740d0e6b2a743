"""PyTorch autograd entry for the probe objective.

``probe_objective(solver, eps_r, sigma_max, p_sigma, ...)`` returns
J = sum over steps and probes of |E(x_p)|^2 (excitation 0) as a tensor whose
gradient with respect to the per-element relative permittivity ``eps_r`` and
the PML profile scalars ``sigma_max`` and ``p_sigma`` (shared by the three
axes) comes from the library's discrete adjoint (``wadg_adjoint``): the forward
call runs the forward pass with checkpoints and the reverse pass at once and
keeps the gradients for ``backward``.
"""
from __future__ import annotations

from dataclasses import replace

import numpy as np
import torch


class _ProbeObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, eps_r, sigma_max, p_sigma, solver, profile, nsteps, dt, ckpt_every):
        solver.set_materials(eps_r.detach().cpu().double().numpy())
        prof = replace(profile, sigma_max=float(sigma_max), p_sigma=float(p_sigma))
        solver.set_pml(prof)
        solver.set_state(None, 0.0)
        J, ge, gs, gp = solver.adjoint(nsteps, dt, ckpt_every)
        ctx.save_for_backward(torch.from_numpy(ge[0].copy()).to(eps_r.dtype),
                              torch.tensor(gs[0].sum(), dtype=torch.float64),
                              torch.tensor(gp[0].sum(), dtype=torch.float64))
        return torch.tensor(J[0], dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        ge, gs, gp = ctx.saved_tensors
        return gJ * ge, gJ * gs, gJ * gp, None, None, None, None, None


def probe_objective(solver, eps_r, sigma_max, p_sigma, profile, nsteps, dt, ckpt_every=45):
    """Differentiable J(eps_r, sigma_max, p_sigma) for an already configured
    solver (mesh, sources, probes); the remaining profile fields come from
    ``profile`` (a synthetic.PmlProfile-like record)."""
    return _ProbeObjective.apply(eps_r, sigma_max, p_sigma, solver, profile, nsteps, dt,
                                 ckpt_every)
